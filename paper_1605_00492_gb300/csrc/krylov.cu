// FP64 vector kernels of the outer Krylov solve (Sec. 5) on the finest level,
// tiled layout, and the COLUMN <-> TILED layout conversions.  Every kernel
// that needs a global dot product folds it into the same pass (deterministic
// grid reduction, reduce.cuh) and forms the Krylov scalar on the device.
#include "convert.cuh"
#include "hmg_internal.h"
#include "reduce.cuh"

namespace hmg {

namespace {

// COLUMN <-> TILED.  The 32 columns of a tile are one contiguous block in
// both layouts (columns c0..c0+31 x nzc values in the COLUMN layout, rows
// 0..nz-1 x 32 lanes in the TILED one), so each CTA transposes one tile
// through shared memory and both sides move in whole 128/256-byte rows.
// nzc <= nz values per column (the vertical-face vectors of the
// velocity-pressure system have nz - 1; the tiled rows beyond nzc are zero).
template <typename T>
__global__ void k_transpose(bool to_tiled, int nitems, int nz, int nzc, int ntiles, const T* __restrict__ src,
                            T* __restrict__ dst) {
  extern __shared__ __align__(16) unsigned char tsm_raw[];
  T* sm = reinterpret_cast<T*>(tsm_raw);   // [nz][33]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int c0 = tile * TW;
    const int64_t tb0 = (int64_t)tile * TW * nz, cb0 = (int64_t)c0 * nzc;
    __syncthreads();
    if (to_tiled) {
      for (int j = warp; j < TW; j += nw)
        for (int l = lane; l < nz; l += 32)
          sm[l * 33 + j] = (c0 + j < nitems && l < nzc) ? src[cb0 + (int64_t)j * nzc + l] : (T)0;
      __syncthreads();
      for (int l = warp; l < nz; l += nw) dst[tb0 + (int64_t)l * TW + lane] = sm[l * 33 + lane];
    } else {
      for (int l = warp; l < nz; l += nw) sm[l * 33 + lane] = src[tb0 + (int64_t)l * TW + lane];
      __syncthreads();
      for (int j = warp; j < TW; j += nw)
        if (c0 + j < nitems)
          for (int l = lane; l < nzc; l += 32) dst[cb0 + (int64_t)j * nzc + l] = sm[l * 33 + j];
    }
  }
}

// The vector kernels below read and write two elements per access (16-byte
// loads and stores; n is even for every tiled vector, since the padded column
// count is a multiple of 32, and an odd last element is handled by thread 0).
// k_dot and k_update_p cover 4 elements per thread and grid-stride step (two
// independent 16-byte loads per operand in flight); k_update_xr, with four
// operands, covers 2 (two elements per step measured faster there: 51.8
// against 53.9 us at 5.2 M cells, while k_update_p went 22.5 -> 20.6 us).

inline __device__ int64_t gtid() { return blockIdx.x * (int64_t)blockDim.x + threadIdx.x; }
inline __device__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

#define HMG_V2(p) reinterpret_cast<const double2*>(p)
#define HMG_W2(p) reinterpret_cast<double2*>(p)

// s0 = a.b, s1 = c.d (NV = 2)
template <int NV>
__global__ void k_dot(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                      const double* __restrict__ c, const double* __restrict__ d, Reduce red) {
  double s0 = 0.0, s1 = 0.0, t0 = 0.0, t1 = 0.0;
  const int64_t n2 = n >> 1, st = gstride();
  int64_t i = gtid();
  for (; i + st < n2; i += 2 * st) {
    const double2 a0 = HMG_V2(a)[i], b0 = HMG_V2(b)[i], a1 = HMG_V2(a)[i + st], b1 = HMG_V2(b)[i + st];
    double2 c0, d0, c1, d1;
    if (NV == 2) {
      c0 = HMG_V2(c)[i];
      d0 = HMG_V2(d)[i];
      c1 = HMG_V2(c)[i + st];
      d1 = HMG_V2(d)[i + st];
    }
    s0 = fma(a0.x, b0.x, s0);
    t0 = fma(a0.y, b0.y, t0);
    s0 = fma(a1.x, b1.x, s0);
    t0 = fma(a1.y, b1.y, t0);
    if (NV == 2) {
      s1 = fma(c0.x, d0.x, s1);
      t1 = fma(c0.y, d0.y, t1);
      s1 = fma(c1.x, d1.x, s1);
      t1 = fma(c1.y, d1.y, t1);
    }
  }
  if (i < n2) {
    const double2 a0 = HMG_V2(a)[i], b0 = HMG_V2(b)[i];
    s0 = fma(a0.x, b0.x, s0);
    t0 = fma(a0.y, b0.y, t0);
    if (NV == 2) {
      const double2 c0 = HMG_V2(c)[i], d0 = HMG_V2(d)[i];
      s1 = fma(c0.x, d0.x, s1);
      t1 = fma(c0.y, d0.y, t1);
    }
  }
  if ((n & 1) && gtid() == 0) {
    s0 = fma(a[n - 1], b[n - 1], s0);
    if (NV == 2) s1 = fma(c[n - 1], d[n - 1], s1);
  }
  HMG_RED_SCRATCH(scratch);
  grid_reduce<NV>(s0 + t0, s1 + t1, red, scratch);
}

// x += alpha p; r -= alpha q; s0 = r.r
__global__ void k_update_xr(int64_t n, double* __restrict__ x, double* __restrict__ r,
                            const double* __restrict__ p, const double* __restrict__ q, Reduce red) {
  const double alpha = red.sc[S_ALPHA];
  double s0 = 0.0, t0 = 0.0;
  const int64_t n2 = n >> 1;
  for (int64_t i = gtid(); i < n2; i += gstride()) {
    double2 xi = HMG_V2(x)[i], ri = HMG_V2(r)[i];
    const double2 pi = HMG_V2(p)[i], qi = HMG_V2(q)[i];
    xi.x = fma(alpha, pi.x, xi.x);
    xi.y = fma(alpha, pi.y, xi.y);
    ri.x = fma(-alpha, qi.x, ri.x);
    ri.y = fma(-alpha, qi.y, ri.y);
    HMG_W2(x)[i] = xi;
    HMG_W2(r)[i] = ri;
    s0 = fma(ri.x, ri.x, s0);
    t0 = fma(ri.y, ri.y, t0);
  }
  if ((n & 1) && gtid() == 0) {
    x[n - 1] = fma(alpha, p[n - 1], x[n - 1]);
    const double rl = fma(-alpha, q[n - 1], r[n - 1]);
    r[n - 1] = rl;
    s0 = fma(rl, rl, s0);
  }
  HMG_RED_SCRATCH(scratch);
  grid_reduce<1>(s0 + t0, 0.0, red, scratch);
}

// p = z + beta p
__global__ void k_update_p(int64_t n, double* __restrict__ p, const double* __restrict__ z,
                           const double* __restrict__ sc) {
  const double beta = sc[S_BETA];
  const int64_t n2 = n >> 1, st = gstride();
  int64_t i = gtid();
  for (; i + st < n2; i += 2 * st) {
    double2 p0 = HMG_V2(p)[i], p1 = HMG_V2(p)[i + st];
    const double2 z0 = HMG_V2(z)[i], z1 = HMG_V2(z)[i + st];
    p0.x = fma(beta, p0.x, z0.x);
    p0.y = fma(beta, p0.y, z0.y);
    p1.x = fma(beta, p1.x, z1.x);
    p1.y = fma(beta, p1.y, z1.y);
    HMG_W2(p)[i] = p0;
    HMG_W2(p)[i + st] = p1;
  }
  if (i < n2) {
    double2 pi = HMG_V2(p)[i];
    const double2 zi = HMG_V2(z)[i];
    pi.x = fma(beta, pi.x, zi.x);
    pi.y = fma(beta, pi.y, zi.y);
    HMG_W2(p)[i] = pi;
  }
  if ((n & 1) && gtid() == 0) p[n - 1] = fma(beta, p[n - 1], z[n - 1]);
}

// s0 = |b - q|^2
__global__ void k_resid_sq(int64_t n, const double* __restrict__ b, const double* __restrict__ q,
                           Reduce red) {
  double s0 = 0.0;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    double v = b[i] - q[i];
    s0 += v * v;
  }
  HMG_RED_SCRATCH(scratch);
  grid_reduce<1>(s0, 0.0, red, scratch);
}

__global__ void k_f64_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = f64_to_f32(a[i]);
}

__global__ void k_f32_to_f64(int64_t n, const float* __restrict__ a, double* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = f32_to_f64(a[i]);
}


}  // namespace

void launch_convert(int64_t n, const void* src, int src_dt, void* dst, cudaStream_t s) {
  const int g = reduce_grid(n);
  if (src_dt == HMG_FP64) k_f64_to_f32<<<g, 256, 0, s>>>(n, (const double*)src, (float*)dst);
  else k_f32_to_f64<<<g, 256, 0, s>>>(n, (const float*)src, (double*)dst);
}

int reduce_grid(int64_t n) {
  int64_t b = (n + 255) / 256;
  int cap = 152 * 8;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

template <typename T>
void transpose(bool to_tiled, int nitems, int nz, int nzc, const void* src, void* dst, cudaStream_t s) {
  const int ntiles = (nitems + TW - 1) / TW;
  const int g = ntiles < 152 * 8 ? ntiles : 152 * 8;
  const size_t smem = (size_t)nz * 33 * sizeof(T);
  static SmemOptIn opt_in;
  allow_smem(k_transpose<T>, smem, opt_in);
  k_transpose<T><<<g, 256, smem, s>>>(to_tiled, nitems, nz, nzc, ntiles, (const T*)src, (T*)dst);
}

void launch_to_tiled(const Level& L, int dt, const void* col, void* tiled, cudaStream_t s) {
  if (dt == HMG_FP64) transpose<double>(true, L.nc, L.nz, L.nz, col, tiled, s);
  else transpose<float>(true, L.nc, L.nz, L.nz, col, tiled, s);
}

void launch_to_column(const Level& L, int dt, const void* tiled, void* col, cudaStream_t s) {
  if (dt == HMG_FP64) transpose<double>(false, L.nc, L.nz, L.nz, tiled, col, s);
  else transpose<float>(false, L.nc, L.nz, L.nz, tiled, col, s);
}

void launch_transpose64(bool to_tiled, int nitems, int nz, int nzc, const double* src, double* dst, cudaStream_t s) {
  transpose<double>(to_tiled, nitems, nz, nzc, src, dst, s);
}

void launch_dot(const Level& L, const double* a, const double* b, const double* c, const double* d,
                const Reduce& red, cudaStream_t s) {
  if (c) k_dot<2><<<reduce_grid(L.Np), 256, 0, s>>>(L.Np, a, b, c, d, red);
  else k_dot<1><<<reduce_grid(L.Np), 256, 0, s>>>(L.Np, a, b, c, d, red);
}

void launch_update_xr(const Level& L, double* x, double* r, const double* p, const double* q,
                      const Reduce& red, cudaStream_t s) {
  k_update_xr<<<reduce_grid(L.Np), 256, 0, s>>>(L.Np, x, r, p, q, red);
}

void launch_update_p(const Level& L, double* p, const double* z, const double* sc, cudaStream_t s) {
  k_update_p<<<reduce_grid(L.Np), 256, 0, s>>>(L.Np, p, z, sc);
}

void launch_resid_sq(const Level& L, const double* b, const double* q, const Reduce& red, cudaStream_t s) {
  k_resid_sq<<<reduce_grid(L.Np), 256, 0, s>>>(L.Np, b, q, red);
}

void launch_check_finite(const Level& L, const double* v, const Reduce& red, cudaStream_t s) {
  k_dot<1><<<reduce_grid(L.Np), 256, 0, s>>>(L.Np, v, v, nullptr, nullptr, red);
}

// Stopping test of the device-side CG loop (the body of a CUDA-graph while
// node).  It runs after the update of x and r of iteration k = loop->k, once,
// on one thread: it stores ||r_k|| / ||b|| in the history and ends the loop
// (condition 0) on a non-finite value or a breakdown flag, on
// ||r_k||^2 < rtol^2 ||b||^2, or at k = max_iter; otherwise it advances k.
// The same test, in the same FP64 operations, as the host-side loop.
__global__ void k_cg_control(CgLoop* loop, const double* __restrict__ sc, cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int k = loop->k;
  const double rr = sc[S_RR], bb = sc[S_BB];
  const int flag = (int)sc[S_FLAG];
  if (k >= 1 && k <= CG_LOOP_HIST) loop->hist[k - 1] = sqrt(rr / bb);
  const bool stop = (flag & (F_NONFINITE | F_BREAKDOWN)) || rr < loop->rtol2 * bb || k >= loop->max_iter ||
                    k >= CG_LOOP_HIST;
  loop->rr = rr;
  loop->flag = flag;
  if (!stop) loop->k = k + 1;
  cudaGraphSetConditional(h, stop ? 0u : 1u);
}

__global__ void k_cg_loop_init(CgLoop* loop, double rtol2, int max_iter) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  loop->rtol2 = rtol2;
  loop->max_iter = max_iter;
  loop->k = 1;
}

void launch_cg_control(CgLoop* loop, const double* sc, cudaGraphConditionalHandle h, cudaStream_t s) {
  k_cg_control<<<1, 32, 0, s>>>(loop, sc, h);
}

void launch_cg_loop_init(CgLoop* loop, double rtol2, int max_iter, cudaStream_t s) {
  k_cg_loop_init<<<1, 32, 0, s>>>(loop, rtol2, max_iter);
}

// Throughput probe of the FP64 FMA pipe (the bound of the FP64 cycle): every
// thread advances 8 independent FMA chains, so each warp always has an FP64
// instruction ready.  The result is stored only if it is not finite, which it
// never is for these inputs; the test keeps the chains live.
__global__ void k_fp64_fma_probe(int iters, double* __restrict__ sink) {
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1.0 + 1e-3 * k + 1e-9 * threadIdx.x;
  const double m = 0.9999999, c = 1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
  }
  double t = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) t += a[k];
  if (!isfinite(t)) sink[0] = t;
}

double measure_fp64_fma_rate(double* sink, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = 8 * (sms > 0 ? sms : 152), threads = 256, iters = 4096;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fp64_fma_probe<<<blocks, threads, 0, s>>>(64, sink);   // warm-up
  cudaEventRecord(e0, s);
  k_fp64_fma_probe<<<blocks, threads, 0, s>>>(iters, sink);
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
  return ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
}

}  // namespace hmg
