// FP64 vector kernels of the outer Krylov solve (Sec. 5) on the finest level,
// tiled layout, and the COLUMN <-> TILED layout conversions.  Every kernel
// that needs a global dot product folds it into the same pass (deterministic
// grid reduction, reduce.cuh) and forms the Krylov scalar on the device.
#include "convert.cuh"
#include "hmg_internal.h"
#include "reduce.cuh"

namespace hmg {

namespace {

__device__ __forceinline__ bool decode(int64_t t, int nz, int nc, int& c, int& l) {
  int lane = (int)(t & 31);
  int64_t tile = t / (TW * nz);
  l = (int)((t >> 5) % nz);
  c = (int)(tile * TW + lane);
  return c < nc;
}

template <typename T>
__global__ void k_to_tiled(int nc, int nz, int64_t Np, const T* __restrict__ col, T* __restrict__ tiled) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= Np) return;
  int c, l;
  tiled[t] = decode(t, nz, nc, c, l) ? col[(int64_t)c * nz + l] : (T)0;
}

template <typename T>
__global__ void k_to_column(int nc, int nz, int64_t Np, const T* __restrict__ tiled, T* __restrict__ col) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= Np) return;
  int c, l;
  if (decode(t, nz, nc, c, l)) col[(int64_t)c * nz + l] = tiled[t];
}

// The vector kernels below read and write two elements per access (16-byte
// loads and stores; n is even for every tiled vector, since the padded column
// count is a multiple of 32, and an odd last element is handled by thread 0).
// Each grid-stride step covers 4 elements per thread, so that 4 independent
// 16-byte loads per operand are in flight.

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
  const int64_t n2 = n >> 1;
  for (int64_t i = gtid(); i < n2; i += gstride()) {
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

inline unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

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

void launch_to_tiled(const Level& L, int dt, const void* col, void* tiled, cudaStream_t s) {
  if (dt == HMG_FP64)
    k_to_tiled<double><<<blocks_for(L.Np, 256), 256, 0, s>>>(L.nc, L.nz, L.Np, (const double*)col, (double*)tiled);
  else
    k_to_tiled<float><<<blocks_for(L.Np, 256), 256, 0, s>>>(L.nc, L.nz, L.Np, (const float*)col, (float*)tiled);
}

void launch_to_column(const Level& L, int dt, const void* tiled, void* col, cudaStream_t s) {
  if (dt == HMG_FP64)
    k_to_column<double><<<blocks_for(L.Np, 256), 256, 0, s>>>(L.nc, L.nz, L.Np, (const double*)tiled, (double*)col);
  else
    k_to_column<float><<<blocks_for(L.Np, 256), 256, 0, s>>>(L.nc, L.nz, L.Np, (const float*)tiled, (float*)col);
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

}  // namespace hmg
