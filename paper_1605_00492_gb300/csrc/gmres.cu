// Vector kernels of the restarted flexible GMRES(m) outer solve (Sec. 5 wraps
// the multigrid preconditioner in GMRES(30); flexible form: Saad, Iterative
// Methods for Sparse Linear Systems, Algorithm 9.6).  The Arnoldi vector
// w = A z_j is orthogonalised against v_0..v_j by classical Gram-Schmidt,
// once (the default of the PETSc GMRES the paper used) or twice, in three
// passes over the basis:
//
//   k_gs_dots    h   = V^T w
//   k_gs_update  w  -= V h;        |w|^2 (and, applied twice, h2 = V^T w) from the same pass
//   k_gs_final   (twice: w -= V h2;)  v_(j+1) = w / h_(j+1,j)
//
// where h_(j+1,j)^2 = |w|^2 - |h2|^2 (Pythagoras: w after the second
// projection is orthogonal to the basis to rounding; |w|^2 once).  Every dot product is
// a deterministic two-level reduction (fixed order within and across blocks)
// whose last block writes the results.  Vectors are the finest level's tiled
// FP64 vectors; the basis vectors are contiguous, vector i at V + i * ld.
#include "hmg_internal.h"
#include "reduce.cuh"

namespace hmg {

namespace {

constexpr int GS_THREADS = 128;
constexpr int GS_WARPS = GS_THREADS / 32;

// Sum per-thread values over the grid: acc[v] for v < nv into out[v] and,
// with `extra`, acc[MAXV] into out[nv].  Block partials go to
// part[v * gridDim.x + block]; the last block to finish adds them in block
// order (warp w takes the outputs v = w, w + GS_WARPS, ...).
template <int MAXV>
__device__ __forceinline__ void multi_reduce(const double (&acc)[MAXV + 1], int nv, bool extra,
                                             double* __restrict__ part, unsigned* counter,
                                             double* __restrict__ out) {
  __shared__ double sm[GS_WARPS][MAXV + 1];
  __shared__ bool is_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nout = nv + (extra ? 1 : 0);
#pragma unroll
  for (int v = 0; v <= MAXV; ++v) {
    if (v < nv || (extra && v == MAXV)) {
      double a = acc[v];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
      if (lane == 0) sm[warp][v == MAXV ? nv : v] = a;
    }
  }
  __syncthreads();
  if (threadIdx.x < nout) {
    double a = sm[0][threadIdx.x];
#pragma unroll
    for (int w = 1; w < GS_WARPS; ++w) a += sm[w][threadIdx.x];
    part[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = a;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  for (int v = warp; v < nout; v += GS_WARPS) {
    double a = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) a += __ldcg(part + (int64_t)v * gridDim.x + b);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
    if (lane == 0) out[v] = a;
  }
  if (threadIdx.x == 0) {
    *counter = 0u;
    __threadfence();
  }
}

// Each thread takes U elements per grid-stride step (elements e0 + u * stride),
// so that U independent loads per vector are in flight: with one element per
// step the passes are bound by memory latency, not bandwidth.
__host__ __device__ constexpr int gs_unroll(int maxv) { return maxv <= 8 ? 4 : (maxv <= 16 ? 2 : 1); }

// out[i] = v_i . w, i < nv
template <int MAXV>
__global__ void __launch_bounds__(GS_THREADS)
k_gs_dots(int64_t n, const double* __restrict__ V, int64_t ld, int nv, const double* __restrict__ w,
          double* part, unsigned* counter, double* out) {
  constexpr int U = gs_unroll(MAXV);
  double acc[MAXV + 1];
#pragma unroll
  for (int v = 0; v <= MAXV; ++v) acc[v] = 0.0;
  const int64_t stride = (int64_t)gridDim.x * GS_THREADS;
  for (int64_t e0 = blockIdx.x * (int64_t)GS_THREADS + threadIdx.x; e0 < n; e0 += stride * U) {
    double we[U];
#pragma unroll
    for (int u = 0; u < U; ++u) we[u] = (e0 + u * stride < n) ? w[e0 + u * stride] : 0.0;
#pragma unroll
    for (int v = 0; v < MAXV; ++v)
      if (v < nv) {
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (e0 + u * stride < n) acc[v] = fma(V[v * ld + e0 + u * stride], we[u], acc[v]);
      }
  }
  multi_reduce<MAXV>(acc, nv, false, part, counter, out);
}

// w -= sum_i h[i] v_i; out[i] = v_i . w (i < nd2: the second pass of the
// twice-applied form, nd2 = nv; 0 for the single pass), out[nd2] = w . w
template <int MAXV>
__global__ void __launch_bounds__(GS_THREADS)
k_gs_update(int64_t n, const double* __restrict__ V, int64_t ld, int nv, int nd2, double* __restrict__ w,
            const double* __restrict__ h, double* part, unsigned* counter, double* out) {
  constexpr int U = gs_unroll(MAXV);
  __shared__ double hs[MAXV];
  if (threadIdx.x < nv) hs[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  double acc[MAXV + 1];
#pragma unroll
  for (int v = 0; v <= MAXV; ++v) acc[v] = 0.0;
  const int64_t stride = (int64_t)gridDim.x * GS_THREADS;
  for (int64_t e0 = blockIdx.x * (int64_t)GS_THREADS + threadIdx.x; e0 < n; e0 += stride * U) {
    double we[U];
#pragma unroll
    for (int u = 0; u < U; ++u) we[u] = (e0 + u * stride < n) ? w[e0 + u * stride] : 0.0;
#pragma unroll
    for (int v = 0; v < MAXV; ++v)
      if (v < nv) {
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (e0 + u * stride < n) we[u] = fma(-hs[v], V[v * ld + e0 + u * stride], we[u]);
      }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (e0 + u * stride < n) {
        w[e0 + u * stride] = we[u];
        acc[MAXV] = fma(we[u], we[u], acc[MAXV]);
      }
    // the second projection's dots (twice-applied form) re-read the basis from cache
#pragma unroll
    for (int v = 0; v < MAXV; ++v)
      if (v < nd2) {
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (e0 + u * stride < n) acc[v] = fma(V[v * ld + e0 + u * stride], we[u], acc[v]);
      }
  }
  multi_reduce<MAXV>(acc, nd2, true, part, counter, out);
}

// w -= sum_i h2[i] v_i, then w /= hn with hn^2 = nrm2 - |h2|^2 (0 if not
// positive: the Krylov space is invariant, w is set to zero); block 0 writes
// hn to *hn_out.  Here nrm2 = h2[nv].
template <int MAXV>
__global__ void __launch_bounds__(GS_THREADS)
k_gs_final(int64_t n, const double* __restrict__ V, int64_t ld, int nv, double* __restrict__ w,
           const double* __restrict__ h2, double* hn_out) {
  constexpr int U = gs_unroll(MAXV);
  __shared__ double hs[MAXV];
  __shared__ double inv;
  if (threadIdx.x < nv) hs[threadIdx.x] = h2[threadIdx.x];
  if (threadIdx.x == 0) {
    double s = h2[nv];
    for (int v = 0; v < nv; ++v) s = fma(-h2[v], h2[v], s);
    const double hn = s > 0.0 ? sqrt(s) : 0.0;
    inv = hn > 0.0 ? 1.0 / hn : 0.0;
    if (blockIdx.x == 0) *hn_out = hn;
  }
  __syncthreads();
  const double sc = inv;
  const int64_t stride = (int64_t)gridDim.x * GS_THREADS;
  for (int64_t e0 = blockIdx.x * (int64_t)GS_THREADS + threadIdx.x; e0 < n; e0 += stride * U) {
    double we[U];
#pragma unroll
    for (int u = 0; u < U; ++u) we[u] = (e0 + u * stride < n) ? w[e0 + u * stride] : 0.0;
#pragma unroll
    for (int v = 0; v < MAXV; ++v)
      if (v < nv) {
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (e0 + u * stride < n) we[u] = fma(-hs[v], V[v * ld + e0 + u * stride], we[u]);
      }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (e0 + u * stride < n) w[e0 + u * stride] = we[u] * sc;
  }
}

// x += sum_i y[i] z_i
template <int MAXV>
__global__ void __launch_bounds__(GS_THREADS)
k_gmres_x(int64_t n, double* __restrict__ x, const double* __restrict__ Z, int64_t ld, int nv,
          const double* __restrict__ y) {
  constexpr int U = gs_unroll(MAXV);
  __shared__ double ys[MAXV];
  if (threadIdx.x < nv) ys[threadIdx.x] = y[threadIdx.x];
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * GS_THREADS;
  for (int64_t e0 = blockIdx.x * (int64_t)GS_THREADS + threadIdx.x; e0 < n; e0 += stride * U) {
    double xe[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xe[u] = (e0 + u * stride < n) ? x[e0 + u * stride] : 0.0;
#pragma unroll
    for (int v = 0; v < MAXV; ++v)
      if (v < nv) {
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (e0 + u * stride < n) xe[u] = fma(ys[v], Z[v * ld + e0 + u * stride], xe[u]);
      }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (e0 + u * stride < n) x[e0 + u * stride] = xe[u];
  }
}

// v = b - q; s0 = |v|^2
__global__ void k_sub_norm(int64_t n, const double* __restrict__ b, const double* __restrict__ q,
                           double* __restrict__ v, Reduce red) {
  double s0 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = b[i] - q[i];
    v[i] = d;
    s0 = fma(d, d, s0);
  }
  HMG_RED_SCRATCH(scratch);
  grid_reduce<1>(s0, 0.0, red, scratch);
}

// s0 = a.b over n entries
__global__ void k_dot_n(int64_t n, const double* __restrict__ a, const double* __restrict__ b, Reduce red) {
  double s0 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s0 = fma(a[i], b[i], s0);
  HMG_RED_SCRATCH(scratch);
  grid_reduce<1>(s0, 0.0, red, scratch);
}

// v = a / sqrt(*nrm2)  (a may be v)
__global__ void k_normalise(int64_t n, const double* a, double* v, const double* __restrict__ nrm2) {
  const double s = 1.0 / sqrt(*nrm2);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = a[i] * s;
}

int gs_blocks(int64_t n) {
  const int64_t b = (n + GS_THREADS - 1) / GS_THREADS;
  return (int)(b < GS_MAX_BLOCKS ? (b < 1 ? 1 : b) : GS_MAX_BLOCKS);
}

template <int MAXV>
void gs_launch(int which, int64_t n, const double* V, int64_t ld, int nv, double* w, const double* h,
               const GsWork& ws, cudaStream_t s) {
  const int g = gs_blocks(n);
  switch (which) {
    case 0: k_gs_dots<MAXV><<<g, GS_THREADS, 0, s>>>(n, V, ld, nv, w, ws.part, ws.counter, ws.h); break;
    case 1: k_gs_update<MAXV><<<g, GS_THREADS, 0, s>>>(n, V, ld, nv, nv, w, ws.h, ws.part, ws.counter, ws.h2); break;
    case 4: k_gs_update<MAXV><<<g, GS_THREADS, 0, s>>>(n, V, ld, nv, 0, w, ws.h, ws.part, ws.counter, ws.h2); break;
    case 2: k_gs_final<MAXV><<<g, GS_THREADS, 0, s>>>(n, V, ld, nv, w, ws.h2, ws.hn); break;
    default: k_gmres_x<MAXV><<<g, GS_THREADS, 0, s>>>(n, w, V, ld, nv, h); break;
  }
}

void gs_dispatch(int which, int64_t n, const double* V, int64_t ld, int nv, double* w, const double* h,
                 const GsWork& ws, cudaStream_t s) {
  if (nv <= 8) gs_launch<8>(which, n, V, ld, nv, w, h, ws, s);
  else if (nv <= 16) gs_launch<16>(which, n, V, ld, nv, w, h, ws, s);
  else gs_launch<GMRES_MAX_RESTART>(which, n, V, ld, nv, w, h, ws, s);
}

}  // namespace

void launch_gs_dots(int64_t n, const double* V, int64_t ld, int nv, const double* w, const GsWork& ws,
                    cudaStream_t s) {
  gs_dispatch(0, n, V, ld, nv, const_cast<double*>(w), nullptr, ws, s);
}

void launch_gs_update(int64_t n, const double* V, int64_t ld, int nv, bool second_dots, double* w,
                      const GsWork& ws, cudaStream_t s) {
  gs_dispatch(second_dots ? 1 : 4, n, V, ld, nv, w, nullptr, ws, s);
}

void launch_gs_final(int64_t n, const double* V, int64_t ld, int nv, double* w, const GsWork& ws,
                     cudaStream_t s) {
  gs_dispatch(2, n, V, ld, nv, w, nullptr, ws, s);
}

void launch_gmres_x(int64_t n, double* x, const double* Z, int64_t ld, int nv, const double* y, cudaStream_t s) {
  gs_dispatch(3, n, Z, ld, nv, x, y, GsWork{}, s);
}

void launch_sub_norm(int64_t n, const double* b, const double* q, double* v, const Reduce& red, cudaStream_t s) {
  k_sub_norm<<<reduce_grid(n), 256, 0, s>>>(n, b, q, v, red);
}

void launch_normalise(int64_t n, const double* a, double* v, const double* nrm2, cudaStream_t s) {
  k_normalise<<<reduce_grid(n), 256, 0, s>>>(n, a, v, nrm2);
}

void launch_dot_n(int64_t n, const double* a, const double* b, const Reduce& red, cudaStream_t s) {
  k_dot_n<<<reduce_grid(n), 256, 0, s>>>(n, a, b, red);
}

}  // namespace hmg
