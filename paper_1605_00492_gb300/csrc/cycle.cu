// Kernels of the horizontal-only multigrid V-cycle (Sec. 4.2.1, Algorithm 1)
// and of the operator application (Sec. 5.4).
//
// The block-Jacobi line smoother u <- u + omega H^_z^-1 (b - H^ u) is
// evaluated in the algebraically identical split form
//     u' = (1 - omega) u + omega H^_z^-1 (b - H^_h u),          H^ = H^_z + H^_h,
// which never touches the diagonal or the vertical band of H^: it needs b, u,
// the three horizontal neighbour columns of u and the L D L^T factors of H^_z
// (with omega folded into D^-1).  With u = 0 (first pre-smoothing step) it is
// u' = omega H^_z^-1 b.
//
// Thread mapping.  Sweeps run one thread per column: the forward elimination
// and back substitution of the tridiagonal column are sequential in the
// layer.  In the tiled layout a warp owns the 32 columns of a tile and every
// load or store of one layer is a single 256-byte (FP64) or 128-byte (FP32)
// coalesced access.  The residual/restriction and the operator application
// are layer parallel: one thread per cell.
#include "hmg_internal.h"
#include "reduce.cuh"

namespace hmg {

namespace {

template <typename T> struct Vec4;
template <> struct Vec4<double> { using type = double4_32a; };
template <> struct Vec4<float> { using type = float4; };

template <typename T>
struct LD {
  int nc, nz;
  int64_t Np;
  const int4* __restrict__ nbr;
  const typename Vec4<T>::type* __restrict__ gh;
  const T* __restrict__ d;
  const T* __restrict__ e;
  const T* __restrict__ lo;
  const T* __restrict__ w;
};

template <typename T> LD<T> view(const Level& L);
template <> LD<double> view<double>(const Level& L) {
  return LD<double>{L.nc, L.nz, L.Np, L.nbr, L.gh, L.d, L.e, L.lo, L.w};
}
template <> LD<float> view<float>(const Level& L) {
  return LD<float>{L.nc, L.nz, L.Np, L.nbr, L.gh32, L.d32, L.e32, L.lo32, L.w32};
}

__device__ __forceinline__ int64_t tile_base(int c, int nz) {
  return (int64_t)(c >> 5) * (TW * nz) + (c & 31);
}

// u = omega H^_z^-1 b   (first pre-smoothing step from u = 0)
template <typename T, typename TB>
__global__ void k_sweep0(LD<T> L, const TB* __restrict__ b, T* u, float* __restrict__ bcopy) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.nc) return;
  const int nz = L.nz;
  const int64_t s = tile_base(c, nz);
  T y = 0;
#pragma unroll 4
  for (int l = 0; l < nz; ++l) {
    int64_t t = s + (int64_t)l * TW;
    T bl = (T)b[t];
    if (bcopy) bcopy[t] = (float)bl;
    y = bl - L.lo[t] * y;
    u[t] = y;
  }
  T x = 0, lnext = 0;
#pragma unroll 4
  for (int l = nz - 1; l >= 0; --l) {
    int64_t t = s + (int64_t)l * TW;
    T lcur = L.lo[t];
    x = L.w[t] * u[t] - lnext * x;
    u[t] = x;
    lnext = lcur;
  }
}

// u' = (1 - omega) u~ + omega H^_z^-1 (b - H^_h u~), with u~ = u, or with
// PRO: u~ = u + P e_c (prolongation of the coarse correction fused in: the
// coarse value of the parent column c / 4 is added to u in every column read,
// the neighbours included).  y is scratch for the forward elimination and may
// be the same buffer as uo.
template <typename T, typename TO, bool PRO, typename TE>
__global__ void k_sweep(LD<T> L, const T* __restrict__ b, const T* __restrict__ u, TO* uo, T* y,
                        const TE* __restrict__ ec, T om1) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.nc) return;
  const int nz = L.nz;
  const int4 nb = L.nbr[c];
  const typename Vec4<T>::type g = L.gh[c];
  const int64_t s = tile_base(c, nz), s0 = tile_base(nb.x, nz), s1 = tile_base(nb.y, nz),
                s2 = tile_base(nb.z, nz);
  int64_t q = 0, q0 = 0, q1 = 0, q2 = 0;
  if (PRO) {
    q = tile_base(c >> 2, nz);
    q0 = tile_base(nb.x >> 2, nz);
    q1 = tile_base(nb.y >> 2, nz);
    q2 = tile_base(nb.z >> 2, nz);
  }
  T yv = 0;
#pragma unroll 4
  for (int l = 0; l < nz; ++l) {
    const int64_t o = (int64_t)l * TW;
    T a0 = u[s0 + o], a1 = u[s1 + o], a2 = u[s2 + o];
    if (PRO) {
      a0 += (T)ec[q0 + o];
      a1 += (T)ec[q1 + o];
      a2 += (T)ec[q2 + o];
    }
    T r = b[s + o] + g.x * a0 + g.y * a1 + g.z * a2;
    yv = r - L.lo[s + o] * yv;
    y[s + o] = yv;
  }
  T x = 0, lnext = 0;
#pragma unroll 4
  for (int l = nz - 1; l >= 0; --l) {
    const int64_t o = (int64_t)l * TW;
    T lcur = L.lo[s + o];
    x = L.w[s + o] * y[s + o] - lnext * x;
    T uc = u[s + o];
    if (PRO) uc += (T)ec[q + o];
    uo[s + o] = (TO)(om1 * uc + x);
    lnext = lcur;
  }
}

// u += P e_c (layer parallel, in place)
template <typename T, typename TE>
__global__ void k_prolong(int nc, int nz, int64_t Np, T* __restrict__ u, const TE* __restrict__ ec) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= Np) return;
  int lane = (int)(t & 31);
  int64_t tile = t / (TW * nz);
  int l = (int)((t >> 5) % nz);
  int c = (int)(tile * TW + lane);
  if (c >= nc) return;
  u[t] += (T)ec[tile_base(c >> 2, nz) + (int64_t)l * TW];
}

// (H^ x) at tiled index t = (column c, layer l)
template <typename T>
__device__ __forceinline__ T stencil(const LD<T>& L, const T* __restrict__ x, int64_t t, int c, int l) {
  const int4 nb = L.nbr[c];
  const typename Vec4<T>::type g = L.gh[c];
  const int64_t o = (int64_t)l * TW;
  T y = L.d[t] * x[t];
  if (l > 0) y += L.e[t] * x[t - TW];
  if (l < L.nz - 1) y += L.e[t + TW] * x[t + TW];
  y -= g.x * x[tile_base(nb.x, L.nz) + o];
  y -= g.y * x[tile_base(nb.y, L.nz) + o];
  y -= g.z * x[tile_base(nb.z, L.nz) + o];
  return y;
}

// b_c = P^T (b - H^ u): the residual summed over the four children.  The
// children 4C..4C+3 of coarse column C sit in four adjacent lanes of one tile
// row, so the sum is two shuffles.  Launched over whole warps of the tiled
// range (Np is a multiple of 32).
template <typename T, typename TC>
__global__ void k_resid_restrict(LD<T> L, const T* __restrict__ b, const T* __restrict__ u,
                                 TC* __restrict__ bc) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= L.Np) return;  // whole warps: Np % 32 == 0 and blockDim % 32 == 0
  const int nz = L.nz;
  int lane = (int)(t & 31);
  int64_t tile = t / (TW * nz);
  int l = (int)((t >> 5) % nz);
  int c = (int)(tile * TW + lane);
  T r = 0;
  if (c < L.nc) r = b[t] - stencil(L, u, t, c, l);
  r += __shfl_xor_sync(0xffffffffu, r, 1);
  r += __shfl_xor_sync(0xffffffffu, r, 2);
  if ((lane & 3) == 0 && c < L.nc) bc[tile_base(c >> 2, nz) + (int64_t)l * TW] = (TC)r;
}

// y = H^ x; with a reduction, also x.y (the p.q of CG).
template <typename T, bool DOT>
__global__ void k_apply(LD<T> L, const T* __restrict__ x, T* __restrict__ y, Reduce red) {
  const int nz = L.nz;
  double acc = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < L.Np;
       t += (int64_t)gridDim.x * blockDim.x) {
    int lane = (int)(t & 31);
    int64_t tile = t / (TW * nz);
    int l = (int)((t >> 5) % nz);
    int c = (int)(tile * TW + lane);
    T v = 0;
    if (c < L.nc) v = stencil(L, x, t, c, l);
    y[t] = v;
    if (DOT) acc += (double)x[t] * (double)v;
  }
  if (DOT) grid_reduce2(acc, 0.0, red);
}

inline unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

constexpr int SWEEP_BS = 64;

template <typename T>
void sweep0_t(const Level& L, const void* b, int b_dt, void* u, float* bcopy, double omega,
              cudaStream_t s) {
  (void)omega;
  unsigned g = blocks_for(L.nc, SWEEP_BS);
  if (b_dt == HMG_FP64)
    k_sweep0<T, double><<<g, SWEEP_BS, 0, s>>>(view<T>(L), (const double*)b, (T*)u, bcopy);
  else
    k_sweep0<T, float><<<g, SWEEP_BS, 0, s>>>(view<T>(L), (const float*)b, (T*)u, bcopy);
}

template <typename T, typename TO>
void sweep_t2(const Level& L, const void* b, const void* u, void* uo, void* ytmp, const void* ec,
              int ec_dt, double omega, cudaStream_t s) {
  unsigned g = blocks_for(L.nc, SWEEP_BS);
  T* y = std::is_same<T, TO>::value ? (T*)uo : (T*)ytmp;
  T om1 = (T)(1.0 - omega);
  if (ec == nullptr)
    k_sweep<T, TO, false, T><<<g, SWEEP_BS, 0, s>>>(view<T>(L), (const T*)b, (const T*)u, (TO*)uo, y,
                                                     (const T*)nullptr, om1);
  else if (ec_dt == HMG_FP64)
    k_sweep<T, TO, true, double><<<g, SWEEP_BS, 0, s>>>(view<T>(L), (const T*)b, (const T*)u, (TO*)uo, y,
                                                          (const double*)ec, om1);
  else
    k_sweep<T, TO, true, float><<<g, SWEEP_BS, 0, s>>>(view<T>(L), (const T*)b, (const T*)u, (TO*)uo, y,
                                                         (const float*)ec, om1);
}

}  // namespace

void launch_sweep0(const Level& L, int dt, const void* b, int b_dt, void* u, float* bcopy, double omega,
                   cudaStream_t s) {
  if (dt == HMG_FP64) sweep0_t<double>(L, b, b_dt, u, nullptr, omega, s);
  else sweep0_t<float>(L, b, b_dt, u, bcopy, omega, s);
}

void launch_sweep(const Level& L, int dt, const void* b, const void* u, void* uo, int uo_dt, void* ytmp,
                  const void* ec, int ec_dt, double omega, cudaStream_t s) {
  if (dt == HMG_FP64) {
    sweep_t2<double, double>(L, b, u, uo, ytmp, ec, ec_dt, omega, s);
  } else if (uo_dt == HMG_FP64) {
    sweep_t2<float, double>(L, b, u, uo, ytmp, ec, ec_dt, omega, s);
  } else {
    sweep_t2<float, float>(L, b, u, uo, ytmp, ec, ec_dt, omega, s);
  }
}

void launch_prolong(const Level& L, int dt, void* u, const void* ec, int ec_dt, cudaStream_t s) {
  unsigned g = blocks_for(L.Np, 256);
  if (dt == HMG_FP64)
    k_prolong<double, double><<<g, 256, 0, s>>>(L.nc, L.nz, L.Np, (double*)u, (const double*)ec);
  else if (ec_dt == HMG_FP64)
    k_prolong<float, double><<<g, 256, 0, s>>>(L.nc, L.nz, L.Np, (float*)u, (const double*)ec);
  else
    k_prolong<float, float><<<g, 256, 0, s>>>(L.nc, L.nz, L.Np, (float*)u, (const float*)ec);
}

void launch_resid_restrict(const Level& L, int dt, const void* b, const void* u, void* bc, int bc_dt,
                           cudaStream_t s) {
  unsigned g = blocks_for(L.Np, 256);
  if (dt == HMG_FP64)
    k_resid_restrict<double, double><<<g, 256, 0, s>>>(view<double>(L), (const double*)b, (const double*)u,
                                                        (double*)bc);
  else if (bc_dt == HMG_FP64)
    k_resid_restrict<float, double><<<g, 256, 0, s>>>(view<float>(L), (const float*)b, (const float*)u,
                                                       (double*)bc);
  else
    k_resid_restrict<float, float><<<g, 256, 0, s>>>(view<float>(L), (const float*)b, (const float*)u,
                                                      (float*)bc);
}

void launch_apply(const Level& L, int dt, const void* x, void* y, const Reduce* red, cudaStream_t s) {
  if (red) {
    int g = reduce_grid(L.Np);
    if (dt == HMG_FP64)
      k_apply<double, true><<<g, 256, 0, s>>>(view<double>(L), (const double*)x, (double*)y, *red);
    else
      k_apply<float, true><<<g, 256, 0, s>>>(view<float>(L), (const float*)x, (float*)y, *red);
  } else {
    unsigned g = blocks_for(L.Np, 256);
    Reduce none{};
    if (dt == HMG_FP64)
      k_apply<double, false><<<g, 256, 0, s>>>(view<double>(L), (const double*)x, (double*)y, none);
    else
      k_apply<float, false><<<g, 256, 0, s>>>(view<float>(L), (const float*)x, (float*)y, none);
  }
}

}  // namespace hmg
