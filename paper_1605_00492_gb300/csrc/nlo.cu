// Kernels of the next-to-lowest-order (NLO) level: operator application,
// residual with the p-restriction DG1 -> DG0 (Sec. 4.2.1), the column block
// relaxation of Eq. (BlockJacobi) with the block-tridiagonal H^_z of Eq.
// (HHgeneralbanded), the p-prolongation and the layout conversion.
//
// One warp owns a tile of five columns: lane 6 c5 + u holds unknown u of the
// cell of column 5 t + c5 in the current layer (lanes 30 and 31 carry zeros),
// so every access to a vector or coefficient row is one aligned 256-byte
// line, and the six unknowns of a cell exchange values by shuffles inside
// their group of six lanes.  The warp walks the layers of its tile; the
// column solve is the block L D L^T recurrence, forward then backward, with
// the forward results kept in a scratch vector (same lane, same thread).  The
// per-cell coefficients (three 6 x 6 blocks per kernel) are the dominant
// memory traffic; the 6 x 6 products run on the FP64 pipe.
#include "hmg_internal.h"

namespace hmg {

namespace {

constexpr int NW = 4;                       // warps per CTA
constexpr unsigned FULL = 0xffffffffu;

struct NloArgs {
  int nt, nz;
  const double* __restrict__ Ad;
  const double* __restrict__ Cs;
  const double* __restrict__ Cu;
  const double* __restrict__ Lf;
  const double* __restrict__ Di;
  const double* __restrict__ Lb;
  const double* __restrict__ Nb;
  const int* __restrict__ nb;
};

NloArgs args_of(const NloSys& X, int nz) {
  return NloArgs{X.nt, nz, X.Ad, X.Cs, X.Cu, X.Lf, X.Di, X.Lb, X.Nb, X.nb};
}

// First lane of the lane's group of six (the padding lanes use group 4).
__device__ __forceinline__ int group_base(int lane) {
  const int g = lane / 6;
  return (g > 4 ? 4 : g) * 6;
}

// Horizontal couplings of one lane (6 c5 + 2 j + m): row j of the horizontal
// factor of each neighbour block, and the neighbours' row offsets plus m.
// The block is that factor times Z2 = [[5, 4], [4, 5]] / 12 over (m, m'), so
// sum_k N_k x_k = (5 S_m + 4 S_(1-m)) / 12 with S_m = sum_k sum_j' H_k[j][j']
// x_k[j', m]: 9 FMA per lane and the partner lane's S by one shuffle.
struct Nbr {
  double h[3][3];
  int base[3];
};

constexpr double Z_SELF = 5.0 / 12.0, Z_OTHER = 4.0 / 12.0;

__device__ __forceinline__ void load_nbr(const NloArgs& A, int t, int lane, Nbr& n) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    n.base[k] = A.nb[(t * 3 + k) * 32 + lane] + (lane & 1);
#pragma unroll
    for (int jj = 0; jj < 3; ++jj) n.h[k][jj] = A.Nb[((size_t)(t * 3 + k) * 3 + jj) * 32 + lane];
  }
}

// the nine neighbour values x_k[j', m] of the lane at layer l
__device__ __forceinline__ void load_nbr_x(const Nbr& n, const double* __restrict__ x, int l, double (&v)[3][3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double* xn = x + n.base[k] + (size_t)l * 32;
#pragma unroll
    for (int jj = 0; jj < 3; ++jj) v[k][jj] = xn[2 * jj];
  }
}

// sum_k sum_j' H_k[j][j'] v[k][j']
__device__ __forceinline__ double nbr_dot(const Nbr& n, const double (&v)[3][3]) {
  double s = n.h[0][0] * v[0][0];
#pragma unroll
  for (int q = 1; q < 9; ++q) s = fma(n.h[q / 3][q % 3], v[q / 3][q % 3], s);
  return s;
}

// uo = u + omega H^_z^-1 (b - H^ u) = (1 - omega) u + omega H^_z^-1 (b - H^_h u)
// (u = nullptr: from zero).  omega is folded into Di.  The operands of layer
// l +- 1 are loaded while layer l is computed.
template <bool FROM_ZERO>
__global__ void __launch_bounds__(NW * 32) k_nlo_sweep(NloArgs A, const double* __restrict__ b,
                                                       const double* __restrict__ u, double* __restrict__ uo,
                                                       double* __restrict__ wbuf, double omega) {
  const int lane = threadIdx.x & 31;
  const int t = blockIdx.x * NW + (threadIdx.x >> 5);
  if (t >= A.nt) return;   // warp-uniform
  const int g = group_base(lane);
  const size_t tile0 = (size_t)t * A.nz * 32;
  const int nz = A.nz;
  Nbr n;
  if (!FROM_ZERO) load_nbr(A, t, lane, n);
  // forward: w_l = (b - H^_h u)_l - L_l w_(l-1)
  double bq = b[tile0 + lane], vq[3][3], Lq[6];
  if (!FROM_ZERO) load_nbr_x(n, u, 0, vq);
#pragma unroll
  for (int e = 0; e < 6; ++e) Lq[e] = 0.0;
  double wprev = 0.0;
  for (int l = 0; l < nz; ++l) {
    const size_t row = tile0 + (size_t)l * 32;
    const double bl = bq;
    double vl[3][3], Ll[6];
#pragma unroll
    for (int q = 0; q < 9; ++q) vl[q / 3][q % 3] = vq[q / 3][q % 3];
#pragma unroll
    for (int e = 0; e < 6; ++e) Ll[e] = Lq[e];
    if (l + 1 < nz) {   // prefetch layer l + 1
      const size_t rn = row + 32;
      bq = b[rn + lane];
      if (!FROM_ZERO) load_nbr_x(n, u, l + 1, vq);
#pragma unroll
      for (int e = 0; e < 6; ++e) Lq[e] = A.Lf[rn * 6 + e * 32 + lane];
    }
    double w = bl;
    if (!FROM_ZERO) {
      const double S = nbr_dot(n, vl);
      const double Sp = __shfl_xor_sync(FULL, S, 1);
      w = fma(-Z_SELF, S, w);
      w = fma(-Z_OTHER, Sp, w);
    }
    if (l > 0) {
#pragma unroll
      for (int e = 0; e < 6; ++e) w = fma(-Ll[e], __shfl_sync(FULL, wprev, g + e), w);
    }
    wbuf[row + lane] = w;
    wprev = w;
  }
  // backward: x_l = omega Dt_l^-1 w_l - L_(l+1)^T x_(l+1)
  const size_t rlast = tile0 + (size_t)(nz - 1) * 32;
  double wq = wprev, uq = FROM_ZERO ? 0.0 : u[rlast + lane], Dq[6], Bq[6];
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    Dq[e] = A.Di[rlast * 6 + e * 32 + lane];
    Bq[e] = 0.0;
  }
  double xnext = 0.0;
  for (int l = nz - 1; l >= 0; --l) {
    const size_t row = tile0 + (size_t)l * 32;
    const double wl = wq, ul = uq;
    double Dl[6], Bl[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      Dl[e] = Dq[e];
      Bl[e] = Bq[e];
    }
    if (l > 0) {   // prefetch layer l - 1
      const size_t rp = row - 32;
      wq = wbuf[rp + lane];
      if (!FROM_ZERO) uq = u[rp + lane];
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        Dq[e] = A.Di[rp * 6 + e * 32 + lane];
        Bq[e] = A.Lb[rp * 6 + e * 32 + lane];
      }
    }
    double x = 0.0;
#pragma unroll
    for (int e = 0; e < 6; ++e) x = fma(Dl[e], __shfl_sync(FULL, wl, g + e), x);
    if (l < nz - 1) {
#pragma unroll
      for (int e = 0; e < 6; ++e) x = fma(-Bl[e], __shfl_sync(FULL, xnext, g + e), x);
    }
    double out = x;
    if (!FROM_ZERO) out = fma(1.0 - omega, ul, x);
    uo[row + lane] = lane < 30 ? out : 0.0;
    xnext = x;
  }
}

constexpr int LCH = 8;   // layers per warp in the layer-parallel kernels

// RESID: bc[(c, l)] = sum over the cell's six unknowns of (b - H^ x);
// otherwise y = H^ x.  One warp per (tile, chunk of LCH layers).
template <bool RESID>
__global__ void __launch_bounds__(NW * 32) k_nlo_op(NloArgs A, const double* __restrict__ x,
                                                    const double* __restrict__ b, double* __restrict__ y,
                                                    double* __restrict__ bc, int nchunks) {
  const int lane = threadIdx.x & 31;
  const int wid = blockIdx.x * NW + (threadIdx.x >> 5);
  if (wid >= A.nt * nchunks) return;   // warp-uniform
  const int t = wid / nchunks, l0 = (wid % nchunks) * LCH;
  const int nz = A.nz;
  const int l1 = min(nz, l0 + LCH);
  const int g = group_base(lane);
  const size_t tile0 = (size_t)t * nz * 32;
  Nbr n;
  load_nbr(A, t, lane, n);
  double xm = l0 > 0 ? x[tile0 + (size_t)(l0 - 1) * 32 + lane] : 0.0;
  double x0 = x[tile0 + (size_t)l0 * 32 + lane];
  for (int l = l0; l < l1; ++l) {
    const size_t row = tile0 + (size_t)l * 32;
    const size_t crow = row * 6;
    const double xp = l + 1 < nz ? x[row + 32 + lane] : 0.0;
    double v[3][3];
    load_nbr_x(n, x, l, v);
    const double S = nbr_dot(n, v);
    const double Sp = __shfl_xor_sync(FULL, S, 1);
    double acc = Z_SELF * S;
    acc = fma(Z_OTHER, Sp, acc);
#pragma unroll
    for (int e = 0; e < 6; ++e) acc = fma(A.Ad[crow + e * 32 + lane], __shfl_sync(FULL, x0, g + e), acc);
    if (l > 0) {
#pragma unroll
      for (int e = 0; e < 6; ++e) acc = fma(A.Cs[crow + e * 32 + lane], __shfl_sync(FULL, xm, g + e), acc);
    }
    if (l + 1 < nz) {
#pragma unroll
      for (int e = 0; e < 6; ++e) acc = fma(A.Cu[crow + e * 32 + lane], __shfl_sync(FULL, xp, g + e), acc);
    }
    if (RESID) {
      const double r = lane < 30 ? b[row + lane] - acc : 0.0;
      const double pair = r + __shfl_xor_sync(FULL, r, 1);           // the two unknowns of vertex j
      const double s = pair + __shfl_sync(FULL, pair, g + 2) + __shfl_sync(FULL, pair, g + 4);
      if (lane < 30 && lane == g) {
        const int c = t * NLO_TILE + lane / 6;
        bc[(size_t)(c / TW) * TW * nz + (size_t)l * TW + (c % TW)] = s;
      }
    } else {
      y[row + lane] = lane < 30 ? acc : 0.0;
    }
    xm = x0;
    x0 = xp;
  }
}

// u += P ec: every unknown of a cell gets the cell's coarse value.
__global__ void k_nlo_prolong(int64_t n, int nz, double* __restrict__ u, const double* __restrict__ ec) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int lane = (int)(i & 31);
  if (lane >= 30) return;
  const int64_t tl = i >> 5;                 // t * nz + l
  const int l = (int)(tl % nz);
  const int64_t c = (tl / nz) * NLO_TILE + lane / 6;
  u[i] += ec[(c / TW) * TW * nz + (int64_t)l * TW + (c % TW)];
}

// NLO COLUMN ((c nz + l) 6 + u) <-> NLO tiles
__global__ void k_nlo_layout(int64_t n, int nz, bool to_tiled, const double* __restrict__ src,
                             double* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int lane = (int)(i & 31);
  const int64_t tl = i >> 5;
  const int l = (int)(tl % nz);
  const int64_t c = (tl / nz) * NLO_TILE + lane / 6;
  const int64_t j = (c * nz + l) * 6 + lane % 6;
  if (to_tiled) dst[i] = lane < 30 ? src[j] : 0.0;
  else if (lane < 30) dst[j] = src[i];
}

int warps_grid(int nt) { return (nt + NW - 1) / NW; }

int elem_grid(int64_t n) { return (int)((n + 255) / 256); }

}  // namespace

void launch_nlo_layout(const NloSys& X, int nz, bool to_tiled, const double* src, double* dst, cudaStream_t s) {
  k_nlo_layout<<<elem_grid(X.n), 256, 0, s>>>(X.n, nz, to_tiled, src, dst);
}

int chunks(int nz) { return (nz + LCH - 1) / LCH; }

void launch_nlo_apply(const NloSys& X, int nz, const double* x, double* y, cudaStream_t s) {
  k_nlo_op<false><<<warps_grid(X.nt * chunks(nz)), NW * 32, 0, s>>>(args_of(X, nz), x, nullptr, y, nullptr,
                                                                    chunks(nz));
}

void launch_nlo_resid_restrict(const NloSys& X, const Level& L0, const double* b, const double* u, double* bc,
                               cudaStream_t s) {
  k_nlo_op<true><<<warps_grid(X.nt * chunks(L0.nz)), NW * 32, 0, s>>>(args_of(X, L0.nz), u, b, nullptr, bc,
                                                                      chunks(L0.nz));
}

void launch_nlo_sweep(const NloSys& X, int nz, const double* b, const double* u, double* uo, double omega,
                      cudaStream_t s) {
  if (u)
    k_nlo_sweep<false><<<warps_grid(X.nt), NW * 32, 0, s>>>(args_of(X, nz), b, u, uo, X.w, omega);
  else
    k_nlo_sweep<true><<<warps_grid(X.nt), NW * 32, 0, s>>>(args_of(X, nz), b, nullptr, uo, X.w, omega);
}

void launch_nlo_prolong(const NloSys& X, const Level& L0, double* u, const double* ec, cudaStream_t s) {
  k_nlo_prolong<<<elem_grid(X.n), 256, 0, s>>>(X.n, L0.nz, u, ec);
}

}  // namespace hmg
