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
// memory traffic; in FP64 the 6 x 6 products run on the FP64 pipe, which
// bounds the kernels.  The mixed form runs the level in FP32 (FP32 copies of
// the coefficients, FP32 work vectors): the operator and residual with the
// same kernels, the column sweep with a variant that stages its operands in
// shared memory, since in FP32 memory latency, not arithmetic, bounds it.
#include <atomic>
#include <stdexcept>
#include <string>

#include "hmg_internal.h"

namespace hmg {

namespace {

constexpr int NW = 4;                       // warps per CTA
constexpr unsigned FULL = 0xffffffffu;

template <typename T>
struct NloArgs {
  int nt, nz;
  const T* __restrict__ Ad;
  const T* __restrict__ Cs;
  const T* __restrict__ Cu;
  const T* __restrict__ Lf;
  const T* __restrict__ Di;
  const T* __restrict__ Lb;
  const T* __restrict__ Nb;
  const int* __restrict__ nb;
};

NloArgs<double> args_of(const NloSys& X, int nz, double) {
  return NloArgs<double>{X.nt, nz, X.Ad, X.Cs, X.Cu, X.Lf, X.Di, X.Lb, X.Nb, X.nb};
}
NloArgs<float> args_of(const NloSys& X, int nz, float) {
  return NloArgs<float>{X.nt, nz, X.Ad32, X.Cs32, X.Cu32, X.Lf32, X.Di32, X.Lb32, X.Nb32, X.nb};
}

__device__ __forceinline__ float fmx(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmx(double a, double b, double c) { return __fma_rn(a, b, c); }

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
template <typename T>
struct Nbr {
  T h[3][3];
  int base[3];
};

constexpr double Z_SELF = 5.0 / 12.0, Z_OTHER = 4.0 / 12.0;

template <typename T>
__device__ __forceinline__ void load_nbr(const NloArgs<T>& A, int t, int lane, Nbr<T>& n) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    n.base[k] = A.nb[(t * 3 + k) * 32 + lane] + (lane & 1);
#pragma unroll
    for (int jj = 0; jj < 3; ++jj) n.h[k][jj] = A.Nb[((size_t)(t * 3 + k) * 3 + jj) * 32 + lane];
  }
}

// the nine neighbour values x_k[j', m] of the lane at layer l
template <typename T>
__device__ __forceinline__ void load_nbr_x(const Nbr<T>& n, const T* __restrict__ x, int l, T (&v)[3][3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const T* xn = x + n.base[k] + (size_t)l * 32;
#pragma unroll
    for (int jj = 0; jj < 3; ++jj) v[k][jj] = xn[2 * jj];
  }
}

// sum_k sum_j' H_k[j][j'] v[k][j']
template <typename T>
__device__ __forceinline__ T nbr_dot(const Nbr<T>& n, const T (&v)[3][3]) {
  T s = n.h[0][0] * v[0][0];
#pragma unroll
  for (int q = 1; q < 9; ++q) s = fmx(n.h[q / 3][q % 3], v[q / 3][q % 3], s);
  return s;
}

// uo = u + omega H^_z^-1 (b - H^ u) = (1 - omega) u + omega H^_z^-1 (b - H^_h u)
// (u = nullptr: from zero).  omega is folded into Di.  T: arithmetic,
// coefficients and u; TB: b (converted to T, and copied to bcopy when given);
// TO: uo.  Launched in FP64 (the FP32 sweep is k_nlo_sweep_staged).  The warp
// walks its layers as a serial recurrence, so the operands of the next PF
// layers are kept in flight in registers (staged slots refilled as they are
// consumed).  PF = 1: the FP64 pipe bounds the kernel, and in FP32 four
// layers in flight measured slower (96.8 against 90.3 us at r4x64) before the
// shared-memory staging replaced it there.
template <typename T>
struct SweepPF {
  static constexpr int value = 1;
};

template <typename T, bool FROM_ZERO, typename TB, typename TO>
__global__ void __launch_bounds__(NW * 32) k_nlo_sweep(NloArgs<T> A, const TB* __restrict__ b,
                                                       T* __restrict__ bcopy, const T* __restrict__ u,
                                                       TO* __restrict__ uo, T* __restrict__ wbuf, T omega) {
  constexpr int PF = SweepPF<T>::value;
  const int lane = threadIdx.x & 31;
  const int t = blockIdx.x * NW + (threadIdx.x >> 5);
  if (t >= A.nt) return;   // warp-uniform
  const int g = group_base(lane);
  const size_t tile0 = (size_t)t * A.nz * 32;
  const int nz = A.nz;
  const T zs = T(Z_SELF), zo = T(Z_OTHER);
  Nbr<T> n;
  if (!FROM_ZERO) load_nbr(A, t, lane, n);
  // forward: w_l = (b - H^_h u)_l - L_l w_(l-1); slot d holds layer l0 + d
  T bq[PF], vq[PF][3][3], Lq[PF][6];
  auto load_f = [&](int d, int l) {
    const size_t row = tile0 + (size_t)l * 32;
    bq[d] = T(b[row + lane]);
    if (!FROM_ZERO) load_nbr_x(n, u, l, vq[d]);
#pragma unroll
    for (int e = 0; e < 6; ++e) Lq[d][e] = l > 0 ? A.Lf[row * 6 + e * 32 + lane] : T(0);
  };
#pragma unroll
  for (int d = 0; d < PF; ++d)
    if (d < nz) load_f(d, d);
  T wprev = T(0);
  for (int l0 = 0; l0 < nz; l0 += PF) {
#pragma unroll
    for (int d = 0; d < PF; ++d) {
      const int l = l0 + d;
      if (l >= nz) break;   // warp-uniform
      const size_t row = tile0 + (size_t)l * 32;
      const T bl = bq[d];
      T vl[3][3], Ll[6];
#pragma unroll
      for (int q = 0; q < 9; ++q) vl[q / 3][q % 3] = vq[d][q / 3][q % 3];
#pragma unroll
      for (int e = 0; e < 6; ++e) Ll[e] = Lq[d][e];
      if (l + PF < nz) load_f(d, l + PF);   // refill the slot with layer l + PF
      if (bcopy) bcopy[row + lane] = bl;
      T w = bl;
      if (!FROM_ZERO) {
        const T S = nbr_dot(n, vl);
        const T Sp = __shfl_xor_sync(FULL, S, 1);
        w = fmx(-zs, S, w);
        w = fmx(-zo, Sp, w);
      }
      if (l > 0) {
#pragma unroll
        for (int e = 0; e < 6; ++e) w = fmx(-Ll[e], __shfl_sync(FULL, wprev, g + e), w);
      }
      wbuf[row + lane] = w;
      wprev = w;
    }
  }
  // backward: x_l = omega Dt_l^-1 w_l - L_(l+1)^T x_(l+1); slot d holds layer nz - 1 - (k0 + d)
  T wq[PF], uq[PF], Dq[PF][6], Bq[PF][6];
  auto load_b = [&](int d, int l) {
    const size_t row = tile0 + (size_t)l * 32;
    wq[d] = wbuf[row + lane];
    uq[d] = FROM_ZERO ? T(0) : u[row + lane];
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      Dq[d][e] = A.Di[row * 6 + e * 32 + lane];
      Bq[d][e] = l < nz - 1 ? A.Lb[row * 6 + e * 32 + lane] : T(0);
    }
  };
  __syncwarp();   // the forward results of this warp are read back by the same lanes; order the accesses
#pragma unroll
  for (int d = 0; d < PF; ++d)
    if (d < nz) load_b(d, nz - 1 - d);
  T xnext = T(0);
  for (int k0 = 0; k0 < nz; k0 += PF) {
#pragma unroll
    for (int d = 0; d < PF; ++d) {
      const int k = k0 + d;
      if (k >= nz) break;   // warp-uniform
      const int l = nz - 1 - k;
      const size_t row = tile0 + (size_t)l * 32;
      const T wl = wq[d], ul = uq[d];
      T Dl[6], Bl[6];
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        Dl[e] = Dq[d][e];
        Bl[e] = Bq[d][e];
      }
      if (k + PF < nz) load_b(d, l - PF);
      T x = T(0);
#pragma unroll
      for (int e = 0; e < 6; ++e) x = fmx(Dl[e], __shfl_sync(FULL, wl, g + e), x);
      if (l < nz - 1) {
#pragma unroll
        for (int e = 0; e < 6; ++e) x = fmx(-Bl[e], __shfl_sync(FULL, xnext, g + e), x);
      }
      T out = x;
      if (!FROM_ZERO) out = fmx(T(1) - omega, ul, x);
      uo[row + lane] = lane < 30 ? TO(out) : TO(0);
      xnext = x;
    }
  }
}

// ---- FP32 sweep with the operands staged in shared memory.  In FP32 the
// column recurrence is bound by memory latency, not arithmetic: the warp
// keeps RING layers of operands in flight in a per-warp ring of shared-memory
// slots filled by cp.async (one commit group per layer; cp.async.wait_group
// leaves RING - 1 groups pending, so the oldest layer has arrived).  Waits
// are the hardware's; nothing spins.
constexpr int RING = 8;

struct FwdSlot {              // forward operands of one layer
  float L[6][32];             // L_l rows
  float nbv[9][32];           // neighbour values u_k[j', m] of each lane
  double b[32];               // b row (FP32 b uses the first half)
};
struct BwdSlot {              // backward operands of one layer
  float D[6][32];             // omega Dt_l^-1 rows
  float B[6][32];             // L_(l+1)^T rows
  float w[32];
  float u[32];
};
union RingSlot {
  FwdSlot f;
  BwdSlot b;
};

__device__ __forceinline__ void cpa16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cpa4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// copy `bytes` (a multiple of 16) from gmem to smem with the warp's lanes
__device__ __forceinline__ void cpa_row(void* smem, const void* gmem, int bytes, int lane) {
  for (int off = lane * 16; off < bytes; off += 32 * 16)
    cpa16(static_cast<char*>(smem) + off, static_cast<const char*>(gmem) + off);
}

template <bool FROM_ZERO, typename TB, typename TO>
__global__ void __launch_bounds__(NW * 32) k_nlo_sweep_staged(NloArgs<float> A, const TB* __restrict__ b,
                                                              float* __restrict__ bcopy, const float* __restrict__ u,
                                                              TO* __restrict__ uo, float* __restrict__ wbuf,
                                                              float omega) {
  extern __shared__ __align__(16) unsigned char nlo_smem[];
  RingSlot* ring = reinterpret_cast<RingSlot*>(nlo_smem) + (threadIdx.x >> 5) * RING;
  const int lane = threadIdx.x & 31;
  const int t = blockIdx.x * NW + (threadIdx.x >> 5);
  if (t >= A.nt) return;   // warp-uniform; no block-wide barrier below
  const int g = group_base(lane);
  const int nz = A.nz;
  const size_t tile0 = (size_t)t * nz * 32;
  const float zs = float(Z_SELF), zo = float(Z_OTHER);
  Nbr<float> n;
  if (!FROM_ZERO) load_nbr(A, t, lane, n);

  auto issue_f = [&](int l) {   // forward operands of layer l into slot l % RING
    if (l < nz) {
      FwdSlot& S = ring[l % RING].f;
      const size_t row = tile0 + (size_t)l * 32;
      cpa_row(S.L, A.Lf + row * 6, 6 * 32 * 4, lane);
      cpa_row(S.b, b + row, 32 * (int)sizeof(TB), lane);
      if (!FROM_ZERO) {
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int jj = 0; jj < 3; ++jj) cpa4(&S.nbv[3 * k + jj][lane], u + n.base[k] + (size_t)l * 32 + 2 * jj);
      }
    }
    cpa_commit();
  };
#pragma unroll
  for (int l = 0; l < RING; ++l) issue_f(l);
  float wprev = 0.f;
  for (int l = 0; l < nz; ++l) {
    cpa_wait<RING - 1>();
    __syncwarp();
    const FwdSlot& S = ring[l % RING].f;
    const float bl = float(reinterpret_cast<const TB*>(S.b)[lane]);
    if (bcopy) bcopy[tile0 + (size_t)l * 32 + lane] = bl;
    float w = bl;
    if (!FROM_ZERO) {
      float v[3][3];
#pragma unroll
      for (int q = 0; q < 9; ++q) v[q / 3][q % 3] = S.nbv[q][lane];
      const float Sm = nbr_dot(n, v);
      const float Sp = __shfl_xor_sync(FULL, Sm, 1);
      w = fmx(-zs, Sm, w);
      w = fmx(-zo, Sp, w);
    }
    if (l > 0) {
#pragma unroll
      for (int e = 0; e < 6; ++e) w = fmx(-S.L[e][lane], __shfl_sync(FULL, wprev, g + e), w);
    }
    wbuf[tile0 + (size_t)l * 32 + lane] = w;
    wprev = w;
    __syncwarp();          // every lane is done with the slot before it is refilled
    issue_f(l + RING);
  }
  cpa_wait<0>();
  __syncwarp();            // the forward results are in memory before the backward copies read them

  auto issue_b = [&](int k) {   // backward operands of step k (layer nz - 1 - k) into slot k % RING
    if (k < nz) {
      BwdSlot& S = ring[k % RING].b;
      const int l = nz - 1 - k;
      const size_t row = tile0 + (size_t)l * 32;
      cpa_row(S.D, A.Di + row * 6, 6 * 32 * 4, lane);
      cpa_row(S.B, A.Lb + row * 6, 6 * 32 * 4, lane);
      cpa_row(S.w, wbuf + row, 32 * 4, lane);
      if (!FROM_ZERO) cpa_row(S.u, u + row, 32 * 4, lane);
    }
    cpa_commit();
  };
#pragma unroll
  for (int k = 0; k < RING; ++k) issue_b(k);
  float xnext = 0.f;
  for (int k = 0; k < nz; ++k) {
    cpa_wait<RING - 1>();
    __syncwarp();
    const BwdSlot& S = ring[k % RING].b;
    const int l = nz - 1 - k;
    const float wl = S.w[lane];
    float x = 0.f;
#pragma unroll
    for (int e = 0; e < 6; ++e) x = fmx(S.D[e][lane], __shfl_sync(FULL, wl, g + e), x);
    if (l < nz - 1) {
#pragma unroll
      for (int e = 0; e < 6; ++e) x = fmx(-S.B[e][lane], __shfl_sync(FULL, xnext, g + e), x);
    }
    float out = x;
    if (!FROM_ZERO) out = fmx(1.f - omega, S.u[lane], x);
    uo[tile0 + (size_t)l * 32 + lane] = lane < 30 ? TO(out) : TO(0);
    xnext = x;
    __syncwarp();
    issue_b(k + RING);
  }
  cpa_wait<0>();
}

constexpr size_t STAGED_SMEM = sizeof(RingSlot) * RING * NW;

constexpr int LCH = 8;   // layers per warp in the layer-parallel kernels

// RESID: bc[(c, l)] = sum over the cell's six unknowns of (b - H^ x);
// otherwise y = H^ x.  One warp per (tile, chunk of LCH layers).
template <typename T, bool RESID, typename TBC>
__global__ void __launch_bounds__(NW * 32) k_nlo_op(NloArgs<T> A, const T* __restrict__ x,
                                                    const T* __restrict__ b, T* __restrict__ y,
                                                    TBC* __restrict__ bc, int nchunks) {
  const int lane = threadIdx.x & 31;
  const int wid = blockIdx.x * NW + (threadIdx.x >> 5);
  if (wid >= A.nt * nchunks) return;   // warp-uniform
  const int t = wid / nchunks, l0 = (wid % nchunks) * LCH;
  const int nz = A.nz;
  const int l1 = min(nz, l0 + LCH);
  const int g = group_base(lane);
  const size_t tile0 = (size_t)t * nz * 32;
  Nbr<T> n;
  load_nbr(A, t, lane, n);
  T xm = l0 > 0 ? x[tile0 + (size_t)(l0 - 1) * 32 + lane] : T(0);
  T x0 = x[tile0 + (size_t)l0 * 32 + lane];
  // FP32 loads the next layer ahead (residual 75 -> 42 us at r4x64); in FP64,
  // bound by the FP64 pipe, the lookahead measured slower (140 -> 150 us)
  constexpr bool AHEAD = sizeof(T) == 4;
  T xq, vq[3][3], Aq[6], Sq[6], Uq[6];
  auto load_op = [&](int l) {
    const size_t row = tile0 + (size_t)l * 32;
    const size_t crow = row * 6;
    xq = l + 1 < nz ? x[row + 32 + lane] : T(0);
    load_nbr_x(n, x, l, vq);
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      Aq[e] = A.Ad[crow + e * 32 + lane];
      Sq[e] = l > 0 ? A.Cs[crow + e * 32 + lane] : T(0);
      Uq[e] = l + 1 < nz ? A.Cu[crow + e * 32 + lane] : T(0);
    }
  };
  if (AHEAD) load_op(l0);
  for (int l = l0; l < l1; ++l) {
    const size_t row = tile0 + (size_t)l * 32;
    const size_t crow = row * 6;
    T acc, xp;
    if constexpr (AHEAD) {
      xp = xq;
      T v[3][3], Al[6], Sl[6], Ul[6];
#pragma unroll
      for (int q = 0; q < 9; ++q) v[q / 3][q % 3] = vq[q / 3][q % 3];
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        Al[e] = Aq[e];
        Sl[e] = Sq[e];
        Ul[e] = Uq[e];
      }
      if (l + 1 < l1) load_op(l + 1);
      const T S = nbr_dot(n, v);
      const T Sp = __shfl_xor_sync(FULL, S, 1);
      acc = T(Z_SELF) * S;
      acc = fmx(T(Z_OTHER), Sp, acc);
#pragma unroll
      for (int e = 0; e < 6; ++e) acc = fmx(Al[e], __shfl_sync(FULL, x0, g + e), acc);
      if (l > 0) {
#pragma unroll
        for (int e = 0; e < 6; ++e) acc = fmx(Sl[e], __shfl_sync(FULL, xm, g + e), acc);
      }
      if (l + 1 < nz) {
#pragma unroll
        for (int e = 0; e < 6; ++e) acc = fmx(Ul[e], __shfl_sync(FULL, xp, g + e), acc);
      }
    } else {
      xp = l + 1 < nz ? x[row + 32 + lane] : T(0);
      T v[3][3];
      load_nbr_x(n, x, l, v);
      const T S = nbr_dot(n, v);
      const T Sp = __shfl_xor_sync(FULL, S, 1);
      acc = T(Z_SELF) * S;
      acc = fmx(T(Z_OTHER), Sp, acc);
#pragma unroll
      for (int e = 0; e < 6; ++e) acc = fmx(A.Ad[crow + e * 32 + lane], __shfl_sync(FULL, x0, g + e), acc);
      if (l > 0) {
#pragma unroll
        for (int e = 0; e < 6; ++e) acc = fmx(A.Cs[crow + e * 32 + lane], __shfl_sync(FULL, xm, g + e), acc);
      }
      if (l + 1 < nz) {
#pragma unroll
        for (int e = 0; e < 6; ++e) acc = fmx(A.Cu[crow + e * 32 + lane], __shfl_sync(FULL, xp, g + e), acc);
      }
    }
    if (RESID) {
      const T r = lane < 30 ? b[row + lane] - acc : T(0);
      const T pair = r + __shfl_xor_sync(FULL, r, 1);           // the two unknowns of vertex j
      const T sum = pair + __shfl_sync(FULL, pair, g + 2) + __shfl_sync(FULL, pair, g + 4);
      if (lane < 30 && lane == g) {
        const int c = t * NLO_TILE + lane / 6;
        bc[(size_t)(c / TW) * TW * nz + (size_t)l * TW + (c % TW)] = TBC(sum);
      }
    } else {
      y[row + lane] = lane < 30 ? acc : T(0);
    }
    xm = x0;
    x0 = xp;
  }
}

// u += P ec: every unknown of a cell gets the cell's coarse value.
template <typename T, typename TE>
__global__ void k_nlo_prolong(int64_t n, int nz, T* __restrict__ u, const TE* __restrict__ ec) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int lane = (int)(i & 31);
  if (lane >= 30) return;
  const int64_t tl = i >> 5;                 // t * nz + l
  const int l = (int)(tl % nz);
  const int64_t c = (tl / nz) * NLO_TILE + lane / 6;
  u[i] += T(ec[(c / TW) * TW * nz + (int64_t)l * TW + (c % TW)]);
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

void cuda_ok_nlo(cudaError_t e) {
  if (e != cudaSuccess) throw std::runtime_error(std::string("NLO kernel setup: ") + cudaGetErrorString(e));
}

int elem_grid(int64_t n) { return (int)((n + 255) / 256); }

}  // namespace

void launch_nlo_layout(const NloSys& X, int nz, bool to_tiled, const double* src, double* dst, cudaStream_t s) {
  k_nlo_layout<<<elem_grid(X.n), 256, 0, s>>>(X.n, nz, to_tiled, src, dst);
}

int chunks(int nz) { return (nz + LCH - 1) / LCH; }

void launch_nlo_apply(const NloSys& X, int nz, const double* x, double* y, cudaStream_t s) {
  k_nlo_op<double, false, double><<<warps_grid(X.nt * chunks(nz)), NW * 32, 0, s>>>(
      args_of(X, nz, 0.0), x, nullptr, y, nullptr, chunks(nz));
}

template <typename T>
void resid_t(const NloSys& X, const Level& L0, const T* b, const T* u, void* bc, int bc_dt, cudaStream_t s) {
  const int g = warps_grid(X.nt * chunks(L0.nz));
  if (bc_dt == HMG_FP64)
    k_nlo_op<T, true, double><<<g, NW * 32, 0, s>>>(args_of(X, L0.nz, T(0)), u, b, nullptr, (double*)bc,
                                                   chunks(L0.nz));
  else
    k_nlo_op<T, true, float><<<g, NW * 32, 0, s>>>(args_of(X, L0.nz, T(0)), u, b, nullptr, (float*)bc,
                                                  chunks(L0.nz));
}

void launch_nlo_resid_restrict(const NloSys& X, const Level& L0, int dt, const void* b, const void* u, void* bc,
                               int bc_dt, cudaStream_t s) {
  if (dt == HMG_FP64) resid_t(X, L0, (const double*)b, (const double*)u, bc, bc_dt, s);
  else resid_t(X, L0, (const float*)b, (const float*)u, bc, bc_dt, s);
}

template <typename TB, typename TO>
void sweep_staged(const NloSys& X, int nz, const TB* b, float* bcopy, const float* u, TO* uo, float* w,
                  double omega, cudaStream_t s) {
  // opt in to the ring's shared memory, once per instantiation and device
  static std::atomic<unsigned long long> done[2];
  int dev = 0;
  cuda_ok_nlo(cudaGetDevice(&dev));
  const unsigned long long bit = 1ull << (dev & 63);
  if (u) {
    if (!(done[0].load() & bit)) {
      cuda_ok_nlo(cudaFuncSetAttribute(k_nlo_sweep_staged<false, TB, TO>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)STAGED_SMEM));
      done[0] |= bit;
    }
    k_nlo_sweep_staged<false, TB, TO><<<warps_grid(X.nt), NW * 32, STAGED_SMEM, s>>>(
        args_of(X, nz, 0.f), b, bcopy, u, uo, w, float(omega));
  } else {
    if (!(done[1].load() & bit)) {
      cuda_ok_nlo(cudaFuncSetAttribute(k_nlo_sweep_staged<true, TB, TO>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)STAGED_SMEM));
      done[1] |= bit;
    }
    k_nlo_sweep_staged<true, TB, TO><<<warps_grid(X.nt), NW * 32, STAGED_SMEM, s>>>(
        args_of(X, nz, 0.f), b, bcopy, nullptr, uo, w, float(omega));
  }
}

template <typename T, typename TB, typename TO>
void sweep_t(const NloSys& X, int nz, const TB* b, T* bcopy, const T* u, TO* uo, T* w, double omega,
             cudaStream_t s) {
  if (u)
    k_nlo_sweep<T, false, TB, TO><<<warps_grid(X.nt), NW * 32, 0, s>>>(args_of(X, nz, T(0)), b, bcopy, u, uo, w,
                                                                      T(omega));
  else
    k_nlo_sweep<T, true, TB, TO><<<warps_grid(X.nt), NW * 32, 0, s>>>(args_of(X, nz, T(0)), b, bcopy, nullptr, uo,
                                                                     w, T(omega));
}

void launch_nlo_sweep(const NloSys& X, int nz, int dt, const void* b, int b_dt, void* bcopy, const void* u,
                      void* uo, int uo_dt, double omega, cudaStream_t s) {
  if (dt == HMG_FP64) {
    if (b_dt != HMG_FP64 || uo_dt != HMG_FP64 || bcopy) throw std::invalid_argument("NLO FP64 sweep: FP64 only");
    sweep_t<double, double, double>(X, nz, (const double*)b, nullptr, (const double*)u, (double*)uo, X.w, omega, s);
    return;
  }
  float* w = X.w32;
  if (b_dt == HMG_FP64) {
    if (u) throw std::invalid_argument("NLO FP32 sweep: an FP64 right-hand side only from zero");
    if (uo_dt == HMG_FP64)
      sweep_staged<double, double>(X, nz, (const double*)b, (float*)bcopy, nullptr, (double*)uo, w, omega, s);
    else
      sweep_staged<double, float>(X, nz, (const double*)b, (float*)bcopy, nullptr, (float*)uo, w, omega, s);
  } else if (uo_dt == HMG_FP64) {
    sweep_staged<float, double>(X, nz, (const float*)b, nullptr, (const float*)u, (double*)uo, w, omega, s);
  } else {
    sweep_staged<float, float>(X, nz, (const float*)b, nullptr, (const float*)u, (float*)uo, w, omega, s);
  }
}

void launch_nlo_prolong(const NloSys& X, const Level& L0, int dt, void* u, const void* ec, int ec_dt,
                        cudaStream_t s) {
  const int g = elem_grid(X.n);
  if (dt == HMG_FP64 && ec_dt == HMG_FP64)
    k_nlo_prolong<double, double><<<g, 256, 0, s>>>(X.n, L0.nz, (double*)u, (const double*)ec);
  else if (dt == HMG_FP32 && ec_dt == HMG_FP32)
    k_nlo_prolong<float, float><<<g, 256, 0, s>>>(X.n, L0.nz, (float*)u, (const float*)ec);
  else if (dt == HMG_FP32)
    k_nlo_prolong<float, double><<<g, 256, 0, s>>>(X.n, L0.nz, (float*)u, (const double*)ec);
  else
    k_nlo_prolong<double, float><<<g, 256, 0, s>>>(X.n, L0.nz, (double*)u, (const float*)ec);
}

}  // namespace hmg
