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

// ---------------------------------------------------------------- sweeps
//
// One CTA per tile of 32 columns, NW warps, two shared arrays of nz x 32:
//   A  (all warps, layer parallel)  R = b + sum_k g_k u[nbr_k]   (u~ with PRO)
//                                   LO = l-multipliers of L D L^T
//   B  (one warp: lane = column)    forward elimination  y_l = R_l - lo_l y_l-1
//   B' (all warps)                  y_l *= omega / D_l
//   C  (one warp)                   back substitution    x_l = y_l - lo_l+1 x_l+1
//   D  (all warps)                  u' = (1 - omega) u~ + x
// Only the two recurrences are sequential, and they read shared memory, so
// the dependent chain never waits for global memory; everything else is
// spread over the CTA.  MODE_ZERO is the first pre-smoothing step (u = 0):
// no neighbour sum and no relaxation term.
enum { MODE_ZERO = 0, MODE_PLAIN = 1, MODE_PRO = 2 };

// DOT = 1: also reduce sum_cells da * u' (the r.z of CG, da = the FP64
// residual); DOT = 2: and sum_cells u' * dc (the z.q of flexible CG).
template <typename T, typename TB, typename TO, int MODE, typename TE, int NW, int DOT>
__global__ void __launch_bounds__(NW * 32)
k_tsweep(LD<T> L, const TB* __restrict__ b, const T* __restrict__ u, TO* __restrict__ uo,
         const TE* __restrict__ ec, float* __restrict__ bcopy, T om1, const double* __restrict__ da,
         const double* __restrict__ dc, Reduce red) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int RB = 4;  // rows per warp per batch: their loads are issued together
  const int nz = L.nz;
  T* R = reinterpret_cast<T*>(smem_raw);
  T* LOs = R + nz * TW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tile = blockIdx.x;
  const int c = tile * TW + lane;
  const bool valid = c < L.nc;
  const int64_t base = (int64_t)tile * TW * nz + lane;
  int64_t s0 = 0, s1 = 0, s2 = 0, q = 0, q0 = 0, q1 = 0, q2 = 0;
  typename Vec4<T>::type g{};
  if (MODE != MODE_ZERO && valid) {
    const int4 nb = L.nbr[c];
    g = L.gh[c];
    s0 = tile_base(nb.x, nz);
    s1 = tile_base(nb.y, nz);
    s2 = tile_base(nb.z, nz);
    if (MODE == MODE_PRO) {
      q = tile_base(c >> 2, nz);
      q0 = tile_base(nb.x >> 2, nz);
      q1 = tile_base(nb.y >> 2, nz);
      q2 = tile_base(nb.z >> 2, nz);
    }
  }
  // A
  for (int l0 = warp; l0 < nz; l0 += RB * NW) {
    T bl[RB], lo[RB], a0[RB], a1[RB], a2[RB];
#pragma unroll
    for (int i = 0; i < RB; ++i) {
      const int l = l0 + i * NW;
      bl[i] = lo[i] = a0[i] = a1[i] = a2[i] = 0;
      if (valid && l < nz) {
        const int64_t o = (int64_t)l * TW;
        bl[i] = (T)b[base + o];
        lo[i] = L.lo[base + o];
        if (MODE != MODE_ZERO) {
          a0[i] = u[s0 + o];
          a1[i] = u[s1 + o];
          a2[i] = u[s2 + o];
          if (MODE == MODE_PRO) {
            a0[i] += (T)ec[q0 + o];
            a1[i] += (T)ec[q1 + o];
            a2[i] += (T)ec[q2 + o];
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < RB; ++i) {
      const int l = l0 + i * NW;
      if (l < nz) {
        T r = bl[i];
        if (MODE != MODE_ZERO) {  // three FMAs: b + g0 u0 + g1 u1 + g2 u2
          r = fma(g.x, a0[i], r);
          r = fma(g.y, a1[i], r);
          r = fma(g.z, a2[i], r);
        }
        if (bcopy && valid) bcopy[base + (int64_t)l * TW] = (float)bl[i];
        R[l * TW + lane] = r;
        LOs[l * TW + lane] = lo[i];
      }
    }
  }
  __syncthreads();
  const int cw = blockIdx.x % NW;  // spread the chain warps over the sub-partitions
  // B
  if (warp == cw) {
    T y = 0;
    int l = 0;
    for (; l + 4 <= nz; l += 4) {
      T r0 = R[(l + 0) * TW + lane], r1 = R[(l + 1) * TW + lane], r2 = R[(l + 2) * TW + lane],
        r3 = R[(l + 3) * TW + lane];
      T m0 = LOs[(l + 0) * TW + lane], m1 = LOs[(l + 1) * TW + lane], m2 = LOs[(l + 2) * TW + lane],
        m3 = LOs[(l + 3) * TW + lane];
      y = r0 - m0 * y;
      R[(l + 0) * TW + lane] = y;
      y = r1 - m1 * y;
      R[(l + 1) * TW + lane] = y;
      y = r2 - m2 * y;
      R[(l + 2) * TW + lane] = y;
      y = r3 - m3 * y;
      R[(l + 3) * TW + lane] = y;
    }
    for (; l < nz; ++l) {
      y = R[l * TW + lane] - LOs[l * TW + lane] * y;
      R[l * TW + lane] = y;
    }
  }
  __syncthreads();
  // B'
  for (int l0 = warp; l0 < nz; l0 += RB * NW) {
    T wv[RB];
#pragma unroll
    for (int i = 0; i < RB; ++i) {
      const int l = l0 + i * NW;
      wv[i] = (l < nz) ? L.w[base + (int64_t)l * TW] : (T)0;
    }
#pragma unroll
    for (int i = 0; i < RB; ++i) {
      const int l = l0 + i * NW;
      if (l < nz) R[l * TW + lane] *= wv[i];
    }
  }
  __syncthreads();
  // C
  if (warp == cw) {
    T x = 0, lnext = 0;
    int l = nz - 1;
    for (; l - 3 >= 0; l -= 4) {
      T z0 = R[l * TW + lane], z1 = R[(l - 1) * TW + lane], z2 = R[(l - 2) * TW + lane],
        z3 = R[(l - 3) * TW + lane];
      T m0 = LOs[l * TW + lane], m1 = LOs[(l - 1) * TW + lane], m2 = LOs[(l - 2) * TW + lane],
        m3 = LOs[(l - 3) * TW + lane];
      x = z0 - lnext * x;
      R[l * TW + lane] = x;
      x = z1 - m0 * x;
      R[(l - 1) * TW + lane] = x;
      x = z2 - m1 * x;
      R[(l - 2) * TW + lane] = x;
      x = z3 - m2 * x;
      R[(l - 3) * TW + lane] = x;
      lnext = m3;
    }
    for (; l >= 0; --l) {
      T m = LOs[l * TW + lane];
      x = R[l * TW + lane] - lnext * x;
      R[l * TW + lane] = x;
      lnext = m;
    }
  }
  __syncthreads();
  // D
  double acc0 = 0.0, acc1 = 0.0;
  if (valid) {
    for (int l0 = warp; l0 < nz; l0 += RB * NW) {
      T uc[RB];
      if (MODE != MODE_ZERO) {
#pragma unroll
        for (int i = 0; i < RB; ++i) {
          const int l = l0 + i * NW;
          uc[i] = 0;
          if (l < nz) {
            uc[i] = u[base + (int64_t)l * TW];
            if (MODE == MODE_PRO) uc[i] += (T)ec[q + (int64_t)l * TW];
          }
        }
      }
      double dav[RB], dcv[RB];
      if (DOT) {
#pragma unroll
        for (int i = 0; i < RB; ++i) {
          const int l = l0 + i * NW;
          dav[i] = (l < nz) ? da[base + (int64_t)l * TW] : 0.0;
          dcv[i] = (DOT == 2 && l < nz) ? dc[base + (int64_t)l * TW] : 0.0;
        }
      }
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        const int l = l0 + i * NW;
        if (l < nz) {
          T xv = R[l * TW + lane];
          TO out = (MODE == MODE_ZERO) ? (TO)xv : (TO)(om1 * uc[i] + xv);
          uo[base + (int64_t)l * TW] = out;
          if (DOT) acc0 += dav[i] * (double)out;
          if (DOT == 2) acc1 += (double)out * dcv[i];
        }
      }
    }
  }
  if (DOT) grid_reduce2(acc0, acc1, red);
}

// ---------------------------------------------------------------- layer-parallel kernels
// A CTA of NW warps handles row group rg of tiles blockIdx.x / RG (grid-stride
// over tiles); warp w of row group rg handles the layers rg * NW + w + k * RG * NW;
// lane = column of the tile.  Large levels use RG = 1; small levels split each
// tile's rows over RG CTAs so that every warp has only a few rows.  No index
// division.

// u += P e_c (in place)
template <typename T, typename TE, int NW>
__global__ void __launch_bounds__(NW * 32)
k_tprolong(int nc, int nz, int ntiles, int RG, T* __restrict__ u, const TE* __restrict__ ec) {
  const int lane = threadIdx.x & 31;
  const int row0 = (blockIdx.x % RG) * NW + (threadIdx.x >> 5), rstep = RG * NW;
  for (int tile = blockIdx.x / RG; tile < ntiles; tile += gridDim.x / RG) {
    const int c = tile * TW + lane;
    if (c >= nc) continue;
    const int64_t base = (int64_t)tile * TW * nz + lane;
    const int64_t q = tile_base(c >> 2, nz);
#pragma unroll 4
    for (int l = row0; l < nz; l += rstep) u[base + (int64_t)l * TW] += (T)ec[q + (int64_t)l * TW];
  }
}

// acc + sgn (H^ x) at (column c, layer l) = tiled index t, as one FMA chain:
// sgn = +1 gives H^ x (acc = 0: one MUL and five FMAs), sgn = -1 with acc = b
// gives the residual b - H^ x in six FMAs.
template <typename T, int SGN>
__device__ __forceinline__ T stencil_acc(const LD<T>& L, const T* __restrict__ x, int64_t t, int l, T acc,
                                         const typename Vec4<T>::type& g, int64_t s0, int64_t s1, int64_t s2) {
  const int64_t o = (int64_t)l * TW;
  T y = (SGN > 0) ? L.d[t] * x[t] : fma(-L.d[t], x[t], acc);
  if (l > 0) y = fma((T)SGN * L.e[t], x[t - TW], y);
  if (l < L.nz - 1) y = fma((T)SGN * L.e[t + TW], x[t + TW], y);
  y = fma((T)(-SGN) * g.x, x[s0 + o], y);
  y = fma((T)(-SGN) * g.y, x[s1 + o], y);
  y = fma((T)(-SGN) * g.z, x[s2 + o], y);
  return y;
}

// b_c = P^T (b - H^ u): the children 4C..4C+3 of coarse column C are four
// adjacent lanes of one tile row, so the sum over them is two shuffles.
template <typename T, typename TC, int NW>
__global__ void __launch_bounds__(NW * 32)
k_tresid_restrict(LD<T> L, int ntiles, int RG, const T* __restrict__ b, const T* __restrict__ u,
                  TC* __restrict__ bc) {
  const int lane = threadIdx.x & 31;
  const int row0 = (blockIdx.x % RG) * NW + (threadIdx.x >> 5), rstep = RG * NW;
  const int nz = L.nz;
  for (int tile = blockIdx.x / RG; tile < ntiles; tile += gridDim.x / RG) {
    const int c = tile * TW + lane;
    const bool valid = c < L.nc;
    const int64_t base = (int64_t)tile * TW * nz + lane;
    typename Vec4<T>::type g{};
    int64_t s0 = 0, s1 = 0, s2 = 0, qc = 0;
    if (valid) {
      const int4 nb = L.nbr[c];
      g = L.gh[c];
      s0 = tile_base(nb.x, nz);
      s1 = tile_base(nb.y, nz);
      s2 = tile_base(nb.z, nz);
      qc = tile_base(c >> 2, nz);
    }
#pragma unroll 2
    for (int l = row0; l < nz; l += rstep) {
      const int64_t t = base + (int64_t)l * TW;
      T r = 0;
      if (valid) r = stencil_acc<T, -1>(L, u, t, l, b[t], g, s0, s1, s2);
      r += __shfl_xor_sync(0xffffffffu, r, 1);
      r += __shfl_xor_sync(0xffffffffu, r, 2);
      if ((lane & 3) == 0 && valid) bc[qc + (int64_t)l * TW] = (TC)r;
    }
  }
}

// y = H^ x; with DOT also x.y (the p.q of CG), reduced over the grid.
template <typename T, bool DOT, int NW>
__global__ void __launch_bounds__(NW * 32)
k_tapply(LD<T> L, int ntiles, int RG, const T* __restrict__ x, T* __restrict__ y, Reduce red) {
  const int lane = threadIdx.x & 31;
  const int row0 = (blockIdx.x % RG) * NW + (threadIdx.x >> 5), rstep = RG * NW;
  const int nz = L.nz;
  double acc = 0.0;
  for (int tile = blockIdx.x / RG; tile < ntiles; tile += gridDim.x / RG) {
    const int c = tile * TW + lane;
    const bool valid = c < L.nc;
    const int64_t base = (int64_t)tile * TW * nz + lane;
    typename Vec4<T>::type g{};
    int64_t s0 = 0, s1 = 0, s2 = 0;
    if (valid) {
      const int4 nb = L.nbr[c];
      g = L.gh[c];
      s0 = tile_base(nb.x, nz);
      s1 = tile_base(nb.y, nz);
      s2 = tile_base(nb.z, nz);
    }
#pragma unroll 2
    for (int l = row0; l < nz; l += rstep) {
      const int64_t t = base + (int64_t)l * TW;
      T v = 0;
      if (valid) v = stencil_acc<T, 1>(L, x, t, l, (T)0, g, s0, s1, s2);
      y[t] = v;
      if (DOT) acc += (double)x[t] * (double)v;
    }
  }
  if (DOT) grid_reduce2(acc, 0.0, red);
}

constexpr int NW_PAR = 8;
// Sweep CTA size: 4 warps while a level has more tiles than the GPU has SMs
// (several CTAs resident per SM keep the FP64 pipes busy, and all CTAs fit in
// one wave), 16 warps on smaller levels (latency bound: each warp loads only
// a few rows).
constexpr int NW_SWEEP_BIG = 4;
constexpr int NW_SWEEP_SMALL = 16;
constexpr int SMALL_LEVEL_TILES = 152;

inline int ntiles_of(const Level& L) { return L.ncp / TW; }

struct ParCfg {
  int grid, rg;
};
// Grid of the layer-parallel kernels: whole tiles on large levels, tiles split
// into row groups on small ones (RG * NW <= nz).
inline ParCfg par_cfg(const Level& L) {
  const int nt = ntiles_of(L);
  const int cap = 152 * 8;
  if (nt >= cap) return {cap, 1};
  int rg = 1;
  while (rg * 2 * NW_PAR <= L.nz && nt * rg * 2 <= cap) rg *= 2;
  return {nt * rg, rg};
}

template <typename K>
void allow_smem(K kern, size_t smem, size_t& configured) {
  if (smem > 48 * 1024 && configured < smem) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = smem;
  }
}

template <typename T, typename TB, typename TO, int MODE, typename TE, int NW, int DOT>
void tsweep_nw(const Level& L, const void* b, const void* u, void* uo, const void* ec, float* bcopy, double omega,
               const SweepDot* dot, cudaStream_t s) {
  auto kern = k_tsweep<T, TB, TO, MODE, TE, NW, DOT>;
  const size_t smem = 2 * (size_t)L.nz * TW * sizeof(T);
  static size_t configured = 0;
  allow_smem(kern, smem, configured);
  Reduce red = dot ? dot->red : Reduce{};
  kern<<<ntiles_of(L), NW * 32, smem, s>>>(view<T>(L), (const TB*)b, (const T*)u, (TO*)uo, (const TE*)ec, bcopy,
                                          (T)(1.0 - omega), dot ? dot->a : nullptr, dot ? dot->c : nullptr, red);
}

template <typename T, typename TB, typename TO, int MODE, typename TE, int NW>
void tsweep_dot(const Level& L, const void* b, const void* u, void* uo, const void* ec, float* bcopy, double omega,
                const SweepDot* dot, cudaStream_t s) {
  if (!dot) tsweep_nw<T, TB, TO, MODE, TE, NW, 0>(L, b, u, uo, ec, bcopy, omega, dot, s);
  else if (!dot->c) tsweep_nw<T, TB, TO, MODE, TE, NW, 1>(L, b, u, uo, ec, bcopy, omega, dot, s);
  else tsweep_nw<T, TB, TO, MODE, TE, NW, 2>(L, b, u, uo, ec, bcopy, omega, dot, s);
}

template <typename T, typename TB, typename TO, int MODE, typename TE>
void tsweep(const Level& L, const void* b, const void* u, void* uo, const void* ec, float* bcopy, double omega,
            cudaStream_t s, const SweepDot* dot = nullptr) {
  if (ntiles_of(L) > SMALL_LEVEL_TILES)
    tsweep_dot<T, TB, TO, MODE, TE, NW_SWEEP_BIG>(L, b, u, uo, ec, bcopy, omega, dot, s);
  else
    tsweep_dot<T, TB, TO, MODE, TE, NW_SWEEP_SMALL>(L, b, u, uo, ec, bcopy, omega, dot, s);
}

}  // namespace

void launch_sweep0(const Level& L, int dt, const void* b, int b_dt, void* u, float* bcopy, double omega,
                   cudaStream_t s) {
  if (dt == HMG_FP64)
    tsweep<double, double, double, MODE_ZERO, double>(L, b, nullptr, u, nullptr, nullptr, omega, s);
  else if (b_dt == HMG_FP64)
    tsweep<float, double, float, MODE_ZERO, float>(L, b, nullptr, u, nullptr, bcopy, omega, s);
  else
    tsweep<float, float, float, MODE_ZERO, float>(L, b, nullptr, u, nullptr, nullptr, omega, s);
}

void launch_sweep(const Level& L, int dt, const void* b, const void* u, void* uo, int uo_dt, const void* ec,
                  int ec_dt, double omega, const SweepDot* dot, cudaStream_t s) {
  if (dt == HMG_FP64) {
    if (ec) tsweep<double, double, double, MODE_PRO, double>(L, b, u, uo, ec, nullptr, omega, s, dot);
    else tsweep<double, double, double, MODE_PLAIN, double>(L, b, u, uo, nullptr, nullptr, omega, s, dot);
    return;
  }
  const bool out64 = uo_dt == HMG_FP64;
  if (!ec) {
    if (out64) tsweep<float, float, double, MODE_PLAIN, float>(L, b, u, uo, nullptr, nullptr, omega, s, dot);
    else tsweep<float, float, float, MODE_PLAIN, float>(L, b, u, uo, nullptr, nullptr, omega, s, dot);
  } else if (ec_dt == HMG_FP64) {
    if (out64) tsweep<float, float, double, MODE_PRO, double>(L, b, u, uo, ec, nullptr, omega, s, dot);
    else tsweep<float, float, float, MODE_PRO, double>(L, b, u, uo, ec, nullptr, omega, s, dot);
  } else {
    if (out64) tsweep<float, float, double, MODE_PRO, float>(L, b, u, uo, ec, nullptr, omega, s, dot);
    else tsweep<float, float, float, MODE_PRO, float>(L, b, u, uo, ec, nullptr, omega, s, dot);
  }
}

void launch_prolong(const Level& L, int dt, void* u, const void* ec, int ec_dt, cudaStream_t s) {
  const ParCfg pc = par_cfg(L);
  const int nt = ntiles_of(L);
  if (dt == HMG_FP64)
    k_tprolong<double, double, NW_PAR><<<pc.grid, NW_PAR * 32, 0, s>>>(L.nc, L.nz, nt, pc.rg, (double*)u,
                                                                      (const double*)ec);
  else if (ec_dt == HMG_FP64)
    k_tprolong<float, double, NW_PAR><<<pc.grid, NW_PAR * 32, 0, s>>>(L.nc, L.nz, nt, pc.rg, (float*)u,
                                                                     (const double*)ec);
  else
    k_tprolong<float, float, NW_PAR><<<pc.grid, NW_PAR * 32, 0, s>>>(L.nc, L.nz, nt, pc.rg, (float*)u,
                                                                    (const float*)ec);
}

void launch_resid_restrict(const Level& L, int dt, const void* b, const void* u, void* bc, int bc_dt,
                           cudaStream_t s) {
  const ParCfg pc = par_cfg(L);
  const int nt = ntiles_of(L), g = pc.grid, rg = pc.rg;
  if (dt == HMG_FP64)
    k_tresid_restrict<double, double, NW_PAR><<<g, NW_PAR * 32, 0, s>>>(view<double>(L), nt, rg, (const double*)b,
                                                                        (const double*)u, (double*)bc);
  else if (bc_dt == HMG_FP64)
    k_tresid_restrict<float, double, NW_PAR><<<g, NW_PAR * 32, 0, s>>>(view<float>(L), nt, rg, (const float*)b,
                                                                       (const float*)u, (double*)bc);
  else
    k_tresid_restrict<float, float, NW_PAR><<<g, NW_PAR * 32, 0, s>>>(view<float>(L), nt, rg, (const float*)b,
                                                                      (const float*)u, (float*)bc);
}

void launch_apply(const Level& L, int dt, const void* x, void* y, const Reduce* red, cudaStream_t s) {
  const ParCfg pc = par_cfg(L);
  const int nt = ntiles_of(L), g = pc.grid, rg = pc.rg;
  Reduce none{};
  if (dt == HMG_FP64) {
    if (red)
      k_tapply<double, true, NW_PAR><<<g, NW_PAR * 32, 0, s>>>(view<double>(L), nt, rg, (const double*)x, (double*)y,
                                                                *red);
    else
      k_tapply<double, false, NW_PAR><<<g, NW_PAR * 32, 0, s>>>(view<double>(L), nt, rg, (const double*)x, (double*)y,
                                                                 none);
  } else {
    if (red)
      k_tapply<float, true, NW_PAR><<<g, NW_PAR * 32, 0, s>>>(view<float>(L), nt, rg, (const float*)x, (float*)y, *red);
    else
      k_tapply<float, false, NW_PAR><<<g, NW_PAR * 32, 0, s>>>(view<float>(L), nt, rg, (const float*)x, (float*)y,
                                                                none);
  }
}

}  // namespace hmg
