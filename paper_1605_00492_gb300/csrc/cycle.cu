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
#include "convert.cuh"
#include "hmg_internal.h"
#include "reduce.cuh"

#include <cooperative_groups.h>
#include <type_traits>

namespace cg = cooperative_groups;

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
  const T* __restrict__ mt;   // per column: mu of the twist row
  int twist;                  // twist row m of the column factorisation
  const T* __restrict__ los;  // FP64: multipliers scaled to their row's pivot (e / D)
  const T* __restrict__ mts;  // FP64: the twist row's mu scaled the same way
};

template <typename T> LD<T> view(const Level& L);
template <> LD<double> view<double>(const Level& L) {
  return LD<double>{L.nc, L.nz, L.Np, L.nbr, L.gh, L.d, L.e, L.lo, L.w, L.mt, L.twist, L.los, L.mts};
}
template <> LD<float> view<float>(const Level& L) {
  return LD<float>{L.nc, L.nz, L.Np, L.nbr, L.gh32, L.d32, L.e32, L.lo32, L.w32, L.mt32, L.twist32, nullptr,
                   nullptr};
}

__device__ __forceinline__ int64_t tile_base(int c, int nz) {
  return (int64_t)(c >> 5) * (TW * nz) + (c & 31);
}

// ---------------------------------------------------------------- sweeps
//
// One CTA per tile of 32 columns, NW warps, shared arrays of nz x 32.
// Twisted solve (twist row m of the level):
//   A  (all warps, layer parallel)  R = b + sum_k g_k u[nbr_k]   (u~ with PRO),
//                                   LO = multipliers of N D N^T, and W
//   B  (two warps: lane = column)   elimination N y = R: rows 0..m-1 top-down
//                                   on one warp, rows nz-1..m+1 bottom-up on
//                                   another, each row stored as z_l = (omega / D_l) y_l
//   C  (the same two warps)         both complete the twist row,
//                                   x_m = (omega / D_m)(R_m - lambda_m y_m-1 - mu_m y_m+1),
//                                   then substitute N^T x = z outwards from row m
//   D  (all warps)                  u' = (1 - omega) u~ + x
// In FP64, W holds the multipliers scaled to their own row's pivot and A
// scales R by omega / D, so B eliminates directly in z with one FMA per row;
// in FP32, W = omega / D and B scales each y as it completes.
// Plain L D L^T (twist row nz - 1, FP32 levels only): one chain warp, and the
// scaling by omega / D is a layer-parallel phase B' between B and C.
// Only the recurrences are sequential, and they read shared memory, so they
// never wait for global memory; everything else is spread over the CTA.
// MODE_ZERO is the first pre-smoothing step (u = 0): no neighbour sum and no
// relaxation term.
enum { MODE_ZERO = 0, MODE_PLAIN = 1, MODE_PRO = 2 };

// count steps of y <- R[l] - LO[l + mshift] y; R[l] = y at l = l0, l0 + step,
// ...; shared-memory loads are issued four steps ahead of the dependent FMAs.
template <typename T>
__device__ __forceinline__ T chain(T* R, const T* LO, int lane, int l0, int step, int mshift, int count, T y) {
  int k = 0;
  for (; k + 4 <= count; k += 4) {
    const int la = l0 + k * step, lb = la + step, lc = lb + step, ld = lc + step;
    const T r0 = R[la * TW + lane], r1 = R[lb * TW + lane], r2 = R[lc * TW + lane], r3 = R[ld * TW + lane];
    const T m0 = LO[(la + mshift) * TW + lane], m1 = LO[(lb + mshift) * TW + lane],
            m2 = LO[(lc + mshift) * TW + lane], m3 = LO[(ld + mshift) * TW + lane];
    y = fma(-m0, y, r0);
    R[la * TW + lane] = y;
    y = fma(-m1, y, r1);
    R[lb * TW + lane] = y;
    y = fma(-m2, y, r2);
    R[lc * TW + lane] = y;
    y = fma(-m3, y, r3);
    R[ld * TW + lane] = y;
  }
  for (; k < count; ++k) {
    const int l = l0 + k * step;
    y = fma(-LO[(l + mshift) * TW + lane], y, R[l * TW + lane]);
    R[l * TW + lane] = y;
  }
  return y;
}

// count steps of y <- R[l] - LO[l] y with R[l] = W[l] y stored (the row
// scaled by omega / D_l as soon as it is eliminated); returns the last y,
// unscaled.  Shared-memory loads are issued four steps ahead.
template <typename T>
__device__ __forceinline__ T chain_scaled(T* R, const T* LO, const T* W, int lane, int l0, int step, int count,
                                          T y) {
  int k = 0;
  for (; k + 4 <= count; k += 4) {
    const int la = l0 + k * step, lb = la + step, lc = lb + step, ld = lc + step;
    const T r0 = R[la * TW + lane], r1 = R[lb * TW + lane], r2 = R[lc * TW + lane], r3 = R[ld * TW + lane];
    const T m0 = LO[la * TW + lane], m1 = LO[lb * TW + lane], m2 = LO[lc * TW + lane], m3 = LO[ld * TW + lane];
    const T w0 = W[la * TW + lane], w1 = W[lb * TW + lane], w2 = W[lc * TW + lane], w3 = W[ld * TW + lane];
    const T y0 = fma(-m0, y, r0);
    const T y1 = fma(-m1, y0, r1);
    const T y2 = fma(-m2, y1, r2);
    y = fma(-m3, y2, r3);
    R[la * TW + lane] = w0 * y0;
    R[lb * TW + lane] = w1 * y1;
    R[lc * TW + lane] = w2 * y2;
    R[ld * TW + lane] = w3 * y;
  }
  for (; k < count; ++k) {
    const int l = l0 + k * step;
    y = fma(-LO[l * TW + lane], y, R[l * TW + lane]);
    R[l * TW + lane] = W[l * TW + lane] * y;
  }
  return y;
}

// Spare shared rows after R of the tile sweep: y_m-1, y_m+1 (and, twisted,
// R_m, mu_m and the scaled mu_m).  The twisted solve also stages a third
// nz x 32 array: omega / D (FP32) or the scaled multipliers (FP64).
__host__ __device__ constexpr int tsweep_spare_rows(bool twisted) { return twisted ? 5 : 2; }
__host__ __device__ constexpr int tsweep_arrays(bool twisted) { return twisted ? 3 : 2; }

// DOT = 1: also reduce sum_cells da * u' (the r.z of CG, da = the FP64
// residual); DOT = 2: and sum_cells u' * dc (the z.q of flexible CG).
// The sweep of one tile by the whole CTA (NW warps); k_tsweep runs it with
// tile = blockIdx.x, the fused coarse-level cycle (k_coarse_cycle) for the
// tiles its CTA owns in each sweep phase.
template <typename T, typename TB, typename TO, int MODE, typename TE, int NW, int DOT, bool TW2>
__device__ __forceinline__ void tsweep_tile(const LD<T>& L, const int tile, const TB* __restrict__ b,
                                            const T* __restrict__ u, TO* __restrict__ uo,
                                            const TE* __restrict__ ec, float* __restrict__ bcopy, T om1,
                                            const double* __restrict__ da, const double* __restrict__ dc,
                                            const Reduce& red) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int RB = 4;  // rows per warp per batch: their loads are issued together
  const int nz = L.nz;
  // shared: R[nz][32], spare rows (plain: y_m-1, y_m+1; twisted: y_m-1,
  // y_m+1, R_m, mu_m, scaled mu_m), LO[nz][32], and for the twisted solve a
  // third array W[nz][32]: omega / D (FP32) or the scaled multipliers (FP64)
  T* R = reinterpret_cast<T*>(smem_raw);
  T* LOs = R + (nz + tsweep_spare_rows(TW2)) * TW;
  T* Ws = LOs + nz * TW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
  // Small levels (TW2) where one batch of RB rows per warp covers the column
  // (nz <= RB * NW): phase A also loads u~ for phase D, so the CTA waits for
  // global memory once instead of twice.  (The twisted solve always stages
  // its third array in shared memory in phase A.)
  const bool carry = TW2 && nz <= RB * NW;
  T uc_c[RB];
#pragma unroll
  for (int i = 0; i < RB; ++i) uc_c[i] = 0;
  // FP64 twisted solve: the elimination runs in z = (omega / D) y with the
  // scaled multipliers, so R is scaled once here and the recurrence is one FMA
  constexpr bool SC = TW2 && std::is_same<T, double>::value;
  if (TW2 && warp == 0) {
    R[(nz + 3) * TW + lane] = valid ? L.mt[c] : (T)0;
    if (SC) R[(nz + 4) * TW + lane] = valid ? L.mts[c] : (T)0;
  }
  // A
  for (int l0 = warp; l0 < nz; l0 += RB * NW) {
    T bl[RB], lo[RB], a0[RB], a1[RB], a2[RB], wl[RB], ls[RB];
#pragma unroll
    for (int i = 0; i < RB; ++i) {
      const int l = l0 + i * NW;
      bl[i] = lo[i] = a0[i] = a1[i] = a2[i] = wl[i] = ls[i] = 0;
      if (valid && l < nz) {
        const int64_t o = (int64_t)l * TW;
        bl[i] = cvt<T>(b[base + o]);
        lo[i] = L.lo[base + o];
        if (TW2) wl[i] = L.w[base + o];
        if (SC) ls[i] = L.los[base + o];
        if (TW2 && carry && MODE != MODE_ZERO) {
          uc_c[i] = u[base + o];
          if (MODE == MODE_PRO) uc_c[i] += cvt<T>(ec[q + o]);
        }
        if (MODE != MODE_ZERO) {
          a0[i] = u[s0 + o];
          a1[i] = u[s1 + o];
          a2[i] = u[s2 + o];
          if (MODE == MODE_PRO) {
            a0[i] += cvt<T>(ec[q0 + o]);
            a1[i] += cvt<T>(ec[q1 + o]);
            a2[i] += cvt<T>(ec[q2 + o]);
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
        // the FP32 copy of an FP64 right-hand side exists only on FP32
        // levels; for FP64 levels the conversion is compiled out, so it can
        // never be executed speculatively on the FP64 pipe
        if constexpr (std::is_same<T, float>::value && std::is_same<TB, double>::value) {
          if (bcopy && valid) bcopy[base + (int64_t)l * TW] = (float)bl[i];
        }
        if (SC) r *= wl[i];
        R[l * TW + lane] = r;
        LOs[l * TW + lane] = lo[i];
        if (TW2) {
          Ws[l * TW + lane] = SC ? ls[i] : wl[i];
          if (l == L.twist) R[(nz + 2) * TW + lane] = r;
        }
      }
    }
  }
  __syncthreads();
  if (!TW2) {
    // one chain warp (plain L D L^T: twist row nz - 1), spread over the sub-partitions
    const int cw = tile % NW;
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
        T mm = LOs[l * TW + lane];
        x = R[l * TW + lane] - lnext * x;
        R[l * TW + lane] = x;
        lnext = mm;
      }
    }
    __syncthreads();
  } else {
    // two chain warps on different sub-partitions, spread over the CTAs
    const int cw0 = tile % NW, cw1 = (cw0 + 1) % NW;
    const int m = L.twist;
    T* YT = R + nz * TW;    // y_m-1 and y_m+1 for the twist row (FP64: z_m-1, z_m+1)
    T* YB = YT + TW;
    const T* RM = YB + TW;  // R_m, kept apart from R[m], which becomes x_m
    const T* MT = RM + TW;  // mu_m
    const T* MTS = MT + TW; // mu_m scaled (FP64)
    // B: elimination, each row stored as z = W y: FP64 eliminates the scaled
    // R with the scaled multipliers (one FMA a row), FP32 scales y as it goes
    if (warp == cw0) {
      T y = SC ? chain<T>(R, Ws, lane, 0, +1, 0, m, (T)0) : chain_scaled<T>(R, LOs, Ws, lane, 0, +1, m, (T)0);
      YT[lane] = y;
    } else if (warp == cw1) {
      T y = SC ? chain<T>(R, Ws, lane, nz - 1, -1, 0, nz - 1 - m, (T)0)
               : chain_scaled<T>(R, LOs, Ws, lane, nz - 1, -1, nz - 1 - m, (T)0);
      YB[lane] = y;
    }
    __syncthreads();
    // C: both chain warps complete the twist row,
    // x_m = (omega / D_m)(R_m - lambda_m y_m-1 - mu_m y_m+1)  (FP64: from z_m-1,
    // z_m+1 and the scaled multipliers), and substitute outwards
    if (warp == cw0 || warp == cw1) {
      const T mtv = MT[lane];
      const T xm = SC ? fma(-MTS[lane], YB[lane], fma(-Ws[m * TW + lane], YT[lane], RM[lane]))
                      : Ws[m * TW + lane] * fma(-mtv, YB[lane], fma(-LOs[m * TW + lane], YT[lane], RM[lane]));
      if (warp == cw0) {
        R[m * TW + lane] = xm;
        chain<T>(R, LOs, lane, m - 1, -1, +1, m, xm);
      } else if (m + 1 < nz) {
        T x = R[(m + 1) * TW + lane] - mtv * xm;
        R[(m + 1) * TW + lane] = x;
        chain<T>(R, LOs, lane, m + 2, +1, -1, nz - 2 - m, x);
      }
    }
    __syncthreads();
  }
  // D (one accumulator per row of a batch: no dependent FP64 chain)
  double acc0[RB], acc1[RB];
#pragma unroll
  for (int i = 0; i < RB; ++i) acc0[i] = acc1[i] = 0.0;
  if (valid) {
    for (int l0 = warp; l0 < nz; l0 += RB * NW) {
      T uc[RB];
      if (MODE != MODE_ZERO) {
#pragma unroll
        for (int i = 0; i < RB; ++i) {
          const int l = l0 + i * NW;
          uc[i] = 0;
          if (carry) {
            uc[i] = uc_c[i];
          } else if (l < nz) {
            uc[i] = u[base + (int64_t)l * TW];
            if (MODE == MODE_PRO) uc[i] += cvt<T>(ec[q + (int64_t)l * TW]);
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
          TO out = (MODE == MODE_ZERO) ? cvt<TO>(xv) : cvt<TO>(om1 * uc[i] + xv);
          uo[base + (int64_t)l * TW] = out;
          if (DOT) acc0[i] = fma(dav[i], (double)out, acc0[i]);
          if (DOT == 2) acc1[i] = fma((double)out, dcv[i], acc1[i]);
        }
      }
    }
  }
  if (DOT) {
    double a0 = 0.0, a1 = 0.0;
#pragma unroll
    for (int i = 0; i < RB; ++i) {
      a0 += acc0[i];
      a1 += acc1[i];
    }
    // the tile's shared arrays are free now: reuse them as scratch
    grid_reduce<(DOT == 2 ? 2 : 1)>(a0, a1, red, reinterpret_cast<double*>(smem_raw));
  }
}

template <typename T, typename TB, typename TO, int MODE, typename TE, int NW, int DOT, bool TW2>
__global__ void __launch_bounds__(NW * 32)
k_tsweep(LD<T> L, const TB* __restrict__ b, const T* __restrict__ u, TO* __restrict__ uo,
         const TE* __restrict__ ec, float* __restrict__ bcopy, T om1, const double* __restrict__ da,
         const double* __restrict__ dc, Reduce red) {
  tsweep_tile<T, TB, TO, MODE, TE, NW, DOT, TW2>(L, blockIdx.x, b, u, uo, ec, bcopy, om1, da, dc, red);
}

// ---------------------------------------------------------------- FP64 half-column sweep
//
// FP64 levels.  The FP64 pipe issues one warp instruction per 64 cycles per
// SM sub-partition, and a dependent FMA is ready exactly when the next may
// issue, so one warp whose operands are in registers keeps a sub-partition's
// pipe busy on its own.  Here each tile is relaxed by a pair of warps, one
// per half of the twisted factorisation N D N^T of H^_z (twist row m): the
// top warp eliminates rows 0..m-1 downwards, the bottom warp rows nz-1..m+1
// upwards, lane = column.  A row's right-hand side R = b + sum_k g_k u~[nbr_k]
// is formed as the row is eliminated, from loads issued RB rows at a time,
// and the unscaled y_l is parked in the row's output cell (each lane reads
// back only what it wrote; uo is never u).  The pair swaps y_m-1, y_m+1 and
// R_m through shared memory at one 64-thread named barrier, both warps
// complete the twist row, x_m = (omega / D_m)(R_m - lambda_m y_m-1 - mu_m y_m+1),
// and each substitutes outwards through its half, scaling by omega / D_l and
// relaxing, u' = (1 - omega) u~ + x, as it goes.  The recurrences never touch
// shared memory, and no CTA-wide barrier holds a warp.  Two tiles per CTA.
//
// u~ = u, or u + P e_c with the coarse correction e_c (MODE_PRO); MODE_ZERO
// relaxes from u = 0.  DOT as in tsweep_tile.
template <int MODE, int DOT, int RB, int MINB>
__global__ void __launch_bounds__(128, MINB)
k_hsweep(LD<double> L, int ntiles, const double* __restrict__ b, const double* __restrict__ u,
         double* __restrict__ uo, const double* __restrict__ ec, double om1, const double* __restrict__ da,
         const double* __restrict__ dc, Reduce red) {
  constexpr int TPB = 2;
  __shared__ double xch[TPB][3][TW];   // y_m-1, y_m+1, R_m of each tile
  __shared__ double scratch[DOT ? 2 * TPB * 64 : 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int pair = warp >> 1, half = warp & 1;
  const int tile = blockIdx.x * TPB + pair;
  const int nz = L.nz, m = L.twist;
  const int c = tile * TW + lane;
  const bool valid = tile < ntiles && c < L.nc;
  const int64_t base = (int64_t)tile * TW * nz + lane;
  int64_t s0 = 0, s1 = 0, s2 = 0, q = 0, q0 = 0, q1 = 0, q2 = 0;
  double4_32a g{};
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
  // rows of this half before the twist row, walked away from the ends
  const int cnt = half ? nz - 1 - m : m;
  const int64_t st = half ? -(int64_t)TW : (int64_t)TW;
  const int64_t o0 = half ? (int64_t)(nz - 1) * TW : 0;
  // Both passes are software pipelined: the loads of the next RB rows are
  // issued before the arithmetic of the current ones, and a row's store is
  // issued one batch later, when its value is long ready (the FP64 result of
  // a recurrence would otherwise hold up the warp's in-order issue).
  double y = 0.0;
  if (valid) {
    double cb[RB], cl[RB], c0[RB], c1[RB], c2[RB], ys[RB];
    auto fload = [&](int k, double (&xb)[RB], double (&xl)[RB], double (&x0)[RB], double (&x1)[RB],
                     double (&x2)[RB]) {
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        xb[i] = xl[i] = x0[i] = x1[i] = x2[i] = 0.0;
        if (k + i < cnt) {
          const int64_t o = o0 + (k + i) * st;
          xb[i] = b[base + o];
          xl[i] = L.lo[base + o];
          if (MODE != MODE_ZERO) {
            x0[i] = u[s0 + o];
            x1[i] = u[s1 + o];
            x2[i] = u[s2 + o];
            if (MODE == MODE_PRO) {
              x0[i] += ec[q0 + o];
              x1[i] += ec[q1 + o];
              x2[i] += ec[q2 + o];
            }
          }
        }
      }
    };
    fload(0, cb, cl, c0, c1, c2);
#pragma unroll
    for (int i = 0; i < RB; ++i) ys[i] = 0.0;
    int k = 0;
    for (; k < cnt; k += RB) {
      double nb[RB], nl[RB], n0[RB], n1[RB], n2[RB];
      fload(k + RB, nb, nl, n0, n1, n2);
      if (k > 0) {
#pragma unroll
        for (int i = 0; i < RB; ++i) uo[base + o0 + (k - RB + i) * st] = ys[i];
      }
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        double r = cb[i];
        if (MODE != MODE_ZERO) {
          r = fma(g.x, c0[i], r);
          r = fma(g.y, c1[i], r);
          r = fma(g.z, c2[i], r);
        }
        if (k + i < cnt) y = fma(-cl[i], y, r);
        ys[i] = y;
      }
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        cb[i] = nb[i];
        cl[i] = nl[i];
        c0[i] = n0[i];
        c1[i] = n1[i];
        c2[i] = n2[i];
      }
    }
    if (k > 0) {
#pragma unroll
      for (int i = 0; i < RB; ++i)
        if (k - RB + i < cnt) uo[base + o0 + (k - RB + i) * st] = ys[i];
    }
  }
  // the twist row: R_m from the top warp, y_m-1 / y_m+1 from each side
  const int64_t om = (int64_t)m * TW;
  if (half == 0) {
    double r = 0.0;
    if (valid) {
      r = b[base + om];
      if (MODE != MODE_ZERO) {
        double a0 = u[s0 + om], a1 = u[s1 + om], a2 = u[s2 + om];
        if (MODE == MODE_PRO) {
          a0 += ec[q0 + om];
          a1 += ec[q1 + om];
          a2 += ec[q2 + om];
        }
        r = fma(g.x, a0, r);
        r = fma(g.y, a1, r);
        r = fma(g.z, a2, r);
      }
    }
    xch[pair][2][lane] = r;
    xch[pair][0][lane] = y;
  } else {
    xch[pair][1][lane] = y;
  }
  if (pair == 0) asm volatile("barrier.sync 1, 64;" ::: "memory");
  else asm volatile("barrier.sync 2, 64;" ::: "memory");
  double acc0 = 0.0, acc1 = 0.0;
  if (valid) {
    const double lam = L.lo[base + om], wm = L.w[base + om], mu = L.mt[c];
    const double ym = fma(-mu, xch[pair][1][lane], fma(-lam, xch[pair][0][lane], xch[pair][2][lane]));
    double x = wm * ym;
    if (half == 0) {   // the top warp writes the twist row
      double ut = 0.0;
      if (MODE != MODE_ZERO) {
        ut = u[base + om];
        if (MODE == MODE_PRO) ut += ec[q + om];
      }
      const double out = (MODE == MODE_ZERO) ? x : fma(om1, ut, x);
      uo[base + om] = out;
      if (DOT) acc0 = fma(da[base + om], out, acc0);
      if (DOT == 2) acc1 = fma(out, dc[base + om], acc1);
    }
    // outwards from the twist row: rows m-1..0 (top), m+1..nz-1 (bottom);
    // the first multiplier is lambda_m (top) or mu_m (bottom)
    double mprev = half ? mu : lam;
    const int64_t bst = -st, b0 = om + bst;
    double cy[RB], cw[RB], cl[RB], cu[RB], ca[RB], cc[RB], outs[RB];
    auto bload = [&](int k, double (&xy)[RB], double (&xw)[RB], double (&xl)[RB], double (&xu)[RB],
                     double (&xa)[RB], double (&xc)[RB]) {
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        xy[i] = xw[i] = xl[i] = xu[i] = xa[i] = xc[i] = 0.0;
        if (k + i < cnt) {
          const int64_t o = b0 + (k + i) * bst;
          xy[i] = uo[base + o];
          xw[i] = L.w[base + o];
          xl[i] = L.lo[base + o];
          if (MODE != MODE_ZERO) {
            xu[i] = u[base + o];
            if (MODE == MODE_PRO) xu[i] += ec[q + o];
          }
          if (DOT) xa[i] = da[base + o];
          if (DOT == 2) xc[i] = dc[base + o];
        }
      }
    };
    bload(0, cy, cw, cl, cu, ca, cc);
#pragma unroll
    for (int i = 0; i < RB; ++i) outs[i] = 0.0;
    int k = 0;
    for (; k < cnt; k += RB) {
      double ny[RB], nw[RB], nl[RB], nu[RB], na[RB], nc[RB];
      bload(k + RB, ny, nw, nl, nu, na, nc);
      if (k > 0) {
#pragma unroll
        for (int i = 0; i < RB; ++i) uo[base + b0 + (k - RB + i) * bst] = outs[i];
      }
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        if (k + i < cnt) {
          x = fma(-mprev, x, cw[i] * cy[i]);
          mprev = cl[i];
          const double out = (MODE == MODE_ZERO) ? x : fma(om1, cu[i], x);
          outs[i] = out;
          if (DOT) acc0 = fma(ca[i], out, acc0);
          if (DOT == 2) acc1 = fma(out, cc[i], acc1);
        }
      }
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        cy[i] = ny[i];
        cw[i] = nw[i];
        cl[i] = nl[i];
        cu[i] = nu[i];
        ca[i] = na[i];
        cc[i] = nc[i];
      }
    }
    if (k > 0) {
#pragma unroll
      for (int i = 0; i < RB; ++i)
        if (k - RB + i < cnt) uo[base + b0 + (k - RB + i) * bst] = outs[i];
    }
  }
  if (DOT) grid_reduce<(DOT == 2 ? 2 : 1)>(acc0, acc1, red, scratch);
}

// ---------------------------------------------------------------- FP32 staged sweep
//
// FP32 cycle (HBM bound): the tile's whole input is copied to shared memory
// with asynchronous copies issued at once (16-byte copies of the tile's
// contiguous rows of b, lo, w, u; 4-byte copies of the neighbour columns of
// u), so a CTA waits for memory once instead of once per phase; the phases
// then run from shared memory as in k_tsweep.  Padding columns copy zeros
// (their neighbours are themselves and their coefficients are zero).
// MODE_ZERO or MODE_PLAIN only (the prolongation is a pass of its own).  Used
// on small levels: with 4-CTA-per-SM occupancy it loses to k_tsweep on large
// ones.

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

template <int NTH>
__device__ __forceinline__ void stage_rows(void* dst, const void* src, int bytes) {
  for (int off = (int)threadIdx.x * 16; off < bytes; off += NTH * 16)
    cp_async16(static_cast<char*>(dst) + off, static_cast<const char*>(src) + off);
}

template <typename TB, typename TO, int MODE, int NW, int DOT, bool TW2>
__global__ void __launch_bounds__(NW * 32)
k_asweep(LD<float> L, const TB* __restrict__ b, const float* __restrict__ u, TO* __restrict__ uo,
         float* __restrict__ bcopy, float om1, const double* __restrict__ da, const double* __restrict__ dc,
         Reduce red) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nz = L.nz;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tile = blockIdx.x;
  const int c = tile * TW + lane;
  const bool valid = c < L.nc;
  const int cells = nz * TW;
  const int64_t tb = (int64_t)tile * cells;   // first element of the tile
  const int64_t base = tb + lane;
  // shared: Bs (TB), LOs, Ws, [Us, N0 (= R), N1, N2] (float), R for MODE_ZERO, 2 twist rows
  TB* Bs = reinterpret_cast<TB*>(smem_raw);
  float* LOs = reinterpret_cast<float*>(Bs + cells);
  float* Ws = LOs + cells;
  float* Us = Ws + cells;
  float* N0 = Us + cells;
  float* N1 = N0 + cells;
  float* N2 = N1 + cells;
  float* R = (MODE == MODE_ZERO) ? Us : N0;
  float* YT = R + cells;  // MODE_ZERO: the 2 rows after R; otherwise rows after N2
  if (MODE != MODE_ZERO) YT = N2 + cells;
  float* YB = YT + TW;

  stage_rows<NW * 32>(Bs, b + tb, cells * (int)sizeof(TB));
  stage_rows<NW * 32>(LOs, L.lo + tb, cells * 4);
  stage_rows<NW * 32>(Ws, L.w + tb, cells * 4);
  typename Vec4<float>::type g{};
  if (MODE != MODE_ZERO) {
    stage_rows<NW * 32>(Us, u + tb, cells * 4);
    const int4 nb = L.nbr[c];
    g = L.gh[c];
    const int64_t s0 = tile_base(nb.x, nz), s1 = tile_base(nb.y, nz), s2 = tile_base(nb.z, nz);
    for (int l = warp; l < nz; l += NW) {
      const int64_t o = (int64_t)l * TW;
      cp_async4(N0 + l * TW + lane, u + s0 + o);
      cp_async4(N1 + l * TW + lane, u + s1 + o);
      cp_async4(N2 + l * TW + lane, u + s2 + o);
    }
  }
  const float mtv = valid ? L.mt[c] : 0.f;
  cp_async_wait_all();
  __syncthreads();
  // A: R = b + g0 u0 + g1 u1 + g2 u2 (in place over N0, or over Us for MODE_ZERO)
  for (int l = warp; l < nz; l += NW) {
    const int i = l * TW + lane;
    float r = cvt<float>(Bs[i]);
    if (bcopy && valid) bcopy[base + (int64_t)l * TW] = r;
    if (MODE != MODE_ZERO) {
      r = fmaf(g.x, N0[i], r);
      r = fmaf(g.y, N1[i], r);
      r = fmaf(g.z, N2[i], r);
    }
    R[i] = r;
  }
  __syncthreads();
  const int m = L.twist;
  if (!TW2) {
    const int cw = blockIdx.x % NW;
    if (warp == cw) chain<float>(R, LOs, lane, 0, +1, 0, nz, 0.f);
  } else {
    const int cw0 = blockIdx.x % NW, cw1 = (cw0 + 1) % NW;
    if (warp == cw0) YT[lane] = chain<float>(R, LOs, lane, 0, +1, 0, m, 0.f);
    else if (warp == cw1) YB[lane] = chain<float>(R, LOs, lane, nz - 1, -1, 0, nz - 1 - m, 0.f);
  }
  __syncthreads();
  // B'
  for (int l = warp; l < nz; l += NW) {
    const int i = l * TW + lane;
    float y = R[i];
    if (TW2 && l == m) y = fmaf(-mtv, YB[lane], fmaf(-LOs[i], YT[lane], y));
    R[i] = y * Ws[i];
  }
  __syncthreads();
  // C
  if (!TW2) {
    const int cw = blockIdx.x % NW;
    if (warp == cw) chain<float>(R, LOs, lane, nz - 2, -1, +1, nz - 1, R[(nz - 1) * TW + lane]);
  } else {
    const int cw0 = blockIdx.x % NW, cw1 = (cw0 + 1) % NW;
    if (warp == cw0) {
      chain<float>(R, LOs, lane, m - 1, -1, +1, m, R[m * TW + lane]);
    } else if (warp == cw1 && m + 1 < nz) {
      float x = R[(m + 1) * TW + lane] - mtv * R[m * TW + lane];
      R[(m + 1) * TW + lane] = x;
      chain<float>(R, LOs, lane, m + 2, +1, -1, nz - 2 - m, x);
    }
  }
  __syncthreads();
  // D (two accumulators per dot, alternating rows: no long dependent FP64 chain)
  double acc0[2] = {0.0, 0.0}, acc1[2] = {0.0, 0.0};
  if (valid) {
    int k = 0;
    for (int l = warp; l < nz; l += NW, ++k) {
      const int i = l * TW + lane;
      const float xv = R[i];
      const TO out = (MODE == MODE_ZERO) ? cvt<TO>(xv) : cvt<TO>(fmaf(om1, Us[i], xv));
      uo[base + (int64_t)l * TW] = out;
      if (DOT) acc0[k & 1] = fma(da[base + (int64_t)l * TW], (double)out, acc0[k & 1]);
      if (DOT == 2) acc1[k & 1] = fma((double)out, dc[base + (int64_t)l * TW], acc1[k & 1]);
    }
  }
  if (DOT)
    grid_reduce<(DOT == 2 ? 2 : 1)>(acc0[0] + acc0[1], acc1[0] + acc1[1], red, reinterpret_cast<double*>(smem_raw));
}

// ---------------------------------------------------------------- FP32 register sweep
//
// Large FP32 levels with a fixed layer count NZ (16, 32 or 64): one warp per
// tile, one lane per column, the whole column in registers.  The forward
// loop is fully unrolled, so the loads of all layers are free to run ahead of
// the (short, FP32) elimination chain; no shared memory and no barrier, so
// many tiles are in flight per SM.  Plain L D L^T (twist row nz - 1).
template <int NZ, typename TB, typename TO, int MODE, typename TE>
__global__ void __launch_bounds__(128)
k_rsweep(LD<float> L, int ntiles, const TB* __restrict__ b, const float* __restrict__ u, TO* __restrict__ uo,
         const TE* __restrict__ ec, float* __restrict__ bcopy, float om1) {
  const int lane = threadIdx.x & 31;
  const int tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (tile >= ntiles) return;
  const int c = tile * TW + lane;
  if (c >= L.nc) return;  // padding columns stay zero
  const int64_t base = (int64_t)tile * TW * NZ + lane;
  typename Vec4<float>::type g{};
  int64_t s0 = 0, s1 = 0, s2 = 0, q = 0, q0 = 0, q1 = 0, q2 = 0;
  if (MODE != MODE_ZERO) {
    const int4 nb = L.nbr[c];
    g = L.gh[c];
    s0 = tile_base(nb.x, NZ);
    s1 = tile_base(nb.y, NZ);
    s2 = tile_base(nb.z, NZ);
    if (MODE == MODE_PRO) {
      q = tile_base(c >> 2, NZ);
      q0 = tile_base(nb.x >> 2, NZ);
      q1 = tile_base(nb.y >> 2, NZ);
      q2 = tile_base(nb.z >> 2, NZ);
    }
  }
  float y[NZ], lo[NZ];
  float yp = 0.f;
#pragma unroll
  for (int l = 0; l < NZ; ++l) {
    const int64_t o = (int64_t)l * TW;
    float r = cvt<float>(b[base + o]);
    if (bcopy) bcopy[base + o] = r;
    if (MODE != MODE_ZERO) {
      float a0 = u[s0 + o], a1 = u[s1 + o], a2 = u[s2 + o];
      if (MODE == MODE_PRO) {
        a0 += cvt<float>(ec[q0 + o]);
        a1 += cvt<float>(ec[q1 + o]);
        a2 += cvt<float>(ec[q2 + o]);
      }
      r = fmaf(g.x, a0, r);
      r = fmaf(g.y, a1, r);
      r = fmaf(g.z, a2, r);
    }
    lo[l] = L.lo[base + o];
    yp = fmaf(-lo[l], yp, r);
    y[l] = yp;
  }
  float x = 0.f;
#pragma unroll
  for (int l = NZ - 1; l >= 0; --l) {
    const int64_t o = (int64_t)l * TW;
    const float lnext = (l + 1 < NZ) ? lo[l + 1] : 0.f;
    x = fmaf(-lnext, x, L.w[base + o] * y[l]);
    float out = x;
    if (MODE != MODE_ZERO) {
      float uc = u[base + o];
      if (MODE == MODE_PRO) uc += cvt<float>(ec[q + o]);
      out = fmaf(om1, uc, x);
    }
    uo[base + o] = cvt<TO>(out);
  }
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
    for (int l = row0; l < nz; l += rstep) u[base + (int64_t)l * TW] += cvt<T>(ec[q + (int64_t)l * TW]);
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
// Large levels (RG = 0): every resident warp takes one contiguous run of the
// level's (tile, layer) rows, so the work is balanced to one row per warp
// whatever the ratio of tiles to CTAs; a warp reloads the column data only
// when its run enters a new tile.
#define HMG_BALANCED_ROWS(NTILES, NZ, ...)                                                    \
  {                                                                                           \
    const int nwt = gridDim.x * NW, gw = blockIdx.x * NW + (threadIdx.x >> 5);                \
    const int total = (NTILES) * (NZ);                                                        \
    const int per = (total + nwt - 1) / nwt;                                                  \
    const int r0 = gw * per, r1 = min(total, r0 + per);                                       \
    int cur = -1;                                                                             \
    for (int wr = r0; wr < r1; ++wr) {                                                        \
      const int tile = wr / (NZ), l = wr - tile * (NZ);                                       \
      const bool fresh = tile != cur;                                                         \
      cur = tile;                                                                             \
      __VA_ARGS__                                                                             \
    }                                                                                         \
  }

template <typename T, typename TC, int NW>
__global__ void __launch_bounds__(NW * 32)
k_tresid_restrict(LD<T> L, int ntiles, int RG, const T* __restrict__ b, const T* __restrict__ u,
                  TC* __restrict__ bc) {
  const int lane = threadIdx.x & 31;
  if (RG == 0 && (L.nz & 3) == 0) {
    // Runs of RC = 4 consecutive layers of one tile per step, every load of
    // the run issued before the arithmetic: four times the bytes in flight
    // per warp of the one-row loop below (which was bound by memory latency).
    constexpr int RC = 4;
    const int nz = L.nz, nch = nz / RC;
    const int nwt = gridDim.x * NW, gw = blockIdx.x * NW + (threadIdx.x >> 5);
    const int total = ntiles * nch;
    const int per = (total + nwt - 1) / nwt;
    const int i0 = gw * per, i1 = min(total, i0 + per);
    typename Vec4<T>::type g{};
    int64_t s0 = 0, s1 = 0, s2 = 0, qc = 0, base = 0;
    bool valid = false;
    int cur = -1;
    for (int it = i0; it < i1; ++it) {
      const int tile = it / nch, l0 = (it - tile * nch) * RC;
      if (tile != cur) {
        cur = tile;
        const int c = tile * TW + lane;
        valid = c < L.nc;
        base = (int64_t)tile * TW * nz + lane;
        const int4 nb = L.nbr[c];
        g = L.gh[c];
        s0 = tile_base(nb.x, nz);
        s1 = tile_base(nb.y, nz);
        s2 = tile_base(nb.z, nz);
        qc = tile_base(c >> 2, nz);
      }
      const int64_t t0 = base + (int64_t)l0 * TW, o0 = (int64_t)l0 * TW;
      T bv[RC], dv[RC], ev[RC + 1], uv[RC + 2], a0[RC], a1[RC], a2[RC];
#pragma unroll
      for (int i = 0; i < RC; ++i) {
        const int64_t t = t0 + i * TW, o = o0 + i * TW;
        bv[i] = b[t];
        dv[i] = L.d[t];
        uv[i + 1] = u[t];
        a0[i] = u[s0 + o];
        a1[i] = u[s1 + o];
        a2[i] = u[s2 + o];
        ev[i] = (l0 + i > 0) ? L.e[t] : (T)0;
      }
      const bool top = l0 + RC < nz;
      ev[RC] = top ? L.e[t0 + RC * TW] : (T)0;
      uv[0] = (l0 > 0) ? u[t0 - TW] : (T)0;
      uv[RC + 1] = top ? u[t0 + RC * TW] : (T)0;
#pragma unroll
      for (int i = 0; i < RC; ++i) {
        // the FMA order of stencil_acc<T, -1>; a missing vertical neighbour
        // contributes fma(-0, 0, y) = y exactly
        T r = fma(-dv[i], uv[i + 1], bv[i]);
        r = fma(-ev[i], uv[i], r);
        r = fma(-ev[i + 1], uv[i + 2], r);
        r = fma(g.x, a0[i], r);
        r = fma(g.y, a1[i], r);
        r = fma(g.z, a2[i], r);
        r += __shfl_xor_sync(0xffffffffu, r, 1);
        r += __shfl_xor_sync(0xffffffffu, r, 2);
        if ((lane & 3) == 0 && valid) bc[qc + o0 + i * TW] = cvt<TC>(r);
      }
    }
    return;
  }
  if (RG == 0) {
    const int nz = L.nz;
    typename Vec4<T>::type g{};
    int64_t s0 = 0, s1 = 0, s2 = 0, qc = 0, base = 0;
    bool valid = false;
    HMG_BALANCED_ROWS(ntiles, nz, {
      if (fresh) {
        const int c = tile * TW + lane;
        valid = c < L.nc;
        base = (int64_t)tile * TW * nz + lane;
        const int4 nb = L.nbr[c];
        g = L.gh[c];
        s0 = tile_base(nb.x, nz);
        s1 = tile_base(nb.y, nz);
        s2 = tile_base(nb.z, nz);
        qc = tile_base(c >> 2, nz);
      }
      const int64_t t = base + (int64_t)l * TW;
      T r = stencil_acc<T, -1>(L, u, t, l, b[t], g, s0, s1, s2);
      r += __shfl_xor_sync(0xffffffffu, r, 1);
      r += __shfl_xor_sync(0xffffffffu, r, 2);
      if ((lane & 3) == 0 && valid) bc[qc + (int64_t)l * TW] = cvt<TC>(r);
    })
    return;
  }
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
      if ((lane & 3) == 0 && valid) bc[qc + (int64_t)l * TW] = cvt<TC>(r);
    }
  }
}

// y = H^ x; with DOT also x.y (the p.q of CG), reduced over the grid.
template <typename T, bool DOT, int NW>
__global__ void __launch_bounds__(NW * 32)
k_tapply(LD<T> L, int ntiles, int RG, const T* __restrict__ x, T* __restrict__ y, Reduce red) {
  const int lane = threadIdx.x & 31;
  const int nz = L.nz;
  double acc[2] = {0.0, 0.0};  // alternate rows: no dependent FP64 chain
  if (RG == 0) {
    typename Vec4<T>::type g{};
    int64_t s0 = 0, s1 = 0, s2 = 0, base = 0;
    HMG_BALANCED_ROWS(ntiles, nz, {
      if (fresh) {
        const int c = tile * TW + lane;   // padding columns: zero stencil (see below)
        base = (int64_t)tile * TW * nz + lane;
        const int4 nb = L.nbr[c];
        g = L.gh[c];
        s0 = tile_base(nb.x, nz);
        s1 = tile_base(nb.y, nz);
        s2 = tile_base(nb.z, nz);
      }
      const int64_t t = base + (int64_t)l * TW;
      const T v = stencil_acc<T, 1>(L, x, t, l, (T)0, g, s0, s1, s2);
      y[t] = v;
      if (DOT) acc[wr & 1] = fma((double)x[t], (double)v, acc[wr & 1]);
    })
  }
  const int rg = RG > 0 ? RG : 1;
  const int row0 = (blockIdx.x % rg) * NW + (threadIdx.x >> 5), rstep = rg * NW;
  for (int tile = RG == 0 ? ntiles : blockIdx.x / rg; tile < ntiles; tile += gridDim.x / rg) {
    // padding columns (levels under 32 columns) are their own neighbours with
    // zero coefficients and data: their stencil is zero, so every lane runs
    // the same branch-free row loop and y stays zero there
    const int c = tile * TW + lane;
    const int64_t base = (int64_t)tile * TW * nz + lane;
    const int4 nb = L.nbr[c];
    const typename Vec4<T>::type g = L.gh[c];
    const int64_t s0 = tile_base(nb.x, nz), s1 = tile_base(nb.y, nz), s2 = tile_base(nb.z, nz);
    int k = 0;
#pragma unroll 4
    for (int l = row0; l < nz; l += rstep, ++k) {
      const int64_t t = base + (int64_t)l * TW;
      const T v = stencil_acc<T, 1>(L, x, t, l, (T)0, g, s0, s1, s2);
      y[t] = v;
      if (DOT) acc[k & 1] = fma((double)x[t], (double)v, acc[k & 1]);
    }
  }
  if (DOT) {
    HMG_RED_SCRATCH(scratch);
    grid_reduce<1>(acc[0] + acc[1], 0.0, red, scratch);
  }
}

constexpr int NW_PAR = 8;
// Tile-sweep CTA size: 4 warps on levels with more tiles than the GPU has
// SMs (FP32 levels the register sweep does not cover: several CTAs resident
// per SM), 16 warps on small levels (latency bound: each warp loads only a
// few rows), 8 on FP64 levels just above the SM count (one wave).  FP64 levels
// of more than 160 tiles take the half-column sweep instead.
constexpr int NW_SWEEP_BIG = 4;
// FP32 levels up to this many tiles use the staged sweep (k_asweep): there it
// beats the register-batched one; on larger levels it does not.
constexpr int STAGED_MAX_TILES = 160;
constexpr int NW_SWEEP_SMALL = 16;
constexpr int NW_SWEEP_MID = 8;

// SMs of the current device, looked up once.
inline int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    n = v > 0 ? v : 152;
  }
  return n;
}

inline int ntiles_of(const Level& L) { return L.ncp / TW; }

struct ParCfg {
  int grid, rg;
};
// Grid of the layer-parallel kernels: whole tiles on large levels, tiles split
// into row groups on small ones (RG * NW <= nz).
// Resident CTAs of a kernel on the whole GPU (one wave), looked up once.
template <typename K>
int resident_grid(K kern, int threads, int& cached) {
  if (cached == 0) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
    cached = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 152);
  }
  return cached;
}

// Large levels: FP32 kernels (memory bound) take balanced rows (RG = 0, one
// resident wave, the launcher sizes the grid); FP64 ones (bound by the FP64
// pipe) keep a capped grid over whole tiles, which keeps more warps resident.
inline ParCfg par_cfg(const Level& L, bool fp32 = false) {
  const int nt = ntiles_of(L);
  const int cap = 152 * 8;
  if (nt >= cap) return {cap, fp32 ? 0 : 1};
  int rg = 1;
  while (rg * 2 * NW_PAR <= L.nz && nt * rg * 2 <= cap) rg *= 2;
  return {nt * rg, rg};
}


template <typename T, typename TB, typename TO, int MODE, typename TE, int NW, int DOT, bool TW2>
void tsweep_k(const Level& L, const void* b, const void* u, void* uo, const void* ec, float* bcopy, double omega,
              const SweepDot* dot, cudaStream_t s) {
  auto kern = k_tsweep<T, TB, TO, MODE, TE, NW, DOT, TW2>;
  size_t smem = (tsweep_arrays(TW2) * (size_t)L.nz + tsweep_spare_rows(TW2)) * TW * sizeof(T);
  if (DOT && smem < (size_t)DOT * NW * 32 * sizeof(double)) smem = (size_t)DOT * NW * 32 * sizeof(double);
  static SmemOptIn opt_in;
  allow_smem(kern, smem, opt_in);
  Reduce red = dot ? dot->red : Reduce{};
  kern<<<ntiles_of(L), NW * 32, smem, s>>>(view<T>(L), (const TB*)b, (const T*)u, (TO*)uo, (const TE*)ec, bcopy,
                                          (T)(1.0 - omega), dot ? dot->a : nullptr, dot ? dot->c : nullptr, red);
}

template <typename T, typename TB, typename TO, int MODE, typename TE, int NW, int DOT>
void tsweep_nw(const Level& L, const void* b, const void* u, void* uo, const void* ec, float* bcopy, double omega,
               const SweepDot* dot, cudaStream_t s) {
  // small levels (16 warps) use the twisted two-chain solve, large ones the
  // single chain: capi.cu sets the twist row with the same tile threshold
  tsweep_k<T, TB, TO, MODE, TE, NW, DOT, (NW == NW_SWEEP_SMALL)>(L, b, u, uo, ec, bcopy, omega, dot, s);
}

template <typename T, typename TB, typename TO, int MODE, typename TE, int NW>
void tsweep_dot(const Level& L, const void* b, const void* u, void* uo, const void* ec, float* bcopy, double omega,
                const SweepDot* dot, cudaStream_t s) {
  if (!dot) tsweep_nw<T, TB, TO, MODE, TE, NW, 0>(L, b, u, uo, ec, bcopy, omega, dot, s);
  else if (!dot->c) tsweep_nw<T, TB, TO, MODE, TE, NW, 1>(L, b, u, uo, ec, bcopy, omega, dot, s);
  else tsweep_nw<T, TB, TO, MODE, TE, NW, 2>(L, b, u, uo, ec, bcopy, omega, dot, s);
}

// FP32 staged sweep: 4 warps on large levels, 8 on small ones (twisted solve)
template <typename TB, typename TO, int MODE, int NW, int DOT, bool TW2>
void asweep_k(const Level& L, const void* b, const void* u, void* uo, float* bcopy, double omega,
              const SweepDot* dot, cudaStream_t s) {
  auto kern = k_asweep<TB, TO, MODE, NW, DOT, TW2>;
  const size_t cells = (size_t)L.nz * TW;
  // b, then lo, w, u (R for MODE_ZERO) and, for MODE_PLAIN, three neighbour arrays, then 2 twist rows
  size_t smem = cells * sizeof(TB) + (MODE == MODE_ZERO ? 3 : 6) * cells * 4 + 2 * TW * 4;
  if (DOT && smem < (size_t)DOT * NW * 32 * sizeof(double)) smem = (size_t)DOT * NW * 32 * sizeof(double);
  static SmemOptIn opt_in;
  allow_smem(kern, smem, opt_in);
  Reduce red = dot ? dot->red : Reduce{};
  kern<<<ntiles_of(L), NW * 32, smem, s>>>(view<float>(L), (const TB*)b, (const float*)u, (TO*)uo, bcopy,
                                          (float)(1.0 - omega), dot ? dot->a : nullptr, dot ? dot->c : nullptr,
                                          red);
}

template <typename TB, typename TO, int MODE, int DOT>
void asweep_dot(const Level& L, const void* b, const void* u, void* uo, float* bcopy, double omega,
                const SweepDot* dot, cudaStream_t s) {
  if (ntiles_of(L) > SMALL_LEVEL_TILES)
    asweep_k<TB, TO, MODE, 4, DOT, false>(L, b, u, uo, bcopy, omega, dot, s);
  else
    asweep_k<TB, TO, MODE, 8, DOT, true>(L, b, u, uo, bcopy, omega, dot, s);
}

template <typename TB, typename TO, int MODE>
void asweep(const Level& L, const void* b, const void* u, void* uo, float* bcopy, double omega, cudaStream_t s,
            const SweepDot* dot = nullptr) {
  if (!dot) asweep_dot<TB, TO, MODE, 0>(L, b, u, uo, bcopy, omega, dot, s);
  else if (!dot->c) asweep_dot<TB, TO, MODE, 1>(L, b, u, uo, bcopy, omega, dot, s);
  else asweep_dot<TB, TO, MODE, 2>(L, b, u, uo, bcopy, omega, dot, s);
}

// Large FP32 levels: the register sweep when the layer count has an
// instantiation (16, 32, 64); returns false otherwise.
template <typename TB, typename TO, int MODE, typename TE>
bool rsweep(const Level& L, const void* b, const void* u, void* uo, const void* ec, float* bcopy, double omega,
            cudaStream_t s) {
  const int nt = ntiles_of(L);
  const int tpb = 4;   // tiles per CTA
  const unsigned grid = (unsigned)((nt + tpb - 1) / tpb);
  const LD<float> v = view<float>(L);
  const float om1 = (float)(1.0 - omega);
  switch (L.nz) {
    case 16:
      k_rsweep<16, TB, TO, MODE, TE><<<grid, 32 * tpb, 0, s>>>(v, nt, (const TB*)b, (const float*)u, (TO*)uo,
                                                              (const TE*)ec, bcopy, om1);
      return true;
    case 32:
      k_rsweep<32, TB, TO, MODE, TE><<<grid, 32 * tpb, 0, s>>>(v, nt, (const TB*)b, (const float*)u, (TO*)uo,
                                                              (const TE*)ec, bcopy, om1);
      return true;
    case 64:
      k_rsweep<64, TB, TO, MODE, TE><<<grid, 32 * tpb, 0, s>>>(v, nt, (const TB*)b, (const float*)u, (TO*)uo,
                                                              (const TE*)ec, bcopy, om1);
      return true;
    default:
      return false;
  }
}

// FP64 levels: the half-column sweep, two tiles per CTA
constexpr int HSWEEP_RB = 1;     // rows per batch of loads
constexpr int HSWEEP_MINB = 9;   // resident CTAs per SM: the finest level in one wave

// Levels with fewer than 8 tiles per SM keep fewer pairs per SM; they take
// four rows per batch of loads (deeper prefetch, 4 CTAs per SM).
constexpr int HSWEEP_DEEP_TILES_PER_SM = 8;

template <int MODE, int DOT>
void hsweep_k(const Level& L, const void* b, const void* u, void* uo, const void* ec, double omega,
              const SweepDot* dot, cudaStream_t s) {
  const int nt = ntiles_of(L);
  const Reduce red = dot ? dot->red : Reduce{};
  if (nt < HSWEEP_DEEP_TILES_PER_SM * num_sms())
    k_hsweep<MODE, DOT, 4, 4><<<(nt + 1) / 2, 128, 0, s>>>(
        view<double>(L), nt, (const double*)b, (const double*)u, (double*)uo, (const double*)ec, 1.0 - omega,
        dot ? dot->a : nullptr, dot ? dot->c : nullptr, red);
  else
    k_hsweep<MODE, DOT, HSWEEP_RB, HSWEEP_MINB><<<(nt + 1) / 2, 128, 0, s>>>(
        view<double>(L), nt, (const double*)b, (const double*)u, (double*)uo, (const double*)ec, 1.0 - omega,
        dot ? dot->a : nullptr, dot ? dot->c : nullptr, red);
}

template <int MODE>
void hsweep(const Level& L, const void* b, const void* u, void* uo, const void* ec, double omega, cudaStream_t s,
            const SweepDot* dot = nullptr) {
  if (!dot) hsweep_k<MODE, 0>(L, b, u, uo, ec, omega, dot, s);
  else if (!dot->c) hsweep_k<MODE, 1>(L, b, u, uo, ec, omega, dot, s);
  else hsweep_k<MODE, 2>(L, b, u, uo, ec, omega, dot, s);
}

template <typename T, typename TB, typename TO, int MODE, typename TE>
void tsweep(const Level& L, const void* b, const void* u, void* uo, const void* ec, float* bcopy, double omega,
            cudaStream_t s, const SweepDot* dot = nullptr) {
  if (ntiles_of(L) > SMALL_LEVEL_TILES)
    tsweep_dot<T, TB, TO, MODE, TE, NW_SWEEP_BIG>(L, b, u, uo, ec, bcopy, omega, dot, s);
  else
    tsweep_dot<T, TB, TO, MODE, TE, NW_SWEEP_SMALL>(L, b, u, uo, ec, bcopy, omega, dot, s);
}

// FP64 levels (factors twisted at nz / 2): the half-column sweep on large
// levels; on small ones, where a lone warp per sub-partition would wait on
// its loads, the 16-warp tile sweep with its twisted two-chain solve.
constexpr int HSWEEP_MIN_TILES = SMALL_LEVEL_TILES;

template <int MODE, int NW>
void tsweep_twisted(const Level& L, const void* b, const void* u, void* uo, const void* ec, double omega,
                    const SweepDot* dot, cudaStream_t s) {
  if (!dot) tsweep_k<double, double, double, MODE, double, NW, 0, true>(L, b, u, uo, ec, nullptr, omega, dot, s);
  else if (!dot->c)
    tsweep_k<double, double, double, MODE, double, NW, 1, true>(L, b, u, uo, ec, nullptr, omega, dot, s);
  else tsweep_k<double, double, double, MODE, double, NW, 2, true>(L, b, u, uo, ec, nullptr, omega, dot, s);
}

template <int MODE>
void fp64_sweep(const Level& L, const void* b, const void* u, void* uo, const void* ec, double omega,
                cudaStream_t s, const SweepDot* dot = nullptr) {
  const int nt = ntiles_of(L);
  if (nt > HSWEEP_MIN_TILES)
    hsweep<MODE>(L, b, u, uo, ec, omega, s, dot);
  else if (nt > SMALL_LEVEL_TILES)
    tsweep_twisted<MODE, NW_SWEEP_BIG>(L, b, u, uo, ec, omega, dot, s);
  else if (nt > num_sms())   // one 16-warp CTA per SM: 8-warp CTAs keep the level in one wave
    tsweep_twisted<MODE, NW_SWEEP_MID>(L, b, u, uo, ec, omega, dot, s);
  else
    tsweep_twisted<MODE, NW_SWEEP_SMALL>(L, b, u, uo, ec, omega, dot, s);
}

// ---------------------------------------------------------------- fused coarse levels
//
// The coarse end of the V-cycle (Algorithm 1 from level ls down to the
// coarsest and back) as one cooperative kernel: each sweep, residual and
// prolongation pass is a phase over the whole grid, and a grid-wide barrier
// separates phases.  On these levels (at most CC_MAX_TILES tiles) every
// separate kernel is bound by launch and memory latency; here the phases
// follow each other without a launch, and the level's data written by one
// phase is read by the next from L2.  The phases are the same per-tile
// sweeps (tsweep_tile, twisted two-chain solve) and the same residual
// stencil as the separate kernels, in the same order, so the result is
// identical.  Every CTA passes the same sequence of barriers: the phase
// sequence depends only on the kernel arguments.

struct CoarseArgs {
  int nlev;                        // levels ls .. ls + nlev - 1, the last the coarsest
  int nu_pre, nu_post, n_coarse;
  double om1;                      // 1 - omega
  LD<double> d[CC_MAX_LEVELS];
  LD<float> f[CC_MAX_LEVELS];
  int ntiles[CC_MAX_LEVELS];
  void* ua[CC_MAX_LEVELS];         // the level's work buffers, of the level's type
  void* ub[CC_MAX_LEVELS];
  void* bb[CC_MAX_LEVELS];         // right-hand side (restricted residual) of levels below the first
  void* ux[CC_MAX_LEVELS];         // result of levels below the first (the coarse correction)
  const void* b_in;                // right-hand side of the first level
  void* out;                       // result of the first level
};

template <typename T> __device__ __forceinline__ const LD<T>& cc_view(const CoarseArgs& a, int k);
template <> __device__ __forceinline__ const LD<double>& cc_view<double>(const CoarseArgs& a, int k) {
  return a.d[k];
}
template <> __device__ __forceinline__ const LD<float>& cc_view<float>(const CoarseArgs& a, int k) {
  return a.f[k];
}

template <typename T, typename TO, int MODE, typename TE, int NW>
__device__ __forceinline__ void cc_sweep(const CoarseArgs& a, int k, const T* b, const T* u, TO* uo, const TE* ec) {
  const LD<T>& L = cc_view<T>(a, k);
  for (int t = blockIdx.x; t < a.ntiles[k]; t += gridDim.x) {
    tsweep_tile<T, T, TO, MODE, TE, NW, 0, true>(L, t, b, u, uo, ec, nullptr, (T)a.om1, nullptr, nullptr,
                                                 Reduce{});
    __syncthreads();   // the next tile reuses the shared arrays
  }
}

// b_c = P^T (b - H^ u), one (tile, layer) row per warp step over the grid
template <typename T, typename TC, int NW>
__device__ __forceinline__ void cc_resid(const CoarseArgs& a, int k, const T* b, const T* u, TC* bc) {
  const LD<T>& L = cc_view<T>(a, k);
  const int lane = threadIdx.x & 31, nz = L.nz;
  const int rows = a.ntiles[k] * nz;
  for (int row = blockIdx.x * NW + (threadIdx.x >> 5); row < rows; row += gridDim.x * NW) {
    const int tile = row / nz, l = row - tile * nz;
    const int c = tile * TW + lane;
    const bool valid = c < L.nc;
    T r = 0;
    if (valid) {
      const int4 nb = L.nbr[c];
      const typename Vec4<T>::type g = L.gh[c];
      const int64_t t = (int64_t)tile * TW * nz + lane + (int64_t)l * TW;
      r = stencil_acc<T, -1>(L, u, t, l, b[t], g, tile_base(nb.x, nz), tile_base(nb.y, nz), tile_base(nb.z, nz));
    }
    r += __shfl_xor_sync(0xffffffffu, r, 1);
    r += __shfl_xor_sync(0xffffffffu, r, 2);
    if ((lane & 3) == 0 && valid) bc[tile_base(c >> 2, nz) + (int64_t)l * TW] = cvt<TC>(r);
  }
}

template <bool MIXED, int NW>
__global__ void __launch_bounds__(NW * 32, 2) k_coarse_cycle(const __grid_constant__ CoarseArgs a) {
  using T = typename std::conditional<MIXED, float, double>::type;
  cg::grid_group grid = cg::this_grid();
  const int last = a.nlev - 1;
  T* cur[CC_MAX_LEVELS];
  T* nxt[CC_MAX_LEVELS];
  // descent: first relaxation from zero, nu_pre - 1 more, residual restricted
  for (int k = 0; k < last; ++k) {
    const T* bk = k == 0 ? (const T*)a.b_in : (const T*)a.bb[k];
    T* c0 = (T*)a.ua[k];
    T* c1 = (T*)a.ub[k];
    cc_sweep<T, T, MODE_ZERO, T, NW>(a, k, bk, nullptr, c0, (const T*)nullptr);
    grid.sync();
    for (int i = 1; i < a.nu_pre; ++i) {
      cc_sweep<T, T, MODE_PLAIN, T, NW>(a, k, bk, c0, c1, (const T*)nullptr);
      grid.sync();
      T* tmp = c0;
      c0 = c1;
      c1 = tmp;
    }
    if (k + 1 == last) cc_resid<T, double, NW>(a, k, bk, c0, (double*)a.bb[k + 1]);
    else cc_resid<T, T, NW>(a, k, bk, c0, (T*)a.bb[k + 1]);
    grid.sync();
    cur[k] = c0;
    nxt[k] = c1;
  }
  // coarsest level (FP64 in both forms): n_coarse relaxations from zero
  {
    const double* bk = last == 0 ? (const double*)a.b_in : (const double*)a.bb[last];
    double* outc = last == 0 ? (double*)a.out : (double*)a.ux[last];
    double* c0 = (double*)a.ua[last];
    double* c1 = (double*)a.ub[last];
    cc_sweep<double, double, MODE_ZERO, double, NW>(a, last, bk, nullptr, a.n_coarse == 1 ? outc : c0,
                                                    (const double*)nullptr);
    for (int i = 1; i < a.n_coarse; ++i) {
      grid.sync();
      cc_sweep<double, double, MODE_PLAIN, double, NW>(a, last, bk, c0, i == a.n_coarse - 1 ? outc : c1,
                                                       (const double*)nullptr);
      double* tmp = c0;
      c0 = c1;
      c1 = tmp;
    }
  }
  // ascent: the first post-relaxation adds the prolonged correction (u + P e_c)
  for (int k = last - 1; k >= 0; --k) {
    grid.sync();
    const T* bk = k == 0 ? (const T*)a.b_in : (const T*)a.bb[k];
    T* outk = k == 0 ? (T*)a.out : (T*)a.ux[k];
    T* c0 = cur[k];
    T* c1 = nxt[k];
    for (int i = 0; i < a.nu_post; ++i) {
      const bool lst = i == a.nu_post - 1;
      T* dst = lst ? outk : c1;
      if (i == 0 && k + 1 == last)
        cc_sweep<T, T, MODE_PRO, double, NW>(a, k, bk, c0, dst, (const double*)a.ux[k + 1]);
      else if (i == 0)
        cc_sweep<T, T, MODE_PRO, T, NW>(a, k, bk, c0, dst, (const T*)a.ux[k + 1]);
      else
        cc_sweep<T, T, MODE_PLAIN, T, NW>(a, k, bk, c0, dst, (const T*)nullptr);
      if (!lst) {
        grid.sync();
        T* tmp = c0;
        c0 = c1;
        c1 = tmp;
      }
    }
  }
}

template <bool MIXED>
cudaError_t coarse_cycle_launch(const CoarseArgs& a, size_t smem, cudaStream_t s) {
  // 8 warps and two CTAs per SM: a level of up to 304 tiles takes one tile per CTA
  constexpr int NW = 8;
  auto kern = k_coarse_cycle<MIXED, NW>;
  static SmemOptIn opt_in;
  cudaError_t e = allow_smem(kern, smem, opt_in);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, coop = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess) return e;
  if (!coop) return cudaErrorNotSupported;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NW * 32, smem)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(per_sm * sms));
  cfg.blockDim = dim3(NW * 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

}  // namespace

void launch_sweep0(const Level& L, int dt, const void* b, int b_dt, void* u, float* bcopy, double omega,
                   cudaStream_t s) {
  if (dt == HMG_FP64)
    fp64_sweep<MODE_ZERO>(L, b, nullptr, u, nullptr, omega, s);
  else if (ntiles_of(L) > STAGED_MAX_TILES && b_dt == HMG_FP64 &&
           rsweep<double, float, MODE_ZERO, float>(L, b, nullptr, u, nullptr, bcopy, omega, s))
    return;
  else if (ntiles_of(L) > STAGED_MAX_TILES && b_dt != HMG_FP64 &&
           rsweep<float, float, MODE_ZERO, float>(L, b, nullptr, u, nullptr, nullptr, omega, s))
    return;
  else if (b_dt == HMG_FP64)
    tsweep<float, double, float, MODE_ZERO, float>(L, b, nullptr, u, nullptr, bcopy, omega, s);
  else if (ntiles_of(L) <= STAGED_MAX_TILES)
    asweep<float, float, MODE_ZERO>(L, b, nullptr, u, nullptr, omega, s);
  else
    tsweep<float, float, float, MODE_ZERO, float>(L, b, nullptr, u, nullptr, nullptr, omega, s);
}

void launch_sweep(const Level& L, int dt, const void* b, const void* u, void* uo, int uo_dt, const void* ec,
                  int ec_dt, double omega, const SweepDot* dot, cudaStream_t s) {
  if (dt == HMG_FP64) {
    if (ec) fp64_sweep<MODE_PRO>(L, b, u, uo, ec, omega, s, dot);
    else fp64_sweep<MODE_PLAIN>(L, b, u, uo, nullptr, omega, s, dot);
    return;
  }
  const bool out64 = uo_dt == HMG_FP64;
  if (ntiles_of(L) > STAGED_MAX_TILES && !dot) {  // large levels: register sweep when it applies
    bool done = false;
    if (!ec) {
      done = out64 ? rsweep<float, double, MODE_PLAIN, float>(L, b, u, uo, nullptr, nullptr, omega, s)
                   : rsweep<float, float, MODE_PLAIN, float>(L, b, u, uo, nullptr, nullptr, omega, s);
    } else if (ec_dt == HMG_FP64) {
      done = out64 ? rsweep<float, double, MODE_PRO, double>(L, b, u, uo, ec, nullptr, omega, s)
                   : rsweep<float, float, MODE_PRO, double>(L, b, u, uo, ec, nullptr, omega, s);
    } else {
      done = out64 ? rsweep<float, double, MODE_PRO, float>(L, b, u, uo, ec, nullptr, omega, s)
                   : rsweep<float, float, MODE_PRO, float>(L, b, u, uo, ec, nullptr, omega, s);
    }
    if (done) return;
  }
  if (!ec) {
    // small levels: staged sweep (the prolongation, if any, was a pass of its own)
    if (ntiles_of(L) <= STAGED_MAX_TILES) {
      if (out64) asweep<float, double, MODE_PLAIN>(L, b, u, uo, nullptr, omega, s, dot);
      else asweep<float, float, MODE_PLAIN>(L, b, u, uo, nullptr, omega, s, dot);
    } else {
      if (out64) tsweep<float, float, double, MODE_PLAIN, float>(L, b, u, uo, nullptr, nullptr, omega, s, dot);
      else tsweep<float, float, float, MODE_PLAIN, float>(L, b, u, uo, nullptr, nullptr, omega, s, dot);
    }
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

// grid of a layer-parallel launch: one resident wave in the balanced mode
#define HMG_PAR_GRID(KERN, PC)                                       \
  ([&] {                                                             \
    static int cached_ = 0;                                          \
    return (PC).rg == 0 ? resident_grid(KERN, NW_PAR * 32, cached_) : (PC).grid; \
  }())

void launch_resid_restrict(const Level& L, int dt, const void* b, const void* u, void* bc, int bc_dt,
                           cudaStream_t s) {
  const ParCfg pc = par_cfg(L, dt == HMG_FP32);
  const int nt = ntiles_of(L), rg = pc.rg;
  if (dt == HMG_FP64) {
    auto k = k_tresid_restrict<double, double, NW_PAR>;
    k<<<HMG_PAR_GRID(k, pc), NW_PAR * 32, 0, s>>>(view<double>(L), nt, rg, (const double*)b, (const double*)u,
                                                  (double*)bc);
  } else if (bc_dt == HMG_FP64) {
    auto k = k_tresid_restrict<float, double, NW_PAR>;
    k<<<HMG_PAR_GRID(k, pc), NW_PAR * 32, 0, s>>>(view<float>(L), nt, rg, (const float*)b, (const float*)u,
                                                  (double*)bc);
  } else {
    auto k = k_tresid_restrict<float, float, NW_PAR>;
    k<<<HMG_PAR_GRID(k, pc), NW_PAR * 32, 0, s>>>(view<float>(L), nt, rg, (const float*)b, (const float*)u,
                                                  (float*)bc);
  }
}

void launch_apply(const Level& L, int dt, const void* x, void* y, const Reduce* red, cudaStream_t s) {
  const ParCfg pc = par_cfg(L, dt == HMG_FP32);
  const int nt = ntiles_of(L), rg = pc.rg;
  const Reduce r = red ? *red : Reduce{};
  if (dt == HMG_FP64) {
    if (red) {
      auto k = k_tapply<double, true, NW_PAR>;
      k<<<HMG_PAR_GRID(k, pc), NW_PAR * 32, 0, s>>>(view<double>(L), nt, rg, (const double*)x, (double*)y, r);
    } else {
      auto k = k_tapply<double, false, NW_PAR>;
      k<<<HMG_PAR_GRID(k, pc), NW_PAR * 32, 0, s>>>(view<double>(L), nt, rg, (const double*)x, (double*)y, r);
    }
  } else {
    if (red) {
      auto k = k_tapply<float, true, NW_PAR>;
      k<<<HMG_PAR_GRID(k, pc), NW_PAR * 32, 0, s>>>(view<float>(L), nt, rg, (const float*)x, (float*)y, r);
    } else {
      auto k = k_tapply<float, false, NW_PAR>;
      k<<<HMG_PAR_GRID(k, pc), NW_PAR * 32, 0, s>>>(view<float>(L), nt, rg, (const float*)x, (float*)y, r);
    }
  }
}


cudaError_t launch_coarse_cycle(const Level* lv, int ls, int nlev, int nu_pre, int nu_post, int n_coarse,
                                double omega, bool mixed, const void* b_in, void* out, cudaStream_t s) {
  const int n = nlev - ls;
  if (n < 1 || n > CC_MAX_LEVELS) return cudaErrorInvalidValue;
  CoarseArgs a{};
  a.nlev = n;
  a.nu_pre = nu_pre;
  a.nu_post = nu_post;
  a.n_coarse = n_coarse;
  a.om1 = 1.0 - omega;
  a.b_in = b_in;
  a.out = out;
  size_t smem = 0;
  for (int k = 0; k < n; ++k) {
    const Level& L = lv[ls + k];
    const bool f32 = mixed && k < n - 1;
    a.d[k] = view<double>(L);
    if (f32) a.f[k] = view<float>(L);
    a.ntiles[k] = ntiles_of(L);
    a.ua[k] = f32 ? (void*)L.ua32 : (void*)L.ua64;
    a.ub[k] = f32 ? (void*)L.ub32 : (void*)L.ub64;
    a.bb[k] = f32 ? (void*)L.b32 : (void*)L.b64;
    a.ux[k] = f32 ? (void*)L.ux32 : (void*)L.ux64;
    const size_t sm = (tsweep_arrays(true) * (size_t)L.nz + tsweep_spare_rows(true)) * TW *
                      (f32 ? sizeof(float) : sizeof(double));
    if (sm > smem) smem = sm;
  }
  return mixed ? coarse_cycle_launch<true>(a, smem, s) : coarse_cycle_launch<false>(a, smem, s);
}

}  // namespace hmg
