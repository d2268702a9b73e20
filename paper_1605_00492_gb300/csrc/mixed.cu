// The velocity-pressure system of the lowest-order discretisation (Sec. 4.1,
// Eq. PressureVelocitySystem) on the finest level, and the two outer factors
// of its Schur-complement preconditioner (Sec. 4.2, Eq. SchurComplement with
// the diagonal velocity-mass inverse of Eq. LumpedMass):
//
//   A (U, P) = ( M2~ U - a D^T P ,  a c^2 D U + M3 P ),  a = dt / 2,
//   M2~ = M2^h (+) (1 + w_N^2) M2^z.
//
// Unit-flux bases: the RT0 function of edge k of a prism's triangle T is
// (x - v_k) / (2 |T| dz) horizontally (v_k the vertex opposite the edge), so
// the prism's 3 x 3 block of M2^h is S_T / dz with the scale-invariant
//   S_T[k, k'] = int_T (x - v_k).(x - v_k') dA / (4 |T|^2)
//              = sum_{m,n} (v_m - v_k).(v_n - v_k') (1 + delta_mn) / (48 |T|)
// on the flat unit-sphere triangle (barycentric moments |T| (1 + delta) / 12),
// and a horizontal face couples with itself and the other two faces of each
// of its two prisms.  The vertical fluxes are P1 in z, z^ phi / A_K on cell K:
// the cell adds dz / (3 A_K) to the diagonal of its two faces and
// dz / (6 A_K) between them.  D has entries +-1: +1 on the lower-numbered
// column of an edge and on the cell below a vertical face.
#include "hmg_internal.h"

namespace hmg {

namespace {

__device__ __forceinline__ int64_t tb(int c, int nz) { return (int64_t)(c >> 5) * (TW * nz) + (c & 31); }

// S_T of one flat triangle with vertices v[0..2]
__device__ void rt0_block(const double* v, double S[3][3]) {
  double e1[3], e2[3], cr[3];
  for (int i = 0; i < 3; ++i) {
    e1[i] = v[3 + i] - v[i];
    e2[i] = v[6 + i] - v[i];
  }
  cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
  cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
  cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
  const double area = 0.5 * sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
  for (int k = 0; k < 3; ++k)
    for (int kk = 0; kk < 3; ++kk) {
      double acc = 0.0;
      for (int m = 0; m < 3; ++m)
        for (int n = 0; n < 3; ++n) {
          double d = 0.0;
          for (int i = 0; i < 3; ++i) d += (v[3 * m + i] - v[3 * k + i]) * (v[3 * n + i] - v[3 * kk + i]);
          acc += d * (m == n ? 2.0 : 1.0);
        }
      S[k][kk] = acc / (48.0 * area);
    }
}

__device__ __forceinline__ int csign(const int4& ce, int k) { return ((ce.w >> k) & 1) ? -1 : 1; }

// +-v by the sign bit of local edge k (an integer operation, no FP64 multiply)
__device__ __forceinline__ double sgn_apply(const int4& ce, int k, double v) {
  const long long neg = (long long)((ce.w >> k) & 1) << 63;
  return __longlong_as_double(__double_as_longlong(v) ^ neg);
}
__device__ __forceinline__ int cedge_k(const int4& ce, int k) { return k == 0 ? ce.x : (k == 1 ? ce.y : ce.z); }

// Per edge: M2^h diagonal and the four coupled edges with their entries.
__global__ void k_mx_edge_coeffs(int ne, int nep, double dz, const int4* __restrict__ edge,
                                 const int4* __restrict__ cedge, const double* __restrict__ verts, int4* enb,
                                 double4_32a* ecoef, double* emass, double* einv) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nep) return;
  if (e >= ne) {
    enb[e] = make_int4(e, e, e, e);
    ecoef[e] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    emass[e] = einv[e] = 0.0;
    return;
  }
  const int4 ed = edge[e];
  double St[3][3], Sn[3][3];
  rt0_block(verts + 9 * (int64_t)ed.x, St);
  rt0_block(verts + 9 * (int64_t)ed.z, Sn);
  const int4 ct = cedge[ed.x], cn = cedge[ed.z];
  const int k = ed.y, kn = ed.w;
  const int k1 = (k + 1) % 3, k2 = (k + 2) % 3, kn1 = (kn + 1) % 3, kn2 = (kn + 2) % 3;
  // the face is +1 on column t (local edge k) and -1 on column tn (local edge kn)
  enb[e] = make_int4(cedge_k(ct, k1), cedge_k(ct, k2), cedge_k(cn, kn1), cedge_k(cn, kn2));
  ecoef[e] = make_double4_32a(csign(ct, k1) * St[k][k1] / dz, csign(ct, k2) * St[k][k2] / dz,
                              -csign(cn, kn1) * Sn[kn][kn1] / dz, -csign(cn, kn2) * Sn[kn][kn2] / dz);
  emass[e] = (St[k][k] + Sn[kn][kn]) / dz;
  einv[e] = 1.0 / emass[e];
}

// Per cell: zd = dz / (3 A_K), m3 = |K| (prism reading: A_K = A1 rho_l^2),
// and for the vertical face above the cell zsi = 1 / (zd_l + zd_(l+1)), the
// reciprocal of its M2^z diagonal (0 at the top)
__global__ void k_mx_cell_coeffs(int nc, int nz, int64_t Np, double R, double dz, const double* __restrict__ A1,
                                 double* zd, double* m3, double* zsi) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= Np) return;
  const int lane = (int)(t & 31);
  const int l = (int)((t >> 5) % nz);
  const int c = (int)((t / (TW * nz)) * TW + lane);
  if (c >= nc) {
    zd[t] = m3[t] = zsi[t] = 0.0;
    return;
  }
  const double rho = R + (l + 0.5) * dz, rhou = R + (l + 1.5) * dz;
  const double A = A1[c] * rho * rho, Au = A1[c] * rhou * rhou;
  zd[t] = dz / (3.0 * A);
  m3[t] = A * dz;
  zsi[t] = l < nz - 1 ? 1.0 / (dz / (3.0 * A) + dz / (3.0 * Au)) : 0.0;
}

struct MxArgs {
  int nc, nz, ne, ntc, nte;   // columns, layers, edges, column tiles, edge tiles
  int64_t Np, nh;
  double a, c2, wn2;
  const int4* edge;
  const int4* enb;
  const double4_32a* ecoef;
  const double* emass;
  const double* einv;         // 1 / emass
  const int4* cedge;
  const double* zd;
  const double* m3;
  const double* zsi;          // 1 / (zd_l + zd_(l+1))
  double inv1wn2;             // 1 / (1 + w_N^2)
  double one_wn2, ac2;        // 1 + w_N^2, a c^2
};

// 1 / M2~ diagonal of the vertical face between layers l and l + 1 (t = its index)
__device__ __forceinline__ double mz_inv(const MxArgs& A, int64_t t) { return A.zsi[t] * A.inv1wn2; }

// The kernels walk (tile, row) pairs without index division: CTAs stride over
// tiles, warps over rows, lanes are the tile's 32 edges or columns.
constexpr int MX_THREADS = 256;   // 8 warps: rows of a tile
constexpr int MX_WARPS = MX_THREADS / 32;

// Rows are unrolled by four so that each thread has several rows' loads in flight.
#define MX_TILE_LOOP(NT)                                                                          \
  for (int tile = blockIdx.x; tile < (NT); tile += gridDim.x)                                     \
    _Pragma("unroll 4") for (int l = threadIdx.x >> 5; l < A.nz; l += MX_WARPS)

// y_h = M2^h x_h - a D_h^T x_p
__global__ void k_mx_apply_h(MxArgs A, const double* __restrict__ x, double* __restrict__ y) {
  const double* xp = x + A.nh + A.Np;
  const int lane = threadIdx.x & 31;
  MX_TILE_LOOP(A.nte) {
    const int e = tile * TW + lane;
    const int64_t i = (int64_t)tile * TW * A.nz + (int64_t)l * TW + lane;
    double v = 0.0;
    if (e < A.ne) {
      const int4 ed = A.edge[e];
      const int4 nb = A.enb[e];
      const double4_32a m = A.ecoef[e];
      const int64_t o = (int64_t)l * TW;
      v = A.emass[e] * x[i];
      v = fma(m.x, x[tb(nb.x, A.nz) + o], v);
      v = fma(m.y, x[tb(nb.y, A.nz) + o], v);
      v = fma(m.z, x[tb(nb.z, A.nz) + o], v);
      v = fma(m.w, x[tb(nb.w, A.nz) + o], v);
      v = fma(-A.a, xp[tb(ed.x, A.nz) + o] - xp[tb(ed.z, A.nz) + o], v);
    }
    y[i] = v;
  }
}

// y_z = (1 + w_N^2) M2^z x_z - a D_z^T x_p;  y_p = a c^2 D x_u + M3 x_p
__global__ void k_mx_apply_zp(MxArgs A, const double* __restrict__ x, double* __restrict__ y) {
  const double* xh = x;
  const double* xz = x + A.nh;
  const double* xp = x + A.nh + A.Np;
  const int lane = threadIdx.x & 31;
  MX_TILE_LOOP(A.ntc) {
    const int c = tile * TW + lane;
    const int64_t t = (int64_t)tile * TW * A.nz + (int64_t)l * TW + lane;
    double vz = 0.0, vp = 0.0;
    if (c < A.nc) {
      const int64_t o = (int64_t)l * TW;
      const double xzc = l < A.nz - 1 ? xz[t] : 0.0, xzd = l > 0 ? xz[t - TW] : 0.0;
      if (l < A.nz - 1) {
        // M2^z row of this face: cell l adds zd_l (x_f + x_below / 2), cell l + 1 adds zd_(l+1) (x_f + x_above / 2)
        const double xzu = l + 1 < A.nz - 1 ? xz[t + TW] : 0.0;
        const double m = fma(A.zd[t], fma(0.5, xzd, xzc), A.zd[t + TW] * fma(0.5, xzu, xzc));
        vz = fma(A.one_wn2, m, -A.a * (xp[t] - xp[t + TW]));
      }
      const int4 ce = A.cedge[c];
      double div = sgn_apply(ce, 0, xh[tb(ce.x, A.nz) + o]);
      div += sgn_apply(ce, 1, xh[tb(ce.y, A.nz) + o]);
      div += sgn_apply(ce, 2, xh[tb(ce.z, A.nz) + o]);
      div += xzc - xzd;
      vp = fma(A.ac2, div, A.m3[t] * xp[t]);
    }
    y[A.nh + t] = vz;
    y[A.nh + A.Np + t] = vp;
  }
}

// rp = r_P - a c^2 D (M2inv r_U)
__global__ void k_mx_pre_lower(MxArgs A, const double* __restrict__ r, double* __restrict__ rp) {
  const double* rh = r;
  const double* rz = r + A.nh;
  const double* rpin = r + A.nh + A.Np;
  const int lane = threadIdx.x & 31;
  MX_TILE_LOOP(A.ntc) {
    const int c = tile * TW + lane;
    const int64_t t = (int64_t)tile * TW * A.nz + (int64_t)l * TW + lane;
    double v = 0.0;
    if (c < A.nc) {
      const int4 ce = A.cedge[c];
      const int64_t o = (int64_t)l * TW;
      double div = sgn_apply(ce, 0, rh[tb(ce.x, A.nz) + o]) * A.einv[ce.x];
      div = fma(sgn_apply(ce, 1, rh[tb(ce.y, A.nz) + o]), A.einv[ce.y], div);
      div = fma(sgn_apply(ce, 2, rh[tb(ce.z, A.nz) + o]), A.einv[ce.z], div);
      // vertical faces: (1 + w_N^2)^-1 applied once to their sum
      double vz = 0.0;
      if (l < A.nz - 1) vz = rz[t] * A.zsi[t];
      if (l > 0) vz = fma(-rz[t - TW], A.zsi[t - TW], vz);
      div = fma(vz, A.inv1wn2, div);
      v = fma(-A.ac2, div, rpin[t]);
    }
    rp[t] = v;
  }
}

// z_h = M2inv (r_h + a D_h^T z_P)
__global__ void k_mx_pre_upper_h(MxArgs A, const double* __restrict__ r, double* __restrict__ z) {
  const double* zp = z + A.nh + A.Np;
  const int lane = threadIdx.x & 31;
  MX_TILE_LOOP(A.nte) {
    const int e = tile * TW + lane;
    const int64_t i = (int64_t)tile * TW * A.nz + (int64_t)l * TW + lane;
    double v = 0.0;
    if (e < A.ne) {
      const int4 ed = A.edge[e];
      const int64_t o = (int64_t)l * TW;
      v = (r[i] + A.a * (zp[tb(ed.x, A.nz) + o] - zp[tb(ed.z, A.nz) + o])) * A.einv[e];
    }
    z[i] = v;
  }
}

// z_z = M2inv (r_z + a D_z^T z_P)
__global__ void k_mx_pre_upper_z(MxArgs A, const double* __restrict__ r, double* __restrict__ z) {
  const double* zp = z + A.nh + A.Np;
  const int lane = threadIdx.x & 31;
  MX_TILE_LOOP(A.ntc) {
    const int c = tile * TW + lane;
    const int64_t t = (int64_t)tile * TW * A.nz + (int64_t)l * TW + lane;
    double v = 0.0;
    if (c < A.nc && l < A.nz - 1) v = (r[A.nh + t] + A.a * (zp[t] - zp[t + TW])) * mz_inv(A, t);
    z[A.nh + t] = v;
  }
}

MxArgs args_of(const Level& L, const MixedSys& M, const Phys& ph) {
  return MxArgs{L.nc, L.nz, M.ne, L.ncp / TW, M.nep / TW, L.Np, M.nh, ph.a, ph.c2, ph.wn2,
                M.edge, M.enb, M.ecoef, M.emass, M.einv, M.cedge, M.zd, M.m3, M.zsi, 1.0 / (1.0 + ph.wn2),
                1.0 + ph.wn2, ph.a * ph.c2};
}


int grid_tiles(int ntiles) { return ntiles < 152 * 8 ? ntiles : 152 * 8; }

}  // namespace

void launch_mixed_coeffs(const Level& L, const MixedSys& M, const Phys& ph, cudaStream_t s) {
  k_mx_edge_coeffs<<<(M.nep + 127) / 128, 128, 0, s>>>(M.ne, M.nep, ph.dz, M.edge, M.cedge, L.verts, M.enb,
                                                      M.ecoef, M.emass, M.einv);
  k_mx_cell_coeffs<<<(unsigned)((L.Np + 255) / 256), 256, 0, s>>>(L.nc, L.nz, L.Np, ph.R, ph.dz, L.A1, M.zd,
                                                                   M.m3, M.zsi);
}

void launch_mixed_apply(const Level& L, const MixedSys& M, const Phys& ph, const double* x, double* y,
                        cudaStream_t s) {
  const MxArgs A = args_of(L, M, ph);
  k_mx_apply_h<<<grid_tiles(A.nte), MX_THREADS, 0, s>>>(A, x, y);
  k_mx_apply_zp<<<grid_tiles(A.ntc), MX_THREADS, 0, s>>>(A, x, y);
}

void launch_mixed_pre_lower(const Level& L, const MixedSys& M, const Phys& ph, const double* r, double* rp,
                            cudaStream_t s) {
  const MxArgs A = args_of(L, M, ph);
  k_mx_pre_lower<<<grid_tiles(A.ntc), MX_THREADS, 0, s>>>(A, r, rp);
}

void launch_mixed_pre_upper(const Level& L, const MixedSys& M, const Phys& ph, const double* r, double* z,
                            cudaStream_t s) {
  const MxArgs A = args_of(L, M, ph);
  k_mx_pre_upper_h<<<grid_tiles(A.nte), MX_THREADS, 0, s>>>(A, r, z);
  k_mx_pre_upper_z<<<grid_tiles(A.ntc), MX_THREADS, 0, s>>>(A, r, z);
}

void launch_mixed_layout(const Level& L, const MixedSys& M, bool to_tiled, const double* u_col, const double* p_col,
                         double* tiled, double* u_out, double* p_out, cudaStream_t s) {
  // horizontal faces e * nz + l; vertical faces c * (nz - 1) + l after them; cells c * nz + l
  const int64_t nhc = (int64_t)M.ne * L.nz;
  if (to_tiled) {
    launch_transpose64(true, M.ne, L.nz, L.nz, u_col, tiled, s);
    launch_transpose64(true, L.nc, L.nz, L.nz - 1, u_col + nhc, tiled + M.nh, s);
    launch_transpose64(true, L.nc, L.nz, L.nz, p_col, tiled + M.nh + L.Np, s);
  } else {
    launch_transpose64(false, M.ne, L.nz, L.nz, tiled, u_out, s);
    launch_transpose64(false, L.nc, L.nz, L.nz - 1, tiled + M.nh, u_out + nhc, s);
    launch_transpose64(false, L.nc, L.nz, L.nz, tiled + M.nh + L.Np, p_out, s);
  }
}

}  // namespace hmg
