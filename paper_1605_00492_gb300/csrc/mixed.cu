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
__device__ __forceinline__ int cedge_k(const int4& ce, int k) { return k == 0 ? ce.x : (k == 1 ? ce.y : ce.z); }

// Per edge: M2^h diagonal and the four coupled edges with their entries.
__global__ void k_mx_edge_coeffs(int ne, int nep, double dz, const int4* __restrict__ edge,
                                 const int4* __restrict__ cedge, const double* __restrict__ verts, int4* enb,
                                 double4_32a* ecoef, double* emass) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nep) return;
  if (e >= ne) {
    enb[e] = make_int4(e, e, e, e);
    ecoef[e] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    emass[e] = 0.0;
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
}

// Per cell: zd = dz / (3 A_K), m3 = |K| (prism reading: A_K = A1 rho_l^2)
__global__ void k_mx_cell_coeffs(int nc, int nz, int64_t Np, double R, double dz, const double* __restrict__ A1,
                                 double* zd, double* m3) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= Np) return;
  const int lane = (int)(t & 31);
  const int l = (int)((t >> 5) % nz);
  const int c = (int)((t / (TW * nz)) * TW + lane);
  if (c >= nc) {
    zd[t] = m3[t] = 0.0;
    return;
  }
  const double rho = R + (l + 0.5) * dz;
  const double A = A1[c] * rho * rho;
  zd[t] = dz / (3.0 * A);
  m3[t] = A * dz;
}

struct MxArgs {
  int nc, nz, ne;
  int64_t Np, nh;
  double a, c2, wn2;
  const int4* edge;
  const int4* enb;
  const double4_32a* ecoef;
  const double* emass;
  const int4* cedge;
  const double* zd;
  const double* m3;
};

__device__ __forceinline__ void decode_h(int64_t t, int nz, int& e, int& l) {
  e = (int)((t / (TW * nz)) * TW + (t & 31));
  l = (int)((t >> 5) % nz);
}
__device__ __forceinline__ void decode_c(int64_t t, int nz, int& c, int& l) {
  c = (int)((t / (TW * nz)) * TW + (t & 31));
  l = (int)((t >> 5) % nz);
}

// M2~ diagonal of the vertical face between layers l and l + 1 of column c (t = its index)
__device__ __forceinline__ double mz_diag(const MxArgs& A, int64_t t) {
  return (1.0 + A.wn2) * (A.zd[t] + A.zd[t + TW]);
}

// y = A x, three sweeps over the parts of the vector
__global__ void k_mx_apply(MxArgs A, const double* __restrict__ x, double* __restrict__ y) {
  const double* xh = x;
  const double* xz = x + A.nh;
  const double* xp = x + A.nh + A.Np;
  const int64_t n = A.nh + 2 * A.Np;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    if (i < A.nh) {
      int e, l;
      decode_h(i, A.nz, e, l);
      if (e < A.ne) {
        const int4 ed = A.edge[e];
        const int4 nb = A.enb[e];
        const double4_32a m = A.ecoef[e];
        const int64_t o = (int64_t)l * TW;
        v = A.emass[e] * xh[i];
        v = fma(m.x, xh[tb(nb.x, A.nz) + o], v);
        v = fma(m.y, xh[tb(nb.y, A.nz) + o], v);
        v = fma(m.z, xh[tb(nb.z, A.nz) + o], v);
        v = fma(m.w, xh[tb(nb.w, A.nz) + o], v);
        v = fma(-A.a, xp[tb(ed.x, A.nz) + o] - xp[tb(ed.z, A.nz) + o], v);
      }
    } else if (i < A.nh + A.Np) {
      const int64_t t = i - A.nh;
      int c, l;
      decode_c(t, A.nz, c, l);
      if (c < A.nc && l < A.nz - 1) {
        double m = (A.zd[t] + A.zd[t + TW]) * xz[t];
        if (l > 0) m = fma(0.5 * A.zd[t], xz[t - TW], m);
        if (l + 1 < A.nz - 1) m = fma(0.5 * A.zd[t + TW], xz[t + TW], m);
        v = fma(1.0 + A.wn2, m, -A.a * (xp[t] - xp[t + TW]));
      }
    } else {
      const int64_t t = i - A.nh - A.Np;
      int c, l;
      decode_c(t, A.nz, c, l);
      if (c < A.nc) {
        const int4 ce = A.cedge[c];
        const int64_t o = (int64_t)l * TW;
        double div = csign(ce, 0) * xh[tb(ce.x, A.nz) + o] + csign(ce, 1) * xh[tb(ce.y, A.nz) + o] +
                     csign(ce, 2) * xh[tb(ce.z, A.nz) + o];
        if (l < A.nz - 1) div += xz[t];
        if (l > 0) div -= xz[t - TW];
        v = fma(A.a * A.c2, div, A.m3[t] * xp[t]);
      }
    }
    y[i] = v;
  }
}

// rp = r_P - a c^2 D (M2inv r_U), written to the cell part of z
__global__ void k_mx_pre_lower(MxArgs A, const double* __restrict__ r, double* __restrict__ rp) {
  const double* rh = r;
  const double* rz = r + A.nh;
  const double* rpin = r + A.nh + A.Np;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < A.Np; t += (int64_t)gridDim.x * blockDim.x) {
    int c, l;
    decode_c(t, A.nz, c, l);
    double v = 0.0;
    if (c < A.nc) {
      const int4 ce = A.cedge[c];
      const int64_t o = (int64_t)l * TW;
      double div = 0.0;
      for (int k = 0; k < 3; ++k) {
        const int e = cedge_k(ce, k);
        div += csign(ce, k) * rh[tb(e, A.nz) + o] / A.emass[e];
      }
      if (l < A.nz - 1) div += rz[t] / mz_diag(A, t);
      if (l > 0) div -= rz[t - TW] / mz_diag(A, t - TW);
      v = fma(-A.a * A.c2, div, rpin[t]);
    }
    rp[t] = v;
  }
}

// z_U = M2inv (r_U + a D^T z_P), z_P already in the cell part of z
__global__ void k_mx_pre_upper(MxArgs A, const double* __restrict__ r, double* __restrict__ z) {
  const double* zp = z + A.nh + A.Np;
  const int64_t nu = A.nh + A.Np;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nu; i += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    if (i < A.nh) {
      int e, l;
      decode_h(i, A.nz, e, l);
      if (e < A.ne) {
        const int4 ed = A.edge[e];
        const int64_t o = (int64_t)l * TW;
        v = (r[i] + A.a * (zp[tb(ed.x, A.nz) + o] - zp[tb(ed.z, A.nz) + o])) / A.emass[e];
      }
    } else {
      const int64_t t = i - A.nh;
      int c, l;
      decode_c(t, A.nz, c, l);
      if (c < A.nc && l < A.nz - 1) v = (r[i] + A.a * (zp[t] - zp[t + TW])) / mz_diag(A, t);
    }
    z[i] = v;
  }
}

// COLUMN <-> tiled for the whole vector: horizontal faces e * nz + l, vertical
// faces c * (nz - 1) + l, cells c * nz + l
__global__ void k_mx_layout(MxArgs A, bool to_tiled, const double* __restrict__ ucol, const double* __restrict__ pcol,
                            double* __restrict__ tiled, double* __restrict__ uout, double* __restrict__ pout) {
  const int64_t n = A.nh + 2 * A.Np;
  const int64_t nhc = (int64_t)A.ne * A.nz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t src = -1;
    const double* from = nullptr;
    double* to = nullptr;
    if (i < A.nh) {
      int e, l;
      decode_h(i, A.nz, e, l);
      if (e < A.ne) {
        src = (int64_t)e * A.nz + l;
        from = ucol;
        to = uout;
      }
    } else if (i < A.nh + A.Np) {
      int c, l;
      decode_c(i - A.nh, A.nz, c, l);
      if (c < A.nc && l < A.nz - 1) {
        src = nhc + (int64_t)c * (A.nz - 1) + l;
        from = ucol;
        to = uout;
      }
    } else {
      int c, l;
      decode_c(i - A.nh - A.Np, A.nz, c, l);
      if (c < A.nc) {
        src = (int64_t)c * A.nz + l;
        from = pcol;
        to = pout;
      }
    }
    if (to_tiled) tiled[i] = src >= 0 ? from[src] : 0.0;
    else if (src >= 0) to[src] = tiled[i];
  }
}

MxArgs args_of(const Level& L, const MixedSys& M, const Phys& ph) {
  return MxArgs{L.nc, L.nz, M.ne, L.Np, M.nh, ph.a, ph.c2, ph.wn2, M.edge, M.enb, M.ecoef, M.emass, M.cedge, M.zd, M.m3};
}

int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

}  // namespace

void launch_mixed_coeffs(const Level& L, const MixedSys& M, const Phys& ph, cudaStream_t s) {
  k_mx_edge_coeffs<<<(M.nep + 127) / 128, 128, 0, s>>>(M.ne, M.nep, ph.dz, M.edge, M.cedge, L.verts, M.enb,
                                                      M.ecoef, M.emass);
  k_mx_cell_coeffs<<<(unsigned)((L.Np + 255) / 256), 256, 0, s>>>(L.nc, L.nz, L.Np, ph.R, ph.dz, L.A1, M.zd,
                                                                   M.m3);
}

void launch_mixed_apply(const Level& L, const MixedSys& M, const Phys& ph, const double* x, double* y,
                        cudaStream_t s) {
  k_mx_apply<<<grid_for(M.n), 256, 0, s>>>(args_of(L, M, ph), x, y);
}

void launch_mixed_pre_lower(const Level& L, const MixedSys& M, const Phys& ph, const double* r, double* rp,
                            cudaStream_t s) {
  k_mx_pre_lower<<<grid_for(L.Np), 256, 0, s>>>(args_of(L, M, ph), r, rp);
}

void launch_mixed_pre_upper(const Level& L, const MixedSys& M, const Phys& ph, const double* r, double* z,
                            cudaStream_t s) {
  k_mx_pre_upper<<<grid_for(M.nh + L.Np), 256, 0, s>>>(args_of(L, M, ph), r, z);
}

void launch_mixed_layout(const Level& L, const MixedSys& M, bool to_tiled, const double* u_col, const double* p_col,
                         double* tiled, double* u_out, double* p_out, cudaStream_t s) {
  k_mx_layout<<<grid_for(M.n), 256, 0, s>>>(MxArgs{L.nc, L.nz, M.ne, L.Np, M.nh, 0, 0, 0}, to_tiled, u_col, p_col,
                                             tiled, u_out, p_out);
}

}  // namespace hmg
