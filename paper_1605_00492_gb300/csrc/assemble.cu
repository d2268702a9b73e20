// Assembly of the lumped Helmholtz operator H^ (Sec. 4.2, Eq. Preconditioner)
// and the factorisation of its column block H^_z (Eq. HHgeneralbanded,
// Thomas solve of Sec. 4.3.1) on the GPU.
//
// Geometry of cell K = (column T, layer l): the straight prism over the flat
// triangle T scaled to the mid-layer radius rho_l = R + (l + 1/2) dz, area
// A_l = A1_T rho_l^2, volume A_l dz.  With unit-flux velocity functions:
//   horizontal face across edge k:   g_k = w_c^2 dz / (sigma_T,k + sigma_T',k')
//   vertical face between l, l+1:    g_z = w_c^2 / (1 + w_N^2) /
//                                          (dz / (3 A_l theta_l) + dz / (3 A_l+1 theta_l+1))
//   H^_KK = |K| + sum of the couplings of its faces, H^_KK' = -g_f,
// where sigma = (|a|^2 + |b|^2 + a.b) / (24 |T|) is the integral of |w|^2 of
// the unit-flux RT0 function (a, b: edge vectors from the opposite vertex).
#include "hmg_internal.h"

namespace hmg {

namespace {

__device__ __forceinline__ int64_t tile_base(int c, int nz) {
  return (int64_t)(c >> 5) * (TW * nz) + (c & 31);
}

__global__ void k_geometry(int nc, const double* __restrict__ verts, double* __restrict__ A1,
                           double4_32a* __restrict__ sigma) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  double p[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int j = 0; j < 3; ++j) p[k][j] = verts[(size_t)c * 9 + 3 * k + j];
  double ux = p[1][0] - p[0][0], uy = p[1][1] - p[0][1], uz = p[1][2] - p[0][2];
  double vx = p[2][0] - p[0][0], vy = p[2][1] - p[0][1], vz = p[2][2] - p[0][2];
  double cx = uy * vz - uz * vy, cy = uz * vx - ux * vz, cz = ux * vy - uy * vx;
  double area = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
  double s[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    int i = (k + 1) % 3, j = (k + 2) % 3;
    double ax = p[i][0] - p[k][0], ay = p[i][1] - p[k][1], az = p[i][2] - p[k][2];
    double bx = p[j][0] - p[k][0], by = p[j][1] - p[k][1], bz = p[j][2] - p[k][2];
    double aa = ax * ax + ay * ay + az * az;
    double bb = bx * bx + by * by + bz * bz;
    double ab = ax * bx + ay * by + az * bz;
    s[k] = (aa + bb + ab) / (24.0 * area);
  }
  A1[c] = area;
  sigma[c] = make_double4_32a(s[0], s[1], s[2], 0.0);
}

__device__ __forceinline__ double comp(const double4_32a& v, int k) {
  return k == 0 ? v.x : (k == 1 ? v.y : v.z);
}
__device__ __forceinline__ int compi(const int4& v, int k) {
  return k == 0 ? v.x : (k == 1 ? v.y : v.z);
}

__global__ void k_couplings(int nc, const int4* __restrict__ nbr, const double4_32a* __restrict__ sigma,
                            double wc2_dz, double4_32a* __restrict__ gh) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  int4 nb = nbr[c];
  double4_32a sc = sigma[c];
  double g[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    int n = compi(nb, k);
    int4 nn = nbr[n];
    int kn = nn.x == c ? 0 : (nn.y == c ? 1 : 2);
    // sum in a fixed operand order on both sides of the face: a + b == b + a
    g[k] = wc2_dz / (comp(sc, k) + comp(sigma[n], kn));
  }
  gh[c] = make_double4_32a(g[0], g[1], g[2], g[0] + g[1] + g[2]);
}

struct BandArgs {
  int nc, nz;
  double R, dz, vfac;
  const double* A1;
  const double4_32a* gh;
  const double* theta;   // tiled, may be null
};

// Coupling of the vertical face between layers l and l+1 of column c; both
// neighbouring cells evaluate the same expression, so H^ is exactly symmetric.
__device__ __forceinline__ double vface(const BandArgs& a, int c, int l, int64_t t_l) {
  double rl = a.R + (l + 0.5) * a.dz, ru = a.R + (l + 1.5) * a.dz;
  double Al = a.A1[c] * rl * rl, Au = a.A1[c] * ru * ru;
  double tl = a.theta ? a.theta[t_l] : 1.0;
  double tu = a.theta ? a.theta[t_l + TW] : 1.0;
  return a.vfac / (a.dz / (3.0 * Al * tl) + a.dz / (3.0 * Au * tu));
}

__global__ void k_bands(BandArgs a, int64_t Np, double* __restrict__ d, double* __restrict__ e) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= Np) return;
  int lane = (int)(t & 31);
  int64_t tile = t / (TW * a.nz);
  int l = (int)((t >> 5) % a.nz);
  int c = (int)(tile * TW + lane);
  if (c >= a.nc) {
    d[t] = 0.0;
    e[t] = 0.0;
    return;
  }
  double rho = a.R + (l + 0.5) * a.dz;
  double vol = a.A1[c] * rho * rho * a.dz;
  double gdn = l > 0 ? vface(a, c, l - 1, t - TW) : 0.0;
  double gup = l < a.nz - 1 ? vface(a, c, l, t) : 0.0;
  d[t] = vol + a.gh[c].w + gdn + gup;
  e[t] = -gdn;
}

// Twisted factorisation of each column block H^_z = N D N^T (no pivoting:
// H^_z is strictly diagonally dominant), twist at layer m (nz / 2, or nz - 1
// which is the plain L D L^T):
//   rows l < m:  N[l][l-1] = lambda_l, eliminated top-down
//   rows l > m:  N[l][l+1] = mu_l,     eliminated bottom-up
//   row m:       both lambda_m and mu_m.
// With m = nz / 2, solving N y = r, D z = y, N^T x = z runs two recurrences
// of about nz / 2 steps each (top and bottom halves) instead of one of nz,
// with the same 3 operations per cell as a Thomas solve.  Stored per cell:
//   lo[l] = lambda_l (l <= m, lo[0] = 0), mu_l (m < l < nz - 1), 0 at l = nz - 1
//   w[l]  = omega / D_l
// and per column mt = mu_m (0 when m = nz - 1).  Computed in FP64; TF = float
// rounds the FP64 factors once as they are stored (the FP32 copies, which may
// twist at another row).  Optionally (los, mts not null) the multipliers
// scaled to their own row's pivot, lambda_l D_l-1 / D_l = e_l / D_l and
// mu_l D_l+1 / D_l = e_l+1 / D_l: with them the elimination runs directly in
// z = (omega / D) y, z_l = (omega / D_l) R_l - los_l z_l-1 (resp. z_l+1).
template <typename TF>
__global__ void k_ldl(int nc, int nz, int m, double omega, const double* __restrict__ d,
                      const double* __restrict__ e, TF* __restrict__ lo, TF* __restrict__ w,
                      TF* __restrict__ mt, TF* __restrict__ los, TF* __restrict__ mts) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const int64_t s = tile_base(c, nz);
  auto at = [&](int l) { return s + (int64_t)l * TW; };
  double Dtop = 0.0, Dbot = 0.0;
  if (m >= 1) {  // top half, rows 0..m-1
    double D = d[at(0)];
    lo[at(0)] = 0.0;
    w[at(0)] = omega / D;
    if (los) los[at(0)] = 0.0;
    for (int l = 1; l < m; ++l) {
      const double el = e[at(l)];
      const double lam = el / D;
      D = d[at(l)] - lam * el;
      lo[at(l)] = lam;
      w[at(l)] = omega / D;
      if (los) los[at(l)] = el / D;
    }
    Dtop = D;
  }
  if (m <= nz - 2) {  // bottom half, rows nz-1..m+1
    double D = d[at(nz - 1)];
    lo[at(nz - 1)] = 0.0;
    w[at(nz - 1)] = omega / D;
    if (los) los[at(nz - 1)] = 0.0;
    for (int l = nz - 2; l > m; --l) {
      const double eu = e[at(l + 1)];
      const double mu = eu / D;
      D = d[at(l)] - mu * eu;
      lo[at(l)] = mu;
      w[at(l)] = omega / D;
      if (los) los[at(l)] = eu / D;
    }
    Dbot = D;
  }
  double Dm = d[at(m)];
  double lam_m = 0.0, mu_m = 0.0;
  if (m >= 1) {
    const double el = e[at(m)];
    lam_m = el / Dtop;
    Dm -= lam_m * el;
  }
  if (m <= nz - 2) {
    const double eu = e[at(m + 1)];
    mu_m = eu / Dbot;
    Dm -= mu_m * eu;
  }
  lo[at(m)] = lam_m;
  w[at(m)] = omega / Dm;
  mt[c] = mu_m;
  if (los) {
    los[at(m)] = m >= 1 ? e[at(m)] / Dm : 0.0;
    mts[c] = m <= nz - 2 ? e[at(m + 1)] / Dm : 0.0;
  }
}

__global__ void k_to_fp32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

__global__ void k_gh_to_fp32(int n, const double4_32a* __restrict__ a, float4* __restrict__ b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    double4_32a v = a[i];
    b[i] = make_float4((float)v.x, (float)v.y, (float)v.z, (float)v.w);
  }
}

// Coarse theta = mean over the four children, layer by layer.
__global__ void k_theta_restrict(int nc_coarse, int nz, const double* __restrict__ fine,
                                 double* __restrict__ coarse) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)nc_coarse * nz) return;
  int C = (int)(t / nz), l = (int)(t % nz);
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 4; ++j) s += fine[tile_base(4 * C + j, nz) + (int64_t)l * TW];
  coarse[tile_base(C, nz) + (int64_t)l * TW] = 0.25 * s;
}

// grad_K = -sum over the vertical faces f of K of
//          (dg_f / dtheta_K) (lambda_K - lambda_K') (p_K - p_K'),
// dg_f / dtheta_K = vfac (dz / (3 A_K theta_K^2)) / Mz_f^2.
// p, lambda, grad in the COLUMN layout (cell c * nz + l); theta tiled.
__global__ void k_theta_grad(BandArgs a, const double* __restrict__ p, const double* __restrict__ lam,
                             double* __restrict__ grad) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)a.nc * a.nz) return;
  int c = (int)(i / a.nz), l = (int)(i % a.nz);
  int64_t t = tile_base(c, a.nz) + (int64_t)l * TW;
  double rho = a.R + (l + 0.5) * a.dz;
  double AK = a.A1[c] * rho * rho;
  double thK = a.theta ? a.theta[t] : 1.0;
  double dm = a.dz / (3.0 * AK * thK * thK);
  double acc = 0.0;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    int ln = side == 0 ? l - 1 : l + 1;
    if (ln < 0 || ln >= a.nz) continue;
    double rn = a.R + (ln + 0.5) * a.dz;
    double An = a.A1[c] * rn * rn;
    double thn = a.theta ? a.theta[t + (side == 0 ? -TW : TW)] : 1.0;
    double M = a.dz / (3.0 * AK * thK) + a.dz / (3.0 * An * thn);
    int64_t j = i + (side == 0 ? -1 : 1);
    acc += (lam[i] - lam[j]) * (p[i] - p[j]) / (M * M);
  }
  grad[i] = -a.vfac * dm * acc;
}

inline unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

void launch_geometry(const Level& L, cudaStream_t s) {
  k_geometry<<<blocks_for(L.nc, 128), 128, 0, s>>>(L.nc, L.verts, L.A1, L.sigma);
}

void launch_couplings(const Level& L, double wc2_dz, cudaStream_t s) {
  k_couplings<<<blocks_for(L.nc, 128), 128, 0, s>>>(L.nc, L.nbr, L.sigma, wc2_dz, L.gh);
}

static BandArgs band_args(const Level& L, const Phys& ph) {
  BandArgs a;
  a.nc = L.nc;
  a.nz = L.nz;
  a.R = ph.R;
  a.dz = ph.dz;
  a.vfac = ph.vfac;
  a.A1 = L.A1;
  a.gh = L.gh;
  a.theta = L.theta;
  return a;
}

void launch_bands(const Level& L, const Phys& ph, cudaStream_t s) {
  k_bands<<<blocks_for(L.Np, 256), 256, 0, s>>>(band_args(L, ph), L.Np, L.d, L.e);
}

void launch_ldl(const Level& L, double omega, cudaStream_t s) {
  k_ldl<double><<<blocks_for(L.nc, 64), 64, 0, s>>>(L.nc, L.nz, L.twist, omega, L.d, L.e, L.lo, L.w, L.mt, L.los,
                                                     L.mts);
  k_ldl<float><<<blocks_for(L.nc, 64), 64, 0, s>>>(L.nc, L.nz, L.twist32, omega, L.d, L.e, L.lo32, L.w32, L.mt32,
                                                    nullptr, nullptr);
}

void launch_to_fp32(const Level& L, cudaStream_t s) {
  unsigned g = blocks_for(L.Np, 256);
  k_to_fp32<<<g, 256, 0, s>>>(L.Np, L.d, L.d32);
  k_to_fp32<<<g, 256, 0, s>>>(L.Np, L.e, L.e32);
  k_gh_to_fp32<<<blocks_for(L.ncp, 128), 128, 0, s>>>(L.ncp, L.gh, L.gh32);
}

void launch_theta_restrict(const Level& fine, const Level& coarse, cudaStream_t s) {
  int64_t n = (int64_t)coarse.nc * coarse.nz;
  k_theta_restrict<<<blocks_for(n, 256), 256, 0, s>>>(coarse.nc, coarse.nz, fine.theta, coarse.theta);
}

void launch_theta_grad(const Level& L, const Phys& ph, const double* p_col, const double* lam_col,
                       double* grad_col, cudaStream_t s) {
  k_theta_grad<<<blocks_for(L.N, 256), 256, 0, s>>>(band_args(L, ph), p_col, lam_col, grad_col);
}

}  // namespace hmg
