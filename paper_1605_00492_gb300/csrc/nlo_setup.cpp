// Host assembly of the next-to-lowest-order (NLO) operator (Table
// "FiniteElements": pressure DG1(T) x DG1(z), horizontal velocity
// BDFM1(T) x DG1(z), vertical velocity DG1(T) x P2(z)) and the block
// factorisation of its column part (Eq. HHgeneralbanded, Sec. 4.3).
//
// The lumped operator is Eq. (Preconditioner):
//   H^ = M3 + w_c^2 D_h Mh_inv D_h^T + w_c^2 / (1 + w_N^2) D_z Mz_inv D_z^T,
// with the lumped inverses of Eq. (LumpedMass).  Its unknowns per cell are
// u = 2 j + m: j the vertex of the face (DG1 nodal at the vertices), m = 0 / 1
// the bottom / top of the layer (DG1 nodal in z).  Per cell the operator has
// three kinds of 6 x 6 blocks: the column-diagonal block (cell with itself),
// the column sub-diagonal block (cell with the cell below) and, per edge,
// the block that couples the cell with the same layer of the neighbour
// column.  The neighbour blocks do not depend on the layer: the horizontal
// integrals are scale invariant and dz is uniform.
//
// BDFM1(T) = P1(T)^2 + span{lam_i lam_j t_k}; its degrees of freedom are the
// length-scaled outward normal components at the points 1/3 and 2/3 of each
// edge (edge k runs from vertex k+1 to vertex k+2) and the moments against
// the Whitney functions lam_i grad lam_j - lam_j grad lam_i.  Both families
// are invariant under the contravariant Piola map, so the basis is built
// once on the reference triangle (0,0), (1,0), (0,1) and mapped: the
// divergence integrals int_T lam_j div v_a are the same on every triangle and
// the energies are int_T |v_a|^2 = int_Tref v^T G v / det J with the metric
// G = J^T J of the triangle's affine map J.
#include <algorithm>
#include <array>
#include <cmath>
#include <stdexcept>
#include <vector>

#include "hmg_internal.h"

namespace hmg {

namespace {

using Mat6 = std::array<double, 36>;

// Gauss-Legendre points and weights on [0, 1] by Newton iteration on P_n.
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (t * p1 - p0) / (t * t - 1.0);
      double dt = p1 / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[i] = 0.5 * (1.0 - t);
    w[i] = 1.0 / ((1.0 - t * t) * dp * dp);   // 2 / ((1 - t^2) P_n'^2), halved for [0, 1]
  }
}

// Quadrature on the reference triangle by the collapsed (Duffy) product rule.
struct TriRule {
  std::vector<double> x, y, w;
};

TriRule tri_rule(int n) {
  std::vector<double> g, gw;
  gauss_legendre01(n, g, gw);
  TriRule r;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      r.x.push_back(g[a]);
      r.y.push_back(g[b] * (1.0 - g[a]));
      r.w.push_back(gw[a] * gw[b] * (1.0 - g[a]));
    }
  return r;
}

const double kVx[3] = {0.0, 1.0, 0.0}, kVy[3] = {0.0, 0.0, 1.0};
const double kGx[3] = {-1.0, 1.0, 0.0}, kGy[3] = {-1.0, 0.0, 1.0};   // grad lam_i on the reference

void bary(double x, double y, double lam[3]) {
  lam[0] = 1.0 - x - y;
  lam[1] = x;
  lam[2] = y;
}

// Spanning function f of the reference space at (x, y): value and divergence.
void span_eval(int f, double x, double y, double v[2], double* div) {
  double lam[3];
  bary(x, y, lam);
  if (f < 6) {                 // lam_m e_axis
    const int m = f / 2, ax = f % 2;
    v[0] = ax == 0 ? lam[m] : 0.0;
    v[1] = ax == 1 ? lam[m] : 0.0;
    *div = ax == 0 ? kGx[m] : kGy[m];
  } else {                     // lam_i lam_j t_k
    const int k = f - 6, i = (k + 1) % 3, j = (k + 2) % 3;
    const double tx = kVx[j] - kVx[i], ty = kVy[j] - kVy[i];
    v[0] = lam[i] * lam[j] * tx;
    v[1] = lam[i] * lam[j] * ty;
    *div = (lam[j] * kGx[i] + lam[i] * kGx[j]) * tx + (lam[j] * kGy[i] + lam[i] * kGy[j]) * ty;
  }
}

// Gauss-Jordan inverse with partial pivoting (n x n, row-major, in place).
void invert(double* a, int n) {
  std::vector<double> inv(n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(a[r * n + col]) > std::fabs(a[piv * n + col])) piv = r;
    if (a[piv * n + col] == 0.0) throw std::runtime_error("singular matrix in the NLO setup");
    if (piv != col)
      for (int c = 0; c < n; ++c) {
        std::swap(a[piv * n + c], a[col * n + c]);
        std::swap(inv[piv * n + c], inv[col * n + c]);
      }
    const double d = 1.0 / a[col * n + col];
    for (int c = 0; c < n; ++c) {
      a[col * n + c] *= d;
      inv[col * n + c] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = a[r * n + col];
      if (f == 0.0) continue;
      for (int c = 0; c < n; ++c) {
        a[r * n + c] -= f * a[col * n + c];
        inv[r * n + c] -= f * inv[col * n + c];
      }
    }
  }
  for (int i = 0; i < n * n; ++i) a[i] = inv[i];
}

}  // namespace

// The reference BDFM1 element: div[j][a] = int lam_j div v_a (the same on
// every triangle) and the second moments Q[a] = int v_a v_a^T (00, 01, 11).
struct RefBDFM {
  double div[3][9];
  double Q[9][3];
  double M[9][9][4];   // int v_a,x v_a',x ; v_a,x v_a',y ; v_a,y v_a',x ; v_a,y v_a',y
};

RefBDFM reference_bdfm() {
  const TriRule rule = tri_rule(5);
  // Phi[dof][f]
  double Phi[81];
  for (int f = 0; f < 9; ++f) {
    for (int k = 0; k < 3; ++k) {
      const int i = (k + 1) % 3, j = (k + 2) % 3;
      const double ex = kVx[j] - kVx[i], ey = kVy[j] - kVy[i];
      const double len = std::sqrt(ex * ex + ey * ey);
      // outward unit normal: perpendicular to the edge, away from vertex k
      double nx = ey / len, ny = -ex / len;
      if (nx * (kVx[i] - kVx[k]) + ny * (kVy[i] - kVy[k]) < 0) {
        nx = -nx;
        ny = -ny;
      }
      for (int q = 0; q < 2; ++q) {
        const double s = (q + 1) / 3.0;
        double v[2], dv;
        span_eval(f, kVx[i] + s * ex, kVy[i] + s * ey, v, &dv);
        Phi[(2 * k + q) * 9 + f] = len * (v[0] * nx + v[1] * ny);
      }
      double mom = 0.0;
      for (size_t p = 0; p < rule.w.size(); ++p) {
        double lam[3], v[2], dv;
        bary(rule.x[p], rule.y[p], lam);
        span_eval(f, rule.x[p], rule.y[p], v, &dv);
        const double wx = lam[i] * kGx[j] - lam[j] * kGx[i], wy = lam[i] * kGy[j] - lam[j] * kGy[i];
        mom += rule.w[p] * (v[0] * wx + v[1] * wy);
      }
      Phi[(6 + k) * 9 + f] = mom;
    }
  }
  invert(Phi, 9);   // now C[f][a] = Phi^-1: basis a = sum_f C[f][a] span_f
  RefBDFM R{};
  for (size_t p = 0; p < rule.w.size(); ++p) {
    double lam[3];
    bary(rule.x[p], rule.y[p], lam);
    double sv[9][2], sd[9];
    for (int f = 0; f < 9; ++f) span_eval(f, rule.x[p], rule.y[p], sv[f], &sd[f]);
    double vx[9], vy[9];
    for (int a = 0; a < 9; ++a) {
      double dv = 0;
      vx[a] = vy[a] = 0;
      for (int f = 0; f < 9; ++f) {
        vx[a] += Phi[f * 9 + a] * sv[f][0];
        vy[a] += Phi[f * 9 + a] * sv[f][1];
        dv += Phi[f * 9 + a] * sd[f];
      }
      const double w = rule.w[p];
      R.Q[a][0] += w * vx[a] * vx[a];
      R.Q[a][1] += w * vx[a] * vy[a];
      R.Q[a][2] += w * vy[a] * vy[a];
      for (int j = 0; j < 3; ++j) R.div[j][a] += w * lam[j] * dv;
    }
    for (int a = 0; a < 9; ++a)
      for (int a2 = 0; a2 < 9; ++a2) {
        const double w = rule.w[p];
        R.M[a][a2][0] += w * vx[a] * vx[a2];
        R.M[a][a2][1] += w * vx[a] * vy[a2];
        R.M[a][a2][2] += w * vy[a] * vx[a2];
        R.M[a][a2][3] += w * vy[a] * vy[a2];
      }
  }
  return R;
}

NloHost nlo_assemble_host(const std::vector<double>& verts, const std::vector<int32_t>& nbrs, int nc, int nz,
                          const Phys& ph) {
  const RefBDFM R = reference_bdfm();
  NloHost out;
  out.nc = nc;
  out.nz = nz;
  out.diag.assign((size_t)nc * nz * 36, 0.0);
  out.sub.assign((size_t)nc * nz * 36, 0.0);
  out.nbr.assign((size_t)nc * 3 * 36, 0.0);
  out.nbr3.assign((size_t)nc * 3 * 9, 0.0);
  const double dz = ph.dz;

  // horizontal energies hm[c][a] = int_T |v_a|^2 on the unit-sphere flat triangle
  std::vector<double> hm((size_t)nc * 9), area1(nc);
  auto vert = [&](int c, int k, int x) { return verts[(size_t)c * 9 + 3 * k + x]; };
  for (int c = 0; c < nc; ++c) {
    double J0[3], J1[3];
    for (int x = 0; x < 3; ++x) {
      J0[x] = vert(c, 1, x) - vert(c, 0, x);
      J1[x] = vert(c, 2, x) - vert(c, 0, x);
    }
    const double g00 = J0[0] * J0[0] + J0[1] * J0[1] + J0[2] * J0[2];
    const double g01 = J0[0] * J1[0] + J0[1] * J1[1] + J0[2] * J1[2];
    const double g11 = J1[0] * J1[0] + J1[1] * J1[1] + J1[2] * J1[2];
    const double det = std::sqrt(g00 * g11 - g01 * g01);   // = 2 |T|
    area1[c] = 0.5 * det;
    for (int a = 0; a < 9; ++a)
      hm[(size_t)c * 9 + a] = (g00 * R.Q[a][0] + 2.0 * g01 * R.Q[a][1] + g11 * R.Q[a][2]) / det;
  }

  // vertical-in-layer integrals (closed forms on [0, 1])
  const double MZ1[2][2] = {{1.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 1.0 / 3.0}};
  const double Z2[2][2] = {{5.0 / 12.0, 4.0 / 12.0}, {4.0 / 12.0, 5.0 / 12.0}};   // 3 MZ1 MZ1
  // G[m][kz] = int_0^1 eta_m zeta_kz' for DG1 nodal eta and P2 nodal zeta
  const double G[2][3] = {{-5.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0}, {-1.0 / 6.0, -2.0 / 3.0, 5.0 / 6.0}};
  const double P2D[3] = {4.0 / 30.0, 16.0 / 30.0, 4.0 / 30.0};   // diagonal of the P2 mass on [0, 1]
  auto PM = [](int j, int i) { return (i == j ? 2.0 : 1.0) / 12.0; };   // int_T lam_j lam_i / |T|

  for (int c = 0; c < nc; ++c) {
    // the horizontal part: own block and the three neighbour blocks
    double own[3][3] = {};
    for (int k = 0; k < 3; ++k) {
      const int n = nbrs[3 * c + k];
      int kn = 0;
      while (kn < 3 && nbrs[3 * n + kn] != c) ++kn;
      if (kn == 3) throw std::runtime_error("mesh neighbours are not symmetric");
      // the same edge seen from n: same or reversed direction
      const int i = (k + 1) % 3, in = (kn + 1) % 3, jn = (kn + 2) % 3;
      double dsame = 0.0, drev = 0.0;
      for (int x = 0; x < 3; ++x) {
        dsame += std::fabs(vert(c, i, x) - vert(n, in, x));
        drev += std::fabs(vert(c, i, x) - vert(n, jn, x));
      }
      if (!(dsame < 1e-12 || drev < 1e-12)) throw std::runtime_error("neighbour edge does not match");
      const bool rev = drev < dsame;
      double nb[3][3] = {};
      for (int q = 0; q < 2; ++q) {
        const int a = 2 * k + q, an = 2 * kn + (rev ? 1 - q : q);
        const double msum = hm[(size_t)c * 9 + a] + hm[(size_t)n * 9 + an];
        for (int j = 0; j < 3; ++j)
          for (int jj = 0; jj < 3; ++jj) {
            own[j][jj] += R.div[j][a] * R.div[jj][a] / msum;
            nb[j][jj] -= R.div[j][a] * R.div[jj][an] / msum;
          }
      }
      double* blk = &out.nbr[((size_t)c * 3 + k) * 36];
      for (int j = 0; j < 3; ++j)
        for (int jj = 0; jj < 3; ++jj) out.nbr3[((size_t)c * 3 + k) * 9 + 3 * j + jj] = ph.wc2 * dz * nb[j][jj];
      for (int u = 0; u < 6; ++u)
        for (int uu = 0; uu < 6; ++uu) blk[u * 6 + uu] = ph.wc2 * dz * nb[u / 2][uu / 2] * Z2[u % 2][uu % 2];
    }
    for (int k = 0; k < 3; ++k) {   // interior unknowns
      const int a = 6 + k;
      const double m = hm[(size_t)c * 9 + a];
      for (int j = 0; j < 3; ++j)
        for (int jj = 0; jj < 3; ++jj) own[j][jj] += R.div[j][a] * R.div[jj][a] / m;
    }
    // the column blocks, layer by layer
    for (int l = 0; l < nz; ++l) {
      const double rho = ph.R + (l + 0.5) * dz;
      const double At = area1[c] * rho * rho;
      auto area = [&](int layer) {
        const double r = ph.R + (layer + 0.5) * dz;
        return area1[c] * r * r;
      };
      // lumped vertical masses of the nodes of this cell (bottom, middle,
      // top); equal for the three vertices i since int lam_i^2 is |T| / 6
      double mz[3];
      mz[1] = dz / 24.0 * P2D[1] / At;
      mz[0] = l > 0 ? dz / 24.0 * P2D[0] * (1.0 / At + 1.0 / area(l - 1)) : 0.0;
      mz[2] = l < nz - 1 ? dz / 24.0 * P2D[2] * (1.0 / At + 1.0 / area(l + 1)) : 0.0;
      double* A = &out.diag[((size_t)c * nz + l) * 36];
      for (int u = 0; u < 6; ++u)
        for (int uu = 0; uu < 6; ++uu) {
          const int j = u / 2, m = u % 2, jj = uu / 2, mm = uu % 2;
          double v = At * dz * PM(j, jj) * MZ1[m][mm];
          v += ph.wc2 * dz * own[j][jj] * Z2[m][mm];
          double vz = 0.0;
          for (int kz = 0; kz < 3; ++kz) {
            if (mz[kz] == 0.0) continue;
            for (int i = 0; i < 3; ++i) vz += (PM(j, i) / 2.0 * G[m][kz]) * (PM(jj, i) / 2.0 * G[mm][kz]) / mz[kz];
          }
          A[u * 6 + uu] = v + ph.vfac * vz;
        }
      if (l > 0) {
        double* C = &out.sub[((size_t)c * nz + l) * 36];
        for (int u = 0; u < 6; ++u)
          for (int uu = 0; uu < 6; ++uu) {
            const int j = u / 2, m = u % 2, jj = uu / 2, mm = uu % 2;
            double vz = 0.0;
            for (int i = 0; i < 3; ++i) vz += (PM(j, i) / 2.0 * G[m][0]) * (PM(jj, i) / 2.0 * G[mm][2]) / mz[0];
            C[u * 6 + uu] = ph.vfac * vz;
          }
      }
    }
  }
  return out;
}

// Block L D L^T of the column part: Dt_0 = A_0, L_l = C_l Dt_(l-1)^-1,
// Dt_l = A_l - L_l C_l^T; returns L_l (l >= 1) and omega Dt_l^-1 per cell.
void nlo_factor_host(const NloHost& H, double omega, std::vector<double>& Lf, std::vector<double>& Dinv) {
  const int nc = H.nc, nz = H.nz;
  Lf.assign((size_t)nc * nz * 36, 0.0);
  Dinv.assign((size_t)nc * nz * 36, 0.0);
  for (int c = 0; c < nc; ++c) {
    Mat6 Dprev{}, Dt{};
    for (int l = 0; l < nz; ++l) {
      const size_t o = ((size_t)c * nz + l) * 36;
      for (int i = 0; i < 36; ++i) Dt[i] = H.diag[o + i];
      if (l > 0) {
        const double* C = &H.sub[o];
        double* Ll = &Lf[o];
        for (int r = 0; r < 6; ++r)            // L = C Dprev^-1 (Dprev holds the inverse)
          for (int s = 0; s < 6; ++s) {
            double v = 0.0;
            for (int t = 0; t < 6; ++t) v += C[r * 6 + t] * Dprev[t * 6 + s];
            Ll[r * 6 + s] = v;
          }
        for (int r = 0; r < 6; ++r)            // Dt -= L C^T
          for (int s = 0; s < 6; ++s) {
            double v = 0.0;
            for (int t = 0; t < 6; ++t) v += Ll[r * 6 + t] * C[s * 6 + t];
            Dt[r * 6 + s] -= v;
          }
      }
      Mat6 inv = Dt;
      invert(inv.data(), 6);
      for (int i = 0; i < 36; ++i) Dinv[o + i] = omega * inv[i];
      Dprev = inv;
    }
  }
}

// ---- the NLO velocity-pressure system (Eq. PressureVelocitySystem at NLO)
//
// Unknowns (the NLO mixed COLUMN layout of hmg.h): horizontal edge velocity
// ((E nz + l) 2 + q) 2 + b for edge E of the edge list (t, k, tn, kn), point
// q along edge k of column t and the normal of t; interior horizontal
// velocity ((c nz + l) 3 + k) 2 + b; vertical velocity (c 3 + i) (2 nz - 1) +
// node - 1 (node 1 .. 2 nz - 1 of P2 in z); pressure ((c nz + l) 3 + j) 2 + m.
// Per cell the element matrices are: the BDFM1 mass of the column (the
// Piola-mapped reference moments and the triangle's metric) times the DG1
// mass in z over dz; the vertical mass lam_i lam_i' / (4 |T_l|^2) times the
// P2 mass in z; the divergence pairings (reference integrals, the same on
// every triangle) and the DG1 pressure mass.  A is assembled as CSR from the
// cells' triplets (counting sort by row, then sort and merge each row).
namespace {

struct Trip {
  int32_t r, c;
  double v;
};

void to_csr(std::vector<Trip>& t, int64_t nrows, int64_t ncols, Csr& out) {
  out.nrows = nrows;
  out.ncols = ncols;
  std::vector<int64_t> cnt(nrows + 1, 0);
  for (const Trip& x : t) ++cnt[x.r + 1];
  for (int64_t i = 0; i < nrows; ++i) cnt[i + 1] += cnt[i];
  std::vector<int32_t> cs(t.size());
  std::vector<double> vs(t.size());
  {
    std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
    for (const Trip& x : t) {
      const int64_t p = pos[x.r]++;
      cs[p] = x.c;
      vs[p] = x.v;
    }
  }
  std::vector<Trip>().swap(t);
  out.ptr.assign(nrows + 1, 0);
  out.col.clear();
  out.val.clear();
  out.col.reserve(cs.size() / 2);
  out.val.reserve(cs.size() / 2);
  std::vector<std::pair<int32_t, double>> row;
  for (int64_t i = 0; i < nrows; ++i) {
    row.clear();
    for (int64_t p = cnt[i]; p < cnt[i + 1]; ++p) row.emplace_back(cs[p], vs[p]);
    std::sort(row.begin(), row.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
    for (size_t k = 0; k < row.size();) {
      double v = 0.0;
      const int32_t c = row[k].first;
      while (k < row.size() && row[k].first == c) v += row[k++].second;
      out.col.push_back(c);
      out.val.push_back(v);
    }
    out.ptr[i + 1] = (int64_t)out.col.size();
  }
}

}  // namespace

NloMixedHost nlo_mixed_assemble_host(const std::vector<double>& verts, const std::vector<int32_t>& nbrs,
                                     const std::vector<int32_t>& edges, int nc, int nz, const Phys& ph) {
  const RefBDFM R = reference_bdfm();
  const int ne = (int)(edges.size() / 4);
  NloMixedHost X;
  X.nue = (int64_t)ne * nz * 4;
  X.nui = (int64_t)nc * nz * 6;
  X.nuz = (int64_t)nc * 3 * (2 * nz - 1);
  X.nu = X.nue + X.nui + X.nuz;
  X.np = (int64_t)nc * nz * 6;
  X.n = X.nu + X.np;
  if (X.n >= (int64_t)1 << 31) throw std::runtime_error("NLO velocity-pressure system too large for 32-bit indices");
  const double dz = ph.dz, a = ph.a, ac2 = ph.a * ph.c2, vz = 1.0 + ph.wn2;
  auto vert = [&](int c, int k, int x) { return verts[(size_t)c * 9 + 3 * k + x]; };
  // per column and local BDFM1 unknown: global edge-or-interior index base and sign
  std::vector<int64_t> gbase((size_t)nc * 9);
  std::vector<double> gsign((size_t)nc * 9, 1.0);
  for (int c = 0; c < nc; ++c)
    for (int k = 0; k < 3; ++k) gbase[(size_t)c * 9 + 6 + k] = -1 - k;   // interior: resolved per layer below
  for (int e = 0; e < ne; ++e) {
    const int t = edges[4 * e], k = edges[4 * e + 1], tn = edges[4 * e + 2], kn = edges[4 * e + 3];
    const int i = (k + 1) % 3, in = (kn + 1) % 3, jn = (kn + 2) % 3;
    double dsame = 0.0, drev = 0.0;
    for (int x = 0; x < 3; ++x) {
      dsame += std::fabs(vert(t, i, x) - vert(tn, in, x));
      drev += std::fabs(vert(t, i, x) - vert(tn, jn, x));
    }
    if (!(dsame < 1e-12 || drev < 1e-12)) throw std::runtime_error("neighbour edge does not match");
    const bool rev = drev < dsame;
    for (int q = 0; q < 2; ++q) {
      gbase[(size_t)t * 9 + 2 * k + q] = ((int64_t)e * nz * 2 + q) * 2;             // + l * 4 + b
      const int qn = rev ? 1 - q : q;
      gbase[(size_t)tn * 9 + 2 * kn + qn] = ((int64_t)e * nz * 2 + q) * 2;
      gsign[(size_t)tn * 9 + 2 * kn + qn] = -1.0;
    }
  }
  (void)nbrs;
  const double MZ1[2][2] = {{1.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 1.0 / 3.0}};
  const double G[2][3] = {{-5.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0}, {-1.0 / 6.0, -2.0 / 3.0, 5.0 / 6.0}};
  const double P2[3][3] = {{4.0 / 30, 2.0 / 30, -1.0 / 30}, {2.0 / 30, 16.0 / 30, 2.0 / 30}, {-1.0 / 30, 2.0 / 30, 4.0 / 30}};
  auto PM = [](int j, int i) { return (i == j ? 2.0 : 1.0) / 12.0; };
  const int nzn = 2 * nz - 1;

  std::vector<Trip> tA, tD, tDt;
  tA.reserve((size_t)nc * nz * 770);
  tD.reserve((size_t)nc * nz * 162);
  tDt.reserve((size_t)nc * nz * 162);
  X.m2diag.assign(X.nu, 0.0);
  for (int c = 0; c < nc; ++c) {
    double J0[3], J1[3];
    for (int x = 0; x < 3; ++x) {
      J0[x] = vert(c, 1, x) - vert(c, 0, x);
      J1[x] = vert(c, 2, x) - vert(c, 0, x);
    }
    const double g00 = J0[0] * J0[0] + J0[1] * J0[1] + J0[2] * J0[2];
    const double g01 = J0[0] * J1[0] + J0[1] * J1[1] + J0[2] * J1[2];
    const double g11 = J1[0] * J1[0] + J1[1] * J1[1] + J1[2] * J1[2];
    const double det = std::sqrt(g00 * g11 - g01 * g01);
    const double area1 = 0.5 * det;
    double mass[9][9];
    for (int p = 0; p < 9; ++p)
      for (int q = 0; q < 9; ++q)
        mass[p][q] = (g00 * R.M[p][q][0] + g01 * (R.M[p][q][1] + R.M[p][q][2]) + g11 * R.M[p][q][3]) / det;
    for (int l = 0; l < nz; ++l) {
      const double rho = ph.R + (l + 0.5) * dz;
      const double At = area1 * rho * rho;
      int64_t h[18];
      double hs[18];
      for (int p = 0; p < 9; ++p)
        for (int b = 0; b < 2; ++b) {
          const int64_t base = gbase[(size_t)c * 9 + p];
          h[2 * p + b] = base >= 0 ? base + (int64_t)l * 4 + b : X.nue + (((int64_t)c * nz + l) * 3 + (p - 6)) * 2 + b;
          hs[2 * p + b] = gsign[(size_t)c * 9 + p];
        }
      int64_t v[9];   // (i, kz): vertical unknowns of the cell, -1 on the top and bottom boundary
      for (int i = 0; i < 3; ++i)
        for (int kz = 0; kz < 3; ++kz) {
          const int node = 2 * l + kz;
          v[3 * i + kz] = (node == 0 || node == 2 * nz) ? -1 : X.nue + X.nui + ((int64_t)c * 3 + i) * nzn + node - 1;
        }
      int64_t pr[6];
      for (int u = 0; u < 6; ++u) pr[u] = X.nu + ((int64_t)c * nz + l) * 6 + u;
      // M2^h
      for (int r1 = 0; r1 < 18; ++r1)
        for (int r2 = 0; r2 < 18; ++r2) {
          const double val = hs[r1] * hs[r2] * mass[r1 / 2][r2 / 2] * MZ1[r1 % 2][r2 % 2] / dz;
          tA.push_back({(int32_t)h[r1], (int32_t)h[r2], val});
          if (r1 == r2) X.m2diag[h[r1]] += val;
        }
      // (1 + w_N^2) M2^z
      for (int r1 = 0; r1 < 9; ++r1) {
        if (v[r1] < 0) continue;
        for (int r2 = 0; r2 < 9; ++r2) {
          if (v[r2] < 0) continue;
          const double val = vz * PM(r1 / 3, r2 / 3) / (4.0 * At) * dz * P2[r1 % 3][r2 % 3];
          tA.push_back({(int32_t)v[r1], (int32_t)v[r2], val});
          if (r1 == r2) X.m2diag[v[r1]] += val;
        }
      }
      // divergence pairings: A(p, u) = a c^2 D, A(u, p) = -a D^T
      for (int u = 0; u < 6; ++u) {
        const int j = u / 2, m = u % 2;
        for (int r = 0; r < 18; ++r) {
          const double d = hs[r] * R.div[j][r / 2] * MZ1[m][r % 2];
          tA.push_back({(int32_t)pr[u], (int32_t)h[r], ac2 * d});
          tA.push_back({(int32_t)h[r], (int32_t)pr[u], -a * d});
          tD.push_back({(int32_t)(pr[u] - X.nu), (int32_t)h[r], d});
          tDt.push_back({(int32_t)h[r], (int32_t)(pr[u] - X.nu), d});
        }
        for (int r = 0; r < 9; ++r) {
          if (v[r] < 0) continue;
          const double d = PM(j, r / 3) / 2.0 * G[m][r % 3];
          tA.push_back({(int32_t)pr[u], (int32_t)v[r], ac2 * d});
          tA.push_back({(int32_t)v[r], (int32_t)pr[u], -a * d});
          tD.push_back({(int32_t)(pr[u] - X.nu), (int32_t)v[r], d});
          tDt.push_back({(int32_t)v[r], (int32_t)(pr[u] - X.nu), d});
        }
        // M3
        for (int u2 = 0; u2 < 6; ++u2)
          tA.push_back({(int32_t)pr[u], (int32_t)pr[u2], At * dz * PM(j, u2 / 2) * MZ1[m][u2 % 2]});
      }
    }
  }
  to_csr(tA, X.n, X.n, X.A);
  to_csr(tD, X.np, X.nu, X.D);
  to_csr(tDt, X.nu, X.np, X.Dt);
  return X;
}

// Repack the per-cell blocks into the NLO tile layout (NloSys).
void nlo_pack_host(const NloHost& H, const std::vector<double>& Lf, const std::vector<double>& Dinv,
                   const std::vector<int32_t>& nbr, std::vector<double>* Ad, std::vector<double>* Cs,
                   std::vector<double>* Cu, std::vector<double>* Lft, std::vector<double>* Dit,
                   std::vector<double>* Lb, std::vector<double>* Nb, std::vector<int>* nb) {
  const int nc = H.nc, nz = H.nz;
  if (nc % NLO_TILE) throw std::runtime_error("column count is not a multiple of 5");
  const int nt = nc / NLO_TILE;
  const size_t cells = (size_t)nt * nz * 6 * 32;
  for (auto* v : {Ad, Cs, Cu, Lft, Dit, Lb}) v->assign(cells, 0.0);
  Nb->assign((size_t)nt * 3 * 3 * 32, 0.0);
  nb->assign((size_t)nt * 3 * 32, 0);
  for (int c = 0; c < nc; ++c) {
    const int t = c / NLO_TILE, c5 = c % NLO_TILE;
    for (int l = 0; l < nz; ++l) {
      const size_t o = ((size_t)c * nz + l) * 36;
      const size_t on = ((size_t)c * nz + l + 1) * 36;   // the cell above (l < nz - 1)
      for (int u = 0; u < 6; ++u)
        for (int e = 0; e < 6; ++e) {
          const size_t idx = (((size_t)t * nz + l) * 6 + e) * 32 + 6 * c5 + u;
          (*Ad)[idx] = H.diag[o + 6 * u + e];
          (*Cs)[idx] = H.sub[o + 6 * u + e];
          (*Lft)[idx] = Lf[o + 6 * u + e];
          (*Dit)[idx] = Dinv[o + 6 * u + e];
          if (l < nz - 1) {
            (*Cu)[idx] = H.sub[on + 6 * e + u];
            (*Lb)[idx] = Lf[on + 6 * e + u];
          }
        }
    }
    for (int k = 0; k < 3; ++k) {
      const int n = nbr[3 * c + k];
      for (int u = 0; u < 6; ++u) {
        (*nb)[((size_t)t * 3 + k) * 32 + 6 * c5 + u] = (n / NLO_TILE) * nz * 32 + 6 * (n % NLO_TILE);
        for (int jj = 0; jj < 3; ++jj)
          (*Nb)[(((size_t)t * 3 + k) * 3 + jj) * 32 + 6 * c5 + u] = H.nbr3[((size_t)c * 3 + k) * 9 + 3 * (u / 2) + jj];
      }
    }
  }
}

}  // namespace hmg
