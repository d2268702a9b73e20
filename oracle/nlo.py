"""Next-to-lowest-order (NLO) pressure-Helmholtz operator and its V-cycle (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Table "FiniteElements" gives the NLO spaces: pressure W3 = DG1(T) x DG1(z)
(6 unknowns per prism), horizontal velocity W2^h = BDFM1(T) x DG1(z) and
vertical velocity W2^z = DG1(T) x P2(z) with u.n = 0 at the top and bottom
(Eq. BoundaryCondition); Table "GridSetup" confirms 24 unknowns per cell
(6 + 12 + 6).  The lumped operator is Eq. (Preconditioner) with the lumped
inverse masses of Eq. (LumpedMass); its column part is Eq. (HHgeneralbanded),
block tridiagonal in each column (6 x 6 blocks, Sec. 4.3 and Sec. 6
"Performance model": m = 6 n_z rows per column).  Sec. 4.2.1 makes the first
coarsening step a p-coarsening DG1 -> DG0 on the same mesh with restriction
and prolongation from the natural embedding DG0 in DG1; the levels below are
the lowest-order hierarchy (helmholtz.py, multigrid.py).

Readings (the paper leaves them open; the CUDA library follows the same
written definitions with its own code):

* BDFM1(T) = {v in P2(T)^2 : v.n restricted to each edge is in P1}, which is
  P1(T)^2 plus the three edge bubbles lam_i lam_j t_k (t_k = P_j - P_i, the
  tangent of edge k from vertex i = k+1 to vertex j = k+2, indices mod 3);
* its degrees of freedom: for each edge k the length-scaled outward normal
  component |e_k| v(x).n_k at the points x = P_i + s (P_j - P_i), s = 1/3
  and 2/3 (q = 0, 1), and for each edge the moment int_T v . W_k against
  the Whitney function W_k = lam_i grad lam_j - lam_j grad lam_i.  Both
  families are invariant under the contravariant Piola map, so the basis
  does not depend on which vertex is taken first;
* DG1(T) is nodal at the three vertices (the barycentric lam_j), DG1(z)
  nodal at the bottom (m = 0) and top (m = 1) of the layer, P2(z) nodal at
  the bottom, middle and top;
* geometry as in helmholtz.py: the straight prism over the flat triangle T
  scaled to the mid-layer radius rho_l; the horizontal velocity basis is
  v_a(x) psi_b(z) / dz with v_a the BDFM1 basis on T (so the horizontal
  integrals are scale invariant), the vertical one z^ lam_i(x) zeta_n(z) /
  (2 |T_l|) (the same flux through an interface from both layers);
* unknown order: cell (col, layer), then vertex j of the face, then m:
  index ((col * nz + layer) * 3 + j) * 2 + m;
* the coarse level below the NLO level is the lowest-order operator
  rediscretised on the same mesh, P copies a cell's value to its six
  unknowns and the restriction is P^T.
"""
from dataclasses import dataclass
from math import factorial

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import helmholtz, multigrid

S_POINTS = (1.0 / 3.0, 2.0 / 3.0)
# int_0^1 of products of the DG1 (z) nodal functions 1 - s, s
MZ1 = np.array([[1.0, 0.5], [0.5, 1.0]]) / 3.0
# int_0^1 of products of the P2 (z) nodal functions at s = 0, 1/2, 1
MP2 = np.array([[4.0, 2.0, -1.0], [2.0, 16.0, 2.0], [-1.0, 2.0, 4.0]]) / 30.0


# ----------------------------------------------------------------- polynomials
# Polynomials on a triangle in barycentric monomials lam0^a lam1^b lam2^c:
# scalar {(a, b, c): float}, vector {(a, b, c): ndarray(3)}.

def _unit(i):
    e = [0, 0, 0]
    e[i] = 1
    return tuple(e)


def _add(a, b):
    return tuple(x + y for x, y in zip(a, b))


def integrate(p, area):
    """int_T lam^alpha dA = 2 |T| a! b! c! / (a + b + c + 2)!."""
    return sum(c * 2.0 * area * factorial(a0) * factorial(a1) * factorial(a2) / factorial(a0 + a1 + a2 + 2)
               for (a0, a1, a2), c in p.items())


def vdot(u, v):
    out = {}
    for a, ua in u.items():
        for b, vb in v.items():
            k = _add(a, b)
            out[k] = out.get(k, 0.0) + float(np.dot(ua, vb))
    return out


def divergence(v, grads):
    """div sum_alpha c_alpha lam^alpha = sum_alpha sum_i alpha_i lam^(alpha - e_i) c_alpha . grad lam_i."""
    out = {}
    for a, ca in v.items():
        for i in range(3):
            if a[i] == 0:
                continue
            k = list(a)
            k[i] -= 1
            k = tuple(k)
            out[k] = out.get(k, 0.0) + a[i] * float(np.dot(ca, grads[i]))
    return out


def evaluate(v, lam):
    return sum(c * lam[0] ** a[0] * lam[1] ** a[1] * lam[2] ** a[2] for a, c in v.items())


# ----------------------------------------------------------------- BDFM1 on one triangle

@dataclass
class TriangleBDFM:
    """The BDFM1 basis of one flat triangle and its integrals.  Local unknowns
    a = 2 k + q (edge k, point q) for a < 6 and a = 6 + k (Whitney moment of
    edge k).  mass[a, a'] = int_T v_a . v_a'; div[j, a] = int_T lam_j div v_a."""
    area: float
    basis: list
    mass: np.ndarray
    div: np.ndarray
    normals: np.ndarray      # (3, 3) outward unit normals of the edges
    grads: np.ndarray        # (3, 3) grad lam_i


def triangle_bdfm(P):
    """BDFM1 on the flat triangle with vertices P[0], P[1], P[2] (3-D points).

    The nine spanning functions lam_m e (e an in-plane unit vector) and
    lam_i lam_j t_k are single monomials times a vector, so every functional
    and integral of them is one integration formula; the basis is the
    spanning set times the inverse of the matrix of the degrees of freedom."""
    P = np.asarray(P, dtype=np.float64)
    N = np.cross(P[1] - P[0], P[2] - P[0])
    nn = float(np.dot(N, N))
    area = 0.5 * np.sqrt(nn)
    grads = np.array([np.cross(N, P[(i + 2) % 3] - P[(i + 1) % 3]) / nn for i in range(3)])
    e1 = (P[1] - P[0]) / np.linalg.norm(P[1] - P[0])
    e2 = np.cross(N / np.sqrt(nn), e1)
    span = []                                   # (exponent triple, vector)
    for m in range(3):
        for ax in (e1, e2):
            span.append((_unit(m), ax))
    for k in range(3):
        i, j = (k + 1) % 3, (k + 2) % 3
        span.append((_add(_unit(i), _unit(j)), P[j] - P[i]))
    normals = np.empty((3, 3))
    for k in range(3):
        i, j = (k + 1) % 3, (k + 2) % 3
        n = np.cross(P[j] - P[i], N)
        n /= np.linalg.norm(n)
        if np.dot(n, P[i] - P[k]) < 0:
            n = -n
        normals[k] = n
    I = lambda alpha: integrate({alpha: 1.0}, area)

    Phi = np.empty((9, 9))                      # Phi[dof, span function]
    for f, (al, c) in enumerate(span):
        for k in range(3):
            i, j = (k + 1) % 3, (k + 2) % 3
            length = np.linalg.norm(P[j] - P[i])
            for q, s in enumerate(S_POINTS):
                lam = np.zeros(3)
                lam[i], lam[j] = 1.0 - s, s
                Phi[2 * k + q, f] = length * evaluate({al: 1.0}, lam) * float(np.dot(c, normals[k]))
            # int lam^al c . (lam_i grad lam_j - lam_j grad lam_i)
            Phi[6 + k, f] = (float(np.dot(c, grads[j])) * I(_add(al, _unit(i)))
                             - float(np.dot(c, grads[i])) * I(_add(al, _unit(j))))
    C = np.linalg.inv(Phi)                      # basis a = sum_f span_f C[f, a]
    S_mass = np.array([[float(np.dot(cf, cg)) * I(_add(af, ag)) for (ag, cg) in span] for (af, cf) in span])
    S_div = np.zeros((3, 9))
    for f, (al, c) in enumerate(span):
        for i in range(3):
            if al[i] == 0:
                continue
            low = list(al)
            low[i] -= 1
            for j in range(3):
                S_div[j, f] += al[i] * float(np.dot(c, grads[i])) * I(_add(tuple(low), _unit(j)))
    basis = []
    for a in range(9):
        v = {}
        for f, (al, c) in enumerate(span):
            v[al] = v.get(al, 0.0) + C[f, a] * c
        basis.append(v)
    return TriangleBDFM(area, basis, C.T @ S_mass @ C, S_div @ C, normals, grads)


def _lam_times(j, s):
    out = {}
    for a, c in s.items():
        k = _add(a, _unit(j))
        out[k] = out.get(k, 0.0) + c
    return out


# ----------------------------------------------------------------- the NLO operator

def pdof(col, layer, j, m, nz):
    return ((col * nz + layer) * 3 + j) * 2 + m


@dataclass
class NLOOperator:
    ncols: int
    nlayers: int
    M3: sp.csr_matrix
    Dh: sp.csr_matrix
    mh: np.ndarray
    Dz: sp.csr_matrix
    mz: np.ndarray
    H: sp.csr_matrix
    Hz: sp.csr_matrix
    Hz_lu: object

    @property
    def n(self):
        return 6 * self.ncols * self.nlayers


def horizontal_dofs(mesh, nz):
    """Global horizontal velocity unknowns as a list of (column, local BDFM1
    unknown a, base, sign): the unknown (layer l, DG1 node b in z) is global
    number base + 2 l + b and equals sign times the column's local function.
    Edge unknowns (edge E, point q) come first, E in the order of
    helmholtz.horizontal_faces, with the outward normal of the edge's first
    (lower-numbered) column; the point q of the second column is the one at
    the same position on the shared edge.  Interior unknowns (column, k)
    follow.  Returns (owner list, number of edge unknowns, total)."""
    edges = helmholtz.horizontal_faces(mesh)
    ne = edges.shape[0]
    nhe = ne * 2 * nz * 2
    owner = []
    for E, (t, k, tn, kn) in enumerate(edges):
        ft, fn = mesh.faces[t], mesh.faces[tn]
        same = ft[(k + 1) % 3] == fn[(kn + 1) % 3] and ft[(k + 2) % 3] == fn[(kn + 2) % 3]
        rev = ft[(k + 1) % 3] == fn[(kn + 2) % 3] and ft[(k + 2) % 3] == fn[(kn + 1) % 3]
        assert same != rev
        for q in range(2):
            qn = q if same else 1 - q
            owner.append((t, 2 * k + q, (E * 2 + q) * nz * 2, 1.0))
            owner.append((tn, 2 * kn + qn, (E * 2 + q) * nz * 2, -1.0))
    for c in range(mesh.ncols):
        for k in range(3):
            owner.append((c, 6 + k, nhe + (c * 3 + k) * nz * 2, 1.0))
    return owner, nhe, nhe + mesh.ncols * 3 * nz * 2


def assemble_nlo(mesh, prm):
    """H^ of Eq. (Preconditioner) for the NLO spaces on one mesh (theta = 1)."""
    nc, nz = mesh.ncols, prm.nlayers
    dz = prm.dz
    rho = prm.rho()
    n = 6 * nc * nz
    tri = [triangle_bdfm(mesh.verts[mesh.faces[c]]) for c in range(nc)]

    PM = np.array([[2.0, 1.0, 1.0], [1.0, 2.0, 1.0], [1.0, 1.0, 2.0]]) / 12.0   # int_T lam lam' / |T|
    At = mesh.area1[:, None] * rho[None, :] ** 2                                 # |T_l|, (nc, nz)
    J, Mi = np.meshgrid(np.arange(3), np.arange(2), indexing="ij")
    J, Mi = J.reshape(-1), Mi.reshape(-1)                                        # local unknown u = 2 j + m
    cells = np.arange(nc * nz)

    # M3 = int_K phi phi' on the prism over T scaled to rho_l
    loc = PM[J[:, None], J[None, :]] * dz * MZ1[Mi[:, None], Mi[None, :]]      # (6, 6) per unit |T_l|
    rows = (6 * cells[:, None, None] + np.arange(6)[None, :, None]) + 0 * np.arange(6)[None, None, :]
    cols = (6 * cells[:, None, None] + np.arange(6)[None, None, :]) + 0 * np.arange(6)[None, :, None]
    vals = At.reshape(-1)[:, None, None] * loc[None]
    M3 = sp.csr_matrix((vals.reshape(-1), (rows.reshape(-1), cols.reshape(-1))), shape=(n, n))

    # horizontal velocity: global edge dofs (edge E, point q, layer, b) with the
    # normal of the lower-numbered face, then interior dofs (col, k, layer, b)
    owner, nhe, nhf = horizontal_dofs(mesh, nz)
    lay = np.arange(nz)
    rows, cols, vals = [], [], []
    mh = np.zeros(nhf)
    for (c, a, base, sgn) in owner:
        f = base + 2 * lay[:, None] + np.arange(2)[None, :]                        # (nz, b)
        np.add.at(mh, f, tri[c].mass[a, a] * MZ1[np.arange(2), np.arange(2)][None, :] / dz)
        r = 6 * (c * nz + lay)[:, None, None] + np.arange(6)[None, :, None] + 0 * f[:, None, :]
        v = sgn * tri[c].div[J, a][:, None] * MZ1[Mi[:, None], np.arange(2)[None, :]]     # (6, b)
        rows.append(r.reshape(-1))
        cols.append(np.broadcast_to(f[:, None, :], r.shape).reshape(-1))
        vals.append(np.broadcast_to(v[None], r.shape).reshape(-1))
    Dh = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, nhf))

    # vertical velocity: (col, vertex i, node 1 .. 2 nz - 1) of P2 in z; cell
    # `lay` holds nodes 2 lay + kz, kz = 0, 1, 2 (bottom, middle, top)
    nzn = 2 * nz - 1
    nvf = nc * 3 * nzn
    # int_0^1 eta_m d/ds zeta_kz ds for DG1 nodal eta and P2 nodal zeta
    s, w = np.polynomial.legendre.leggauss(4)
    s, w = 0.5 * (s + 1.0), 0.5 * w
    eta = np.array([1.0 - s, s])
    dzeta = np.array([4.0 * s - 3.0, 4.0 - 8.0 * s, 4.0 * s - 1.0])
    G = np.einsum("mq,kq,q->mk", eta, dzeta, w)
    rows, cols, vals = [], [], []
    mz = np.zeros(nvf)
    cc, ll = np.meshgrid(np.arange(nc), np.arange(nz), indexing="ij")
    cc, ll = cc.reshape(-1), ll.reshape(-1)
    for kz in range(3):
        node = 2 * ll + kz
        keep = (node > 0) & (node < 2 * nz)
        c_, l_, node = cc[keep], ll[keep], node[keep]
        A_ = At[c_, l_]
        for i in range(3):
            f = (c_ * 3 + i) * nzn + node - 1
            np.add.at(mz, f, PM[i, i] / (4.0 * A_) * dz * MP2[kz, kz])   # int lam_i^2 / (4 |T|^2) * int zeta^2
            for u in range(6):
                rows.append(6 * (c_ * nz + l_) + u)
                cols.append(f)
                vals.append(np.full(f.size, PM[J[u], i] / 2.0 * G[Mi[u], kz]))   # int lam_j lam_i / (2|T|) * int eta zeta'
    Dz = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, nvf))

    wc2 = prm.omega_c ** 2
    wn2 = prm.omega_N ** 2
    horiz = Dh @ sp.diags(1.0 / mh) @ Dh.T
    vert = Dz @ sp.diags(1.0 / mz) @ Dz.T
    H = (M3 + wc2 * (horiz + vert / (1.0 + wn2))).tocsr()
    hcoo = H.tocoo()
    col_of = lambda idx: idx // (6 * nz)
    same = col_of(hcoo.row) == col_of(hcoo.col)
    Hz = sp.csr_matrix((hcoo.data[same], (hcoo.row[same], hcoo.col[same])), shape=(n, n))
    return NLOOperator(nc, nz, M3, Dh, mh, Dz, mz, H, Hz, spla.splu(Hz.tocsc()))


def apply_nlo(nop, x):
    return nop.H @ x


def smooth(nop, u, b, omega):
    """u + omega H^_z^-1 (b - H^ u): the vertical line relaxation of
    Eq. (BlockJacobi); H^_z^-1 is a direct solve of the column-block system."""
    return u + omega * nop.Hz_lu.solve(b - nop.H @ u)


def prolongation(ncols, nlayers):
    """P: DG0 (cell c * nz + l) -> DG1 (its six unknowns), the natural embedding."""
    n = 6 * ncols * nlayers
    rows = np.arange(n)
    return sp.csr_matrix((np.ones(n), (rows, rows // 6)), shape=(n, ncols * nlayers))


def vcycle(nop, lo_ops, b, omega=0.8, nu_pre=2, nu_post=2, n_coarse=2):
    """One V-cycle from zero: NLO smoothing, p-coarsening to the lowest-order
    operator on the same mesh (lo_ops[0]) and the lowest-order V-cycle below."""
    P = prolongation(nop.ncols, nop.nlayers)
    u = np.zeros_like(b)
    for _ in range(nu_pre):
        u = smooth(nop, u, b, omega)
    bc = P.T @ (b - nop.H @ u)
    ec = multigrid.vcycle(lo_ops, bc, omega, nu_pre, nu_post, n_coarse)
    u = u + P @ ec
    for _ in range(nu_post):
        u = smooth(nop, u, b, omega)
    return u
