"""Pins of the oracle's lumped Helmholtz operator (Sec. 4.2, Eq. Preconditioner,
Eq. HHgeneralbanded) and its tridiagonal column solver (Sec. 4.3.1)."""
import numpy as np
import pytest

from oracle import helmholtz, mesh

RNG = np.random.default_rng(1234)

# Degree-2-exact triangle rule (edge midpoints, weight |T|/3) and 3-point
# Gauss-Legendre on [0, 1]: independent of the closed forms they check.
GL_X = np.array([0.5 - 0.5 * np.sqrt(3 / 5), 0.5, 0.5 + 0.5 * np.sqrt(3 / 5)])
GL_W = np.array([5 / 18, 8 / 18, 5 / 18])


def tri_quad(P, fn):
    A = 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
    mids = [(P[0] + P[1]) / 2, (P[1] + P[2]) / 2, (P[2] + P[0]) / 2]
    return A / 3 * sum(fn(m) for m in mids), A


def rt0(P, k):
    """Unit-flux RT0 function of the edge opposite vertex k, from its defining
    properties: w(x) = alpha (x - P_k), alpha fixed by unit flux."""
    A = 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
    return lambda x: (x - P[k]) / (2 * A)


def edge_flux(P, k, w):
    """Flux of w out of the triangle through the edge opposite vertex k."""
    a, b = P[(k + 1) % 3], P[(k + 2) % 3]
    nrm = np.cross(P[1] - P[0], P[2] - P[0])
    t = b - a
    n = np.cross(t, nrm)
    n /= np.linalg.norm(n)
    if np.dot(n, a - P[k]) < 0:
        n = -n
    L = np.linalg.norm(t)
    return sum(wq * np.dot(w(a + xq * t), n) * L for xq, wq in zip(GL_X, GL_W))


def test_shape_factor_is_the_rt0_mass_by_quadrature():
    for _ in range(20):
        P = RNG.standard_normal((3, 3))
        v = P.copy()
        sig = mesh.shape_factor(v, np.array([[0, 1, 2]]))[0]
        for k in range(3):
            w = rt0(P, k)
            assert edge_flux(P, k, w) == pytest.approx(1.0, rel=1e-12)
            assert abs(edge_flux(P, (k + 1) % 3, w)) < 1e-12
            q, _ = tri_quad(P, lambda x: np.dot(w(x), w(x)))
            assert sig[k] == pytest.approx(q, rel=1e-12)


def test_shape_factor_equilateral_closed_form():
    P = np.array([[0, 0, 0], [1, 0, 0], [0.5, np.sqrt(3) / 2, 0]], dtype=float)
    sig = mesh.shape_factor(P, np.array([[0, 1, 2]]))[0]
    assert np.allclose(sig, 2.5 / (6 * np.sqrt(3)), rtol=1e-14)


def _prism_masses_by_quadrature(m, prm, theta):
    """Lumped masses of every face by quadrature over the straight prisms."""
    nz, dz, rho = prm.nlayers, prm.dz, prm.rho()
    hor, ver = {}, {}
    for t in range(m.ncols):
        for l in range(nz):
            P = m.verts[m.faces[t]] * rho[l]
            for k in range(3):
                w = rt0(P, k)
                q, _ = tri_quad(P, lambda x: np.dot(w(x), w(x)))
                # 3-D function w / dz on a prism of height dz: integral q / dz
                tn = m.nbr[t, k]
                key = (min(t, tn), max(t, tn), l)
                hor[key] = hor.get(key, 0.0) + q / dz
            if l < nz - 1:
                for ll in (l, l + 1):
                    A = 0.5 * np.linalg.norm(np.cross(*(m.verts[m.faces[t]][1:] - m.verts[m.faces[t]][0]))) * rho[ll] ** 2
                    phi = (lambda s: s) if ll == l else (lambda s: 1 - s)
                    # w = z^ phi / A: integral of |w|^2 over the prism, over theta
                    qz = A * dz * sum(wq * (phi(xq) / A) ** 2 for xq, wq in zip(GL_X, GL_W))
                    ver[(t, l)] = ver.get((t, l), 0.0) + qz / theta[t * nz + ll]
    return hor, ver


@pytest.mark.parametrize("N", [0.01, 0.0])
def test_energy_identity_face_by_face(N):
    """x^T H^ x = sum_K |K| x_K^2 + sum_f g_f (x_K - x_K')^2 with g_f = w_c^2 / M_ff
    (horizontal) and w_c^2 / ((1 + w_N^2) M_ff) (vertical), masses by quadrature."""
    m = mesh.hierarchy(1, 1)[0]
    prm = helmholtz.Params(refinement=1, nlayers=4, N=N)
    theta = np.exp(0.3 * RNG.standard_normal(m.ncols * 4))
    op = helmholtz.assemble(m, prm, theta)
    hor, ver = _prism_masses_by_quadrature(m, prm, theta)
    nz = prm.nlayers
    wc2, wn2 = prm.omega_c ** 2, prm.omega_N ** 2
    for _ in range(3):
        x = RNG.standard_normal(op.ncells)
        e = 0.0
        for t in range(m.ncols):
            for l in range(nz):
                V = m.area1[t] * prm.rho()[l] ** 2 * prm.dz
                e += V * x[t * nz + l] ** 2
        for (t, tn, l), M in hor.items():
            e += wc2 / M * (x[t * nz + l] - x[tn * nz + l]) ** 2
        for (t, l), M in ver.items():
            e += wc2 / ((1 + wn2) * M) * (x[t * nz + l] - x[t * nz + l + 1]) ** 2
        assert x @ (op.H @ x) == pytest.approx(e, rel=1e-12)


@pytest.mark.parametrize("r,nz", [(1, 4), (3, 16)])
def test_symmetry_rowsum_sign_pattern(r, nz):
    m = mesh.hierarchy(r, 1)[0]
    prm = helmholtz.Params(refinement=r, nlayers=nz)
    op = helmholtz.assemble(m, prm)
    H = op.H
    x, y = RNG.standard_normal((2, op.ncells))
    assert x @ (H @ y) == pytest.approx(y @ (H @ x), rel=1e-13)
    # H^ 1 = M3 1: the +-1 divergence couplings have zero row sum
    scale = H.diagonal()
    assert np.max(np.abs(H @ np.ones(op.ncells) - op.M3) / scale) < 1e-14
    coo = H.tocoo()
    off = coo.row != coo.col
    assert np.all(coo.data[off] < 0) and np.all(H.diagonal() > 0)
    # at most 3 horizontal + 2 vertical neighbours per cell
    assert np.max(np.diff(H.indptr)) == 6
    # H^_z is column block-diagonal; H^ - H^_z couples different columns only
    hz = op.Hz.tocoo()
    assert np.all(hz.row // nz == hz.col // nz)
    d = (H - op.Hz).tocoo()
    same = d.row // nz == d.col // nz
    # within a column the two agree up to the rounding of the diagonal sums
    assert np.all(np.abs(d.data[same]) <= 1e-14 * scale[d.row[same]])
    assert np.count_nonzero(d.data[~same]) == np.count_nonzero(H.tocoo().data[
        H.tocoo().row // nz != H.tocoo().col // nz])
    # H^_z is tridiagonal in each column and strictly diagonally dominant
    sub = op.Hz_sub
    sup = np.zeros_like(sub)
    sup[:, :-1] = sub[:, 1:]
    assert np.all(op.Hz_diag > np.abs(sub) + np.abs(sup))


def test_positive_definite_dense():
    m = mesh.hierarchy(0, 1)[0]
    prm = helmholtz.Params(refinement=0, nlayers=4)
    H = helmholtz.assemble(m, prm).H.toarray()
    np.linalg.cholesky(H)
    assert np.linalg.eigvalsh(H).min() > 0


def test_theta_special_cases():
    m = mesh.hierarchy(1, 1)[0]
    prm = helmholtz.Params(refinement=1, nlayers=5)
    n = m.ncols * 5
    H1 = helmholtz.assemble(m, prm).H
    Ht1 = helmholtz.assemble(m, prm, np.ones(n)).H
    assert abs(H1 - Ht1).max() == 0.0
    # theta = 2 halves every vertical lumped mass: the vertical term doubles
    H2 = helmholtz.assemble(m, prm, 2 * np.ones(n)).H
    prm0 = helmholtz.Params(refinement=1, nlayers=5, c=300.0)
    op = helmholtz.assemble(m, prm0)
    vert = (prm.omega_c ** 2 / (1 + prm.omega_N ** 2)) * (op.Dz @ np.diag(1 / op.mz) @ op.Dz.T)
    assert np.allclose((H2 - H1).toarray(), vert, rtol=1e-12, atol=1e-12 * abs(H1).max())


def test_buoyancy_factor():
    """N = 0 removes the 1/(1 + w_N^2) weakening of the vertical couplings."""
    m = mesh.hierarchy(1, 1)[0]
    p1 = helmholtz.Params(refinement=1, nlayers=4)
    p0 = helmholtz.Params(refinement=1, nlayers=4, N=0.0)
    o1, o0 = helmholtz.assemble(m, p1), helmholtz.assemble(m, p0)
    # vertical off-diagonals scale exactly by 1 + w_N^2
    nz = 4
    i = np.arange(m.ncols) * nz + 1
    ratio = o0.H[i, i - 1].A1 / o1.H[i, i - 1].A1
    assert np.allclose(ratio, 1 + p1.omega_N ** 2, rtol=1e-13)
    # horizontal off-diagonals are unchanged
    t, k, tn, kn = helmholtz.horizontal_faces(m)[0]
    assert o0.H[t * nz, tn * nz] == pytest.approx(o1.H[t * nz, tn * nz], rel=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 16, 64, 128])
def test_thomas_matches_dense_solve(n):
    batch = 7
    sub = RNG.standard_normal((batch, n))
    sup = RNG.standard_normal((batch, n))
    diag = 2.5 + np.abs(sub) + np.abs(sup) + RNG.random((batch, n))
    rhs = RNG.standard_normal((batch, n))
    x = helmholtz.thomas(sub, diag, sup, rhs)
    for b in range(batch):
        A = np.diag(diag[b])
        if n > 1:
            A += np.diag(sub[b, 1:], -1) + np.diag(sup[b, :-1], 1)
        assert np.allclose(x[b], np.linalg.solve(A, rhs[b]), rtol=1e-13, atol=1e-13)


def test_column_solve_inverts_Hz():
    m = mesh.hierarchy(2, 1)[0]
    prm = helmholtz.Params(refinement=2, nlayers=16)
    op = helmholtz.assemble(m, prm)
    r = RNG.standard_normal(op.ncells)
    x = helmholtz.solve_Hz(op, r)
    assert np.linalg.norm(op.Hz @ x - r) / np.linalg.norm(r) < 1e-12
