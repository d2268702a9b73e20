"""Pins of the oracle's next-to-lowest-order operator (oracle/nlo.py): the
BDFM1 element, the assembled H^ of Eq. (Preconditioner) for the NLO spaces
of Table "FiniteElements", the p-coarsening of Sec. 4.2.1 and the V-cycle."""
import os

import numpy as np
import pytest

from oracle import helmholtz, krylov, mesh, nlo

RNG = np.random.default_rng(77)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "grid_setup.txt")


def _triangle():
    return RNG.standard_normal((3, 3))


def _in_plane_eval(T, P, coef, x):
    """sum_a coef_a v_a at the point x of the triangle."""
    lam = _bary(P, x)
    return sum(coef[a] * nlo.evaluate(T.basis[a], lam) for a in range(9))


def _bary(P, x):
    M = np.stack([P[1] - P[0], P[2] - P[0]], axis=1)
    st, *_ = np.linalg.lstsq(M, x - P[0], rcond=None)
    return np.array([1.0 - st[0] - st[1], st[0], st[1]])


def _quad_points(P, n=6):
    """Collapsed Gauss-Legendre rule on the triangle: points and weights,
    exact for polynomials of degree 2n - 2 (independent of the monomial
    integration formula of the oracle)."""
    g, w = np.polynomial.legendre.leggauss(n)
    g, w = 0.5 * (g + 1.0), 0.5 * w
    area2 = np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
    pts, wts = [], []
    for u, wu in zip(g, w):
        for v, wv in zip(g, w):
            x = P[0] + u * (P[1] - P[0]) + v * (1.0 - u) * (P[2] - P[0])
            pts.append(x)
            wts.append(wu * wv * (1.0 - u) * area2)
    return np.array(pts), np.array(wts)


def _dofs_of(T, P, field):
    """The nine degrees of freedom of a vector field given as a function of x:
    normal components at the edge points, Whitney moments by quadrature."""
    out = np.empty(9)
    pts, wts = _quad_points(P)
    for k in range(3):
        i, j = (k + 1) % 3, (k + 2) % 3
        length = np.linalg.norm(P[j] - P[i])
        for q, s in enumerate((1.0 / 3.0, 2.0 / 3.0)):      # the reading: the points 1/3 and 2/3 of the edge
            out[2 * k + q] = length * np.dot(field(P[i] + s * (P[j] - P[i])), T.normals[k])
        Wk = lambda x: _bary(P, x)[i] * T.grads[j] - _bary(P, x)[j] * T.grads[i]
        out[6 + k] = sum(wq * np.dot(field(x), Wk(x)) for x, wq in zip(pts, wts))
    return out


def test_bdfm_basis_is_dual_to_its_degrees_of_freedom():
    P = _triangle()
    T = nlo.triangle_bdfm(P)
    for a in range(9):
        field = lambda x, a=a: nlo.evaluate(T.basis[a], _bary(P, x))
        assert np.allclose(_dofs_of(T, P, field), np.eye(9)[a], atol=1e-11)


def test_bdfm_normal_traces_are_linear_and_fluxes():
    """v.n on every edge is in P1 (the defining property of BDFM1), so the
    flux of an edge function through its edge is |e| times the mean of a
    linear function that is 1/|e| at s = 1/3 and 0 at s = 2/3: 1/2.  The
    interior functions have no normal trace."""
    P = _triangle()
    T = nlo.triangle_bdfm(P)
    for a in range(9):
        for k in range(3):
            i, j = (k + 1) % 3, (k + 2) % 3
            vals = []
            for s in np.linspace(0.0, 1.0, 5):
                lam = np.zeros(3)
                lam[i], lam[j] = 1.0 - s, s
                vals.append(np.dot(nlo.evaluate(T.basis[a], lam), T.normals[k]))
            vals = np.array(vals)
            lin = np.polyfit(np.linspace(0, 1, 5), vals, 1)
            assert np.allclose(np.polyval(lin, np.linspace(0, 1, 5)), vals, atol=1e-10 * (1 + np.abs(vals).max()))
            if a >= 6:
                assert np.abs(vals).max() < 1e-10
    assert np.allclose(T.div.sum(axis=0), [0.5] * 6 + [0.0] * 3, atol=1e-12)


def test_bdfm_contains_rt0_with_the_lowest_order_shape_factor():
    """The unit-flux RT0 function (x - P_k) / (2|T|) of edge k lies in BDFM1;
    rebuilt from its degrees of freedom it is reproduced pointwise, and its
    energy is the shape factor sigma of the lowest-order operator."""
    P = _triangle()
    T = nlo.triangle_bdfm(P)
    faces = np.array([[0, 1, 2]])
    sigma = mesh.shape_factor(P, faces)[0]
    for k in range(3):
        w = lambda x, k=k: (x - P[k]) / (2.0 * T.area)
        coef = _dofs_of(T, P, w)
        assert np.allclose(coef[[2 * k, 2 * k + 1]], 1.0, atol=1e-12)
        for x in (P.mean(0), 0.2 * P[0] + 0.5 * P[1] + 0.3 * P[2]):
            assert np.allclose(_in_plane_eval(T, P, coef, x), w(x), atol=1e-11)
        assert coef @ T.mass @ coef == pytest.approx(sigma[k], rel=1e-11)


def test_bdfm_contains_p1_fields_and_rotated_gradients():
    """P1(T)^2 lies in the space, and so does the rotated gradient of every
    quadratic and of the cubic bubble lam0 lam1 lam2 (the de Rham sequence
    P2 + B3 -> BDFM1 -> DG1 of the element): each is reproduced from its
    degrees of freedom."""
    P = _triangle()
    T = nlo.triangle_bdfm(P)
    nrm = np.cross(P[1] - P[0], P[2] - P[0])
    nrm /= np.linalg.norm(nrm)
    A = RNG.standard_normal((3, 3))
    A -= np.outer(A @ nrm, nrm)                     # in-plane values
    fields = [lambda x: A[0] + _bary(P, x)[1] * A[1] + _bary(P, x)[2] * A[2]]     # a general P1 field
    G = T.grads

    def rotgrad(coeffs):
        # s = sum over monomials; grad s in terms of grad lam_i, rotated by n x
        def f(x):
            lam = _bary(P, x)
            g = np.zeros(3)
            for (e, c) in coeffs:
                for i in range(3):
                    if e[i]:
                        low = list(e)
                        low[i] -= 1
                        g += c * e[i] * np.prod(lam ** np.array(low)) * G[i]
            return np.cross(nrm, g)
        return f
    fields += [rotgrad([((2, 0, 0), 1.0)]), rotgrad([((1, 1, 0), 1.0)]), rotgrad([((0, 1, 1), 1.0), ((2, 0, 0), -0.5)]),
               rotgrad([((1, 1, 1), 1.0)])]
    for field in fields:
        coef = _dofs_of(T, P, field)
        for x in (P.mean(0), 0.1 * P[0] + 0.6 * P[1] + 0.3 * P[2], 0.7 * P[0] + 0.2 * P[1] + 0.1 * P[2]):
            assert np.allclose(_in_plane_eval(T, P, coef, x), field(x), atol=1e-10)
    # div maps onto DG1 (rank 3): the kernel (rotated gradients) has dimension 6
    assert np.linalg.matrix_rank(T.div, tol=1e-10) == 3


def test_bdfm_integrals_against_quadrature():
    P = _triangle()
    T = nlo.triangle_bdfm(P)
    pts, wts = _quad_points(P)
    h = 1e-5
    e1 = (P[1] - P[0]) / np.linalg.norm(P[1] - P[0])
    nrm = np.cross(P[1] - P[0], P[2] - P[0])
    e2 = np.cross(nrm / np.linalg.norm(nrm), e1)
    for a in range(9):
        v = lambda x, a=a: nlo.evaluate(T.basis[a], _bary(P, x))
        for b in range(9):
            vb = lambda x, b=b: nlo.evaluate(T.basis[b], _bary(P, x))
            q = sum(wq * np.dot(v(x), vb(x)) for x, wq in zip(pts, wts))
            assert T.mass[a, b] == pytest.approx(q, rel=1e-9, abs=1e-12 * np.abs(T.mass).max())
        # divergence by central differences in the plane (v is quadratic: exact up to rounding)
        div = lambda x: (np.dot(v(x + h * e1) - v(x - h * e1), e1) + np.dot(v(x + h * e2) - v(x - h * e2), e2)) / (2 * h)
        for j in range(3):
            q = sum(wq * _bary(P, x)[j] * div(x) for x, wq in zip(pts, wts))
            assert T.div[j, a] == pytest.approx(q, abs=1e-6 * max(1.0, np.abs(T.div).max()))


def test_bdfm_does_not_depend_on_the_vertex_order():
    """Relabelling the vertices permutes the local unknowns (edge k follows
    its opposite vertex; a reversed edge swaps its two points) and leaves the
    element matrices otherwise unchanged; similarity maps leave them
    unchanged (the horizontal integrals are scale invariant)."""
    P = _triangle()
    T = nlo.triangle_bdfm(P)
    perm = [1, 2, 0]                              # cyclic: edge directions kept
    Tc = nlo.triangle_bdfm(P[perm])
    amap = [2 * 1 + 0, 2 * 1 + 1, 2 * 2 + 0, 2 * 2 + 1, 0, 1, 7, 8, 6]
    assert np.allclose(Tc.mass, T.mass[np.ix_(amap, amap)], rtol=1e-11, atol=1e-13)
    assert np.allclose(Tc.div, T.div[np.ix_(perm, amap)], rtol=1e-11, atol=1e-13)
    Tr = nlo.triangle_bdfm(P[[0, 2, 1]])          # reversed orientation
    amap = [1, 0, 5, 4, 3, 2, 6, 8, 7]
    sgn = np.array([1, 1, 1, 1, 1, 1, -1, -1, -1.0])   # Whitney functions change sign with their edge
    Mr = T.mass[np.ix_(amap, amap)] * np.outer(sgn, sgn)
    assert np.allclose(Tr.mass, Mr, rtol=1e-11, atol=1e-13)
    assert np.allclose(Tr.div, T.div[np.ix_([0, 2, 1], amap)] * sgn, rtol=1e-11, atol=1e-13)
    Q, _ = np.linalg.qr(RNG.standard_normal((3, 3)))
    Ts = nlo.triangle_bdfm(3.7 * P @ Q.T + RNG.standard_normal(3))
    assert np.allclose(Ts.mass, T.mass, rtol=1e-10, atol=1e-12)
    assert np.allclose(Ts.div, T.div, rtol=1e-10, atol=1e-13)


@pytest.fixture(scope="module")
def tiny():
    ms = mesh.hierarchy(1, 2)
    prm = helmholtz.Params(refinement=1, nlayers=3)
    return ms, prm, nlo.assemble_nlo(ms[0], prm), helmholtz.assemble_hierarchy(ms, prm)


def test_unknown_counts_match_table_grid_setup():
    """24 unknowns per cell at NLO (Table "GridSetup"), counting one
    boundary node per column of vertical velocity as the lowest-order row
    does; the total at 5,120 x 64 cells rounds to the printed 7.9 million."""
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    row = next(r for r in rows if r[0] == "NLO")
    ncols, nz, per_cell, total = int(row[1]), int(row[3]), float(row[4]), float(row[5])
    ms = mesh.hierarchy(1, 1)
    prm = helmholtz.Params(refinement=1, nlayers=3)
    nop = nlo.assemble_nlo(ms[0], prm)
    nc, nzz = nop.ncols, nop.nlayers
    counted = nop.n + nop.mh.size + nop.mz.size + 3 * nc
    assert counted == per_cell * nc * nzz
    assert round(per_cell * ncols * nz / 1e6, 1) == total


def test_nlo_operator_symmetric_positive_definite(tiny):
    ms, prm, nop, lo = tiny
    H = nop.H.toarray()
    assert np.abs(H - H.T).max() <= 1e-14 * np.abs(H).max()
    ev = np.linalg.eigvalsh(H)
    assert ev.min() > 0


def test_nlo_operator_constant_and_embedding(tiny):
    """D^T 1 = 0 (a closed shell: the divergence of every velocity function
    integrates to zero), so H^ 1 = M3 1 with every unknown carrying |K| / 6;
    the embedding DG0 -> DG1 gives P^T M3 P = the lowest-order M3."""
    ms, prm, nop, lo = tiny
    one = np.ones(nop.n)
    assert np.abs(nop.Dh.T @ one).max() <= 1e-12 * np.abs(nop.Dh).max()
    assert np.abs(nop.Dz.T @ one).max() <= 1e-12 * np.abs(nop.Dz).max()
    vol = np.repeat(lo[0].M3, 6) / 6.0
    assert np.allclose(nop.M3 @ one, vol, rtol=1e-13)
    assert np.allclose(nop.H @ one, vol, rtol=1e-9)
    P = nlo.prolongation(nop.ncols, nop.nlayers)
    PMP = (P.T @ nop.M3 @ P).toarray()
    assert np.allclose(PMP, np.diag(lo[0].M3), rtol=1e-13, atol=1e-3)


def test_nlo_operator_structure(tiny):
    """H^_z is block tridiagonal in each column (6 x 6 blocks); the rest of
    H^ couples only unknowns of the same layer in edge-neighbour columns."""
    ms, prm, nop, lo = tiny
    nz = nop.nlayers
    Hz = nop.Hz.tocoo()
    cz, lz = Hz.row // (6 * nz), (Hz.row // 6) % nz
    cz2, lz2 = Hz.col // (6 * nz), (Hz.col // 6) % nz
    assert np.all(cz == cz2) and np.all(np.abs(lz - lz2) <= 1)
    Hh = (nop.H - nop.Hz).tocoo()
    Hh.eliminate_zeros()
    c1, l1 = Hh.row // (6 * nz), (Hh.row // 6) % nz
    c2, l2 = Hh.col // (6 * nz), (Hh.col // 6) % nz
    assert np.all(l1 == l2)
    nb = ms[0].nbr
    assert all(c2[i] in nb[c1[i]] for i in range(len(c1)))
    # the horizontal coupling does not depend on the layer (uniform dz)
    blocks = nop.H.toarray().reshape(nop.ncols, nz, 6, nop.ncols, nz, 6)
    c, n0 = 0, nb[0, 0]
    for layer in range(1, nz):
        assert np.allclose(blocks[c, layer, :, n0, layer], blocks[c, 0, :, n0, 0], rtol=1e-12)


def test_pressure_mass_by_quadrature(tiny):
    """x^T M3 x = sum over prisms of int p_h^2 for a random DG1 x (prism over
    the flat triangle at the mid-layer radius; Gauss rules in both directions)."""
    ms, prm, nop, lo = tiny
    m = ms[0]
    x = RNG.standard_normal(nop.n)
    rho = prm.rho()
    g, w = np.polynomial.legendre.leggauss(3)
    g, w = 0.5 * (g + 1.0), 0.5 * w
    total = 0.0
    for c in range(m.ncols):
        P1 = m.verts[m.faces[c]]
        pts, wts = _quad_points(P1, 3)
        for layer in range(prm.nlayers):
            xs = x[nlo.pdof(c, layer, 0, 0, prm.nlayers):nlo.pdof(c, layer, 0, 0, prm.nlayers) + 6].reshape(3, 2)
            for p, wp in zip(pts, wts):
                lam = _bary(P1, p)
                for s, ws in zip(g, w):
                    val = lam @ xs @ np.array([1.0 - s, s])
                    total += wp * rho[layer] ** 2 * ws * prm.dz * val * val
    assert x @ (nop.M3 @ x) == pytest.approx(total, rel=1e-12)


def test_nlo_vcycle_symmetric_positive(tiny):
    ms, prm, nop, lo = tiny
    x, y = RNG.standard_normal(nop.n), RNG.standard_normal(nop.n)
    Vx, Vy = nlo.vcycle(nop, lo, x), nlo.vcycle(nop, lo, y)
    assert abs(y @ Vx - x @ Vy) <= 1e-12 * abs(y @ Vx)
    assert x @ Vx > 0


def test_nlo_multigrid_beats_single_level_and_is_grid_robust():
    """Multigrid-preconditioned CG on the NLO operator needs far fewer
    iterations than the block-Jacobi preconditioner alone (Sec. 6, Table
    "SingleNodePerformance": 21 against 81 GMRES iterations at NLO), and the
    count does not grow with the resolution at fixed Courant number."""
    its = []
    for r in (2, 3):
        ms = mesh.hierarchy(r, r)
        prm = helmholtz.Params(refinement=r, nlayers=8)
        nop = nlo.assemble_nlo(ms[0], prm)
        lo = helmholtz.assemble_hierarchy(ms, prm)
        b = RNG.standard_normal(nop.n)
        x, info = krylov.pcg(lambda v: nop.H @ v, lambda v: nlo.vcycle(nop, lo, v), b, rtol=1e-8)
        assert info.converged
        assert np.linalg.norm(nop.H @ x - b) <= 1.01e-8 * np.linalg.norm(b)
        its.append(info.iterations)
    assert its[1] <= its[0] + 2, its
    _, info1 = krylov.pcg(lambda v: nop.H @ v, lambda v: 0.8 * nop.Hz_lu.solve(v), b, rtol=1e-8, max_iter=2000)
    assert info1.iterations > 3 * its[1]


def test_nlo_smoother_exact_for_decoupled_columns(tiny):
    """With the horizontal coupling between columns removed and omega = 1,
    one sweep from zero solves the system (the column solve is exact)."""
    ms, prm, nop, lo = tiny
    import dataclasses
    dec = dataclasses.replace(nop, H=nop.Hz)
    b = RNG.standard_normal(nop.n)
    u = nlo.smooth(dec, np.zeros(nop.n), b, 1.0)
    assert np.linalg.norm(nop.Hz @ u - b) <= 1e-12 * np.linalg.norm(b)


def test_horizontal_unknowns_have_continuous_normal_flux():
    """Each global edge unknown is one function on the two columns of its
    edge: its flux density across the edge (the normal component in each
    flat triangle's own plane, oriented from the first column to the second)
    is the same from both sides at every point of the edge (a swapped point
    or a wrong sign breaks this)."""
    m = mesh.hierarchy(1, 1)[0]
    owner, nhe, _ = nlo.horizontal_dofs(m, 1)
    by_base = {}
    for (c, a, base, sgn) in owner:
        if base < nhe:
            by_base.setdefault(base, []).append((c, a, sgn))
    tri = {}
    for base, sides in by_base.items():
        assert len(sides) == 2
        (c0, a0, s0), (c1, a1, s1) = sides
        for c in (c0, c1):
            if c not in tri:
                tri[c] = nlo.triangle_bdfm(m.verts[m.faces[c]])
        k0 = a0 // 2
        i, j = (k0 + 1) % 3, (k0 + 2) % 3
        P = m.verts[m.faces[c0]]
        n0, n1 = tri[c0].normals[k0], tri[c1].normals[a1 // 2]   # outward normals of each column
        for s in (0.0, 0.3, 0.7, 1.0):
            x = P[i] + s * (P[j] - P[i])
            f0 = s0 * np.dot(nlo.evaluate(tri[c0].basis[a0], _bary(P, x)), n0)
            f1 = -s1 * np.dot(nlo.evaluate(tri[c1].basis[a1], _bary(m.verts[m.faces[c1]], x)), n1)
            assert f0 == pytest.approx(f1, abs=1e-10 * (1 + abs(f0)))


def test_nlo_matrices_by_prism_quadrature():
    """Entries of D_h, D_z and the lumped masses of the assembled operator
    against brute-force integration of the basis functions over the physical
    prisms: the triangle scaled to the mid-layer radius, Gauss rules in the
    plane and in z, divergences by central differences."""
    ms = mesh.hierarchy(0, 1)
    m = ms[0]
    prm = helmholtz.Params(refinement=0, nlayers=2)
    nz, dz = prm.nlayers, prm.dz
    nop = nlo.assemble_nlo(m, prm)
    owner, nhe, nhf = nlo.horizontal_dofs(m, nz)
    rho = prm.rho()
    g, w = np.polynomial.legendre.leggauss(4)
    zq, zw = 0.5 * (g + 1.0) * dz, 0.5 * w * dz                      # Gauss points on one layer
    eta = lambda z: np.array([1.0 - z / dz, z / dz])                  # DG1 nodal in z
    s_ = lambda z: z / dz
    zeta = lambda z: np.array([(1 - s_(z)) * (1 - 2 * s_(z)), 4 * s_(z) * (1 - s_(z)), s_(z) * (2 * s_(z) - 1)])
    h = 1e-6
    rng = np.random.default_rng(5)
    Dh, Dz = nop.Dh.tocsc(), nop.Dz.tocsc()
    # horizontal unknowns: mass and divergence pairings
    for (c, a, base, sgn) in [owner[i] for i in rng.choice(len(owner), 12, replace=False)]:
        layer, b = rng.integers(nz), rng.integers(2)
        f = base + 2 * layer + b
        mass_q = 0.0
        for (c2, a2, base2, sgn2) in owner:
            if base2 != base:
                continue
            Pl = m.verts[m.faces[c2]] * rho[layer]
            T = nlo.triangle_bdfm(Pl)
            pts, wts = _quad_points(Pl)
            hm = sum(wq * np.dot(nlo.evaluate(T.basis[a2], _bary(Pl, x)), nlo.evaluate(T.basis[a2], _bary(Pl, x)))
                     for x, wq in zip(pts, wts))
            mass_q += hm * sum(wz * (eta(z)[b] / dz) ** 2 for z, wz in zip(zq, zw))
            e1 = (Pl[1] - Pl[0]) / np.linalg.norm(Pl[1] - Pl[0])
            e2 = np.cross(np.cross(Pl[1] - Pl[0], Pl[2] - Pl[0]), e1)
            e2 /= np.linalg.norm(e2)
            hx = 1e-5 * np.linalg.norm(Pl[1] - Pl[0])     # well above the spacing of doubles near |x| ~ R
            v = lambda x: sgn2 * nlo.evaluate(T.basis[a2], _bary(Pl, x))
            div = lambda x: (np.dot(v(x + hx * e1) - v(x - hx * e1), e1)
                             + np.dot(v(x + hx * e2) - v(x - hx * e2), e2)) / (2 * hx)
            for jv in range(3):
                for mm in range(2):
                    q = sum(wq * _bary(Pl, x)[jv] * div(x) for x, wq in zip(pts, wts)) * \
                        sum(wz * eta(z)[mm] * eta(z)[b] / dz for z, wz in zip(zq, zw))
                    got = Dh[nlo.pdof(c2, layer, jv, mm, nz), f]
                    assert got == pytest.approx(q, abs=1e-6 * max(1.0, abs(q)))
        assert nop.mh[f] == pytest.approx(mass_q, rel=1e-9)
    # vertical unknowns (column c, vertex i, node 1 .. 2 nz - 1)
    nzn = 2 * nz - 1
    for c in rng.choice(m.ncols, 4, replace=False):
        for i in range(3):
            for node in range(1, 2 * nz):
                f = (c * 3 + i) * nzn + node - 1
                mass_q = 0.0
                for layer in range(nz):
                    kz = node - 2 * layer
                    if kz < 0 or kz > 2:
                        continue
                    Pl = m.verts[m.faces[c]] * rho[layer]
                    area = 0.5 * np.linalg.norm(np.cross(Pl[1] - Pl[0], Pl[2] - Pl[0]))
                    pts, wts = _quad_points(Pl)
                    lam = [_bary(Pl, x) for x in pts]
                    mass_q += sum(wq * (lb[i] / (2 * area)) ** 2 for lb, wq in zip(lam, wts)) * \
                        sum(wz * zeta(z)[kz] ** 2 for z, wz in zip(zq, zw))
                    for jv in range(3):
                        for mm in range(2):
                            dzeta = lambda z: (zeta(z + h * dz)[kz] - zeta(z - h * dz)[kz]) / (2 * h * dz)
                            q = sum(wq * lb[jv] * lb[i] / (2 * area) for lb, wq in zip(lam, wts)) * \
                                sum(wz * eta(z)[mm] * dzeta(z) for z, wz in zip(zq, zw))
                            assert Dz[nlo.pdof(c, layer, jv, mm, nz), f] == pytest.approx(q, abs=1e-7 * max(1, abs(q)))
                assert nop.mz[f] == pytest.approx(mass_q, rel=1e-9)


@pytest.mark.parametrize("nz", [1, 2])
def test_nlo_short_columns(nz):
    """One and two layers: the vertical velocity has only the middle nodes
    (and one interface); H^ stays SPD with H^ 1 = M3 1, the column solve is
    exact for decoupled columns and the V-cycle is symmetric."""
    ms = mesh.hierarchy(1, 2)
    prm = helmholtz.Params(refinement=1, nlayers=nz)
    nop = nlo.assemble_nlo(ms[0], prm)
    lo = helmholtz.assemble_hierarchy(ms, prm)
    assert nop.mz.size == ms[0].ncols * 3 * (2 * nz - 1)
    H = nop.H.toarray()
    assert np.abs(H - H.T).max() <= 1e-14 * np.abs(H).max()
    assert np.linalg.eigvalsh(H).min() > 0
    one = np.ones(nop.n)
    assert np.allclose(nop.H @ one, nop.M3 @ one, rtol=1e-9)
    b = RNG.standard_normal(nop.n)
    import dataclasses
    u = nlo.smooth(dataclasses.replace(nop, H=nop.Hz), np.zeros(nop.n), b, 1.0)
    assert np.linalg.norm(nop.Hz @ u - b) <= 1e-12 * np.linalg.norm(b)
    x, y = RNG.standard_normal(nop.n), RNG.standard_normal(nop.n)
    assert abs(y @ nlo.vcycle(nop, lo, x) - x @ nlo.vcycle(nop, lo, y)) <= 1e-12 * abs(y @ nlo.vcycle(nop, lo, x))
