"""Pins of the oracle's velocity-pressure system (Eq. PressureVelocitySystem)
and Schur-complement preconditioner (Eq. SchurComplement, Eq. LumpedMass)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import hmg_inputs as gi
from oracle import helmholtz, krylov, mesh, mixed, multigrid

RNG = np.random.default_rng(2024)


def _random_triangles(n):
    return RNG.standard_normal((n, 3, 3))


def test_rt0_local_mass_against_quadrature_and_flux():
    """S[k, k'] = int_T w_k . w_k' for w_k = (x - v_k) / (2|T|): w_k . w_k'
    is quadratic, so the three-edge-midpoint rule is exact.  The same
    functions have flux 1 through edge k and no normal component on the
    other two edges (the RT0 unit-flux basis)."""
    tri = _random_triangles(50)
    faces = np.arange(150).reshape(50, 3)
    verts = tri.reshape(150, 3)
    m = mesh.Mesh2D(0, verts, faces, np.zeros_like(faces), mesh.flat_area(verts, faces),
                    mesh.shape_factor(verts, faces), verts[faces].mean(axis=1))
    S = mixed.rt0_local_mass(m)
    for F in range(50):
        v = tri[F]
        area = 0.5 * np.linalg.norm(np.cross(v[1] - v[0], v[2] - v[0]))
        mids = [(v[0] + v[1]) / 2, (v[1] + v[2]) / 2, (v[2] + v[0]) / 2]
        w = lambda k, x: (x - v[k]) / (2 * area)
        for k in range(3):
            for kk in range(3):
                q = area / 3 * sum(np.dot(w(k, x), w(kk, x)) for x in mids)
                assert S[F, k, kk] == pytest.approx(q, rel=1e-12)
        nrm = np.cross(v[1] - v[0], v[2] - v[0])
        nrm /= np.linalg.norm(nrm)
        for k in range(3):
            a, b = v[(k + 1) % 3], v[(k + 2) % 3]          # edge k (opposite v_k)
            out = np.cross(b - a, nrm)                      # outward in-plane normal, length |edge|
            if np.dot(out, a - v[k]) < 0:
                out = -out
            for kk in range(3):
                # w_kk . n is constant on a straight edge: flux = value at the midpoint x |edge|
                flux = np.dot(w(kk, (a + b) / 2), out)
                assert flux == pytest.approx(1.0 if kk == k else 0.0, abs=1e-12)
    # the diagonal is the shape factor of the lumped masses
    assert np.allclose(np.einsum("fkk->fk", S), m.sigma, rtol=1e-13)


@pytest.fixture(scope="module")
def small():
    ms = mesh.hierarchy(2, 2)
    prm = helmholtz.Params(refinement=2, nlayers=6)
    mop = mixed.assemble_mixed(ms[0], prm)
    ops = helmholtz.assemble_hierarchy(ms, prm)
    return ms, prm, mop, ops


def test_lumped_diagonal_gives_the_helmholtz_operator(small):
    """diag(M2^h), diag(M2^z) are the lumped masses, and M3 + w_c^2 D M2inv D^T
    with M2inv = 1 / diag(M2~) is exactly the assembled H^ (Eq. Preconditioner)."""
    ms, prm, mop, ops = small
    op = ops[0]
    assert np.allclose(mop.Mh.diagonal(), op.mh, rtol=1e-13)
    assert np.allclose(mop.Mz.diagonal(), op.mz, rtol=1e-13)
    import scipy.sparse as sp
    Hs = sp.diags(mop.M3) + prm.omega_c ** 2 * (mop.D @ sp.diags(1.0 / mop.m2diag) @ mop.D.T)
    d = (Hs - op.H).tocoo()
    assert np.max(np.abs(d.data)) <= 1e-12 * np.max(np.abs(op.H.data))


def test_velocity_mass_spd_and_sparsity(small):
    ms, prm, mop, ops = small
    for M in (mop.Mh, mop.Mz):
        Md = M.toarray()
        assert np.allclose(Md, Md.T, rtol=1e-14, atol=0)
        assert np.linalg.eigvalsh(Md).min() > 0
    # a horizontal face couples with itself and the other two faces of each of its two cells
    assert set(np.diff(mop.Mh.indptr)) == {5}
    # total divergence over the closed shell vanishes (no flux through top and bottom)
    u = RNG.standard_normal(mop.nu)
    assert abs(np.sum(mop.D @ u)) <= 1e-12 * np.sum(np.abs(u))


def test_schur_factorisation_with_exact_inverses_is_the_inverse():
    """With exact M2~^-1 and S^-1 (S = M3 + w_c^2 D M2~^-1 D^T) in place of the
    lumped mass and the V-cycle, Eq. SchurComplement is A^-1 exactly."""
    m = mesh.hierarchy(0, 1)[0]
    prm = helmholtz.Params(refinement=0, nlayers=3)
    mop = mixed.assemble_mixed(m, prm)
    A = mop.A.toarray()
    nu = mop.nu
    M = A[:nu, :nu]
    Minv = np.linalg.inv(M)
    D = mop.D.toarray()
    S = np.diag(mop.M3) + mop.a ** 2 * mop.c2 * D @ Minv @ D.T
    n = mop.n
    up = np.eye(n)
    up[:nu, nu:] = mop.a * Minv @ D.T
    mid = np.zeros((n, n))
    mid[:nu, :nu] = Minv
    mid[nu:, nu:] = np.linalg.inv(S)
    lo = np.eye(n)
    lo[nu:, :nu] = -mop.a * mop.c2 * D @ Minv
    Ainv = up @ mid @ lo
    b = RNG.standard_normal(n)
    x_ref = np.linalg.solve(A, b)
    assert np.linalg.norm(Ainv @ b - x_ref) <= 1e-9 * np.linalg.norm(x_ref)


def test_gmres_with_schur_preconditioner_solves_the_system(small):
    ms, prm, mop, ops = small
    b = mixed.assembled_rhs(mop, gi.mixed_rhs(mop.nu, mop.M3.size))
    x_direct = spla.spsolve(mop.A.tocsc(), b)
    x, info = krylov.fgmres(lambda v: mixed.apply_mixed(mop, v), lambda v: mixed.schur_precondition(mop, ops, v),
                            b, rtol=1e-10, restart=30)
    assert info.converged
    assert np.linalg.norm(mop.A @ x - b) / np.linalg.norm(b) < 1.01e-10
    nu = mop.nu
    assert np.linalg.norm(x[:nu] - x_direct[:nu]) / np.linalg.norm(x_direct[:nu]) < 1e-8
    assert np.linalg.norm(x[nu:] - x_direct[nu:]) / np.linalg.norm(x_direct[nu:]) < 1e-8
    # the lumped Schur preconditioner keeps the outer iteration short (Sec. 6: about 10 at 1e-5)
    _, info5 = krylov.fgmres(lambda v: mixed.apply_mixed(mop, v), lambda v: mixed.schur_precondition(mop, ops, v),
                             b, rtol=1e-5, restart=30)
    assert info5.iterations <= 20


def test_outer_iterations_do_not_grow_with_resolution():
    """Fixed coarsest mesh (refinement 1), Courant number 8 (Sec. 6)."""
    its = []
    for r in (2, 3, 4):
        ms = mesh.hierarchy(r, r)
        prm = helmholtz.Params(refinement=r, nlayers=8)
        mop = mixed.assemble_mixed(ms[0], prm)
        ops = helmholtz.assemble_hierarchy(ms, prm)
        b = mixed.assembled_rhs(mop, gi.mixed_rhs(mop.nu, mop.M3.size))
        _, info = krylov.fgmres(lambda v: mixed.apply_mixed(mop, v),
                                lambda v: mixed.schur_precondition(mop, ops, v), b, rtol=1e-5, restart=30)
        assert info.converged
        its.append(info.iterations)
    assert all(b <= a + 1 for a, b in zip(its, its[1:])), its


def test_velocity_mass_energy_identities(small):
    """U^T M2^h U = sum over cells of (D_K U)^T S_K (D_K U) / dz with the cell's
    signed face fluxes taken from the Helmholtz module's D_h, and
    U^T M2^z U = sum over cells of int_K u_z^2 by Simpson's rule (exact for
    the quadratic u_z^2 of P1-in-z fluxes)."""
    ms, prm, mop, ops = small
    m, op = ms[0], ops[0]
    nz, dz = prm.nlayers, prm.dz
    S = mixed.rt0_local_mass(m)
    Dh = op.Dh.tocsr()
    u = RNG.standard_normal(mop.nhf)
    e_ref = 0.0
    edges = helmholtz.horizontal_faces(m)
    for c in range(m.ncols):
        for lay in range(nz):
            K = c * nz + lay
            loc = np.zeros(3)
            for k in range(3):
                nb = m.nbr[c, k]
                t0, t1 = min(c, nb), max(c, nb)
                e = np.flatnonzero((edges[:, 0] == t0) & (edges[:, 2] == t1))[0]
                f = e * nz + lay
                loc[k] = Dh[K, f] * u[f]
            e_ref += loc @ S[c] @ loc / dz
    assert u @ (mop.Mh @ u) == pytest.approx(e_ref, rel=1e-12)
    w = RNG.standard_normal(mop.nvf)
    area = m.area1[:, None] * prm.rho()[None, :] ** 2
    e_ref = 0.0
    for c in range(m.ncols):
        for lay in range(nz):
            ub = w[c * (nz - 1) + lay - 1] if lay > 0 else 0.0
            ut = w[c * (nz - 1) + lay] if lay < nz - 1 else 0.0
            A = area[c, lay]
            vals = np.array([ub, 0.5 * (ub + ut), ut]) / A
            e_ref += A * dz / 6.0 * (vals[0] ** 2 + 4 * vals[1] ** 2 + vals[2] ** 2)
    assert w @ (mop.Mz @ w) == pytest.approx(e_ref, rel=1e-12)


def test_schur_preconditioner_is_exact_for_a_diagonal_velocity_mass(small, monkeypatch):
    """If the velocity mass were its own diagonal, Eq. SchurComplement with
    the lumped inverse and an exact H^ solve would invert the system: the
    preconditioner applied to A_lumped x returns x."""
    import scipy.sparse as sp
    ms, prm, mop, ops = small
    Hlu = spla.splu(ops[0].H.tocsc())
    monkeypatch.setattr(mixed.multigrid, "vcycle", lambda ops_, r: Hlu.solve(r))
    A_l = sp.bmat([[sp.diags(mop.m2diag), -mop.a * mop.D.T], [mop.a * mop.c2 * mop.D, sp.diags(mop.M3)]]).tocsr()
    x = np.concatenate([RNG.standard_normal(mop.nu) * 1e6, RNG.standard_normal(mop.M3.size)])
    y = mixed.schur_precondition(mop, ops, A_l @ x)
    nu = mop.nu
    assert np.linalg.norm(y[:nu] - x[:nu]) <= 1e-8 * np.linalg.norm(x[:nu])
    assert np.linalg.norm(y[nu:] - x[nu:]) <= 1e-8 * np.linalg.norm(x[nu:])


def test_assembled_rhs_blocks(small):
    ms, prm, mop, ops = small
    r = gi.mixed_rhs(mop.nu, mop.M3.size)
    b = mixed.assembled_rhs(mop, r)
    nh, nu = mop.nhf, mop.nu
    assert np.allclose(b[:nh], mop.Mh @ r[:nh], rtol=1e-14)
    assert np.allclose(b[nh:nu], (1 + prm.omega_N ** 2) * (mop.Mz @ r[nh:nu]), rtol=1e-14)
    assert np.array_equal(b[nu:], mop.M3 * r[nu:])
