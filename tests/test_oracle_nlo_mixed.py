"""Pins of the oracle's next-to-lowest-order velocity-pressure system (Eq.
PressureVelocitySystem with the NLO spaces) and its Schur-complement
preconditioner (Eq. SchurComplement, Eq. LumpedMass)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import hmg_inputs as gi
from oracle import helmholtz, krylov, mesh, nlo, nlo_mixed

RNG = np.random.default_rng(31)


def _bary(P, x):
    M = np.stack([P[1] - P[0], P[2] - P[0]], axis=1)
    st, *_ = np.linalg.lstsq(M, x - P[0], rcond=None)
    return np.array([1.0 - st[0] - st[1], st[0], st[1]])


def _quad_points(P, n=5):
    g, w = np.polynomial.legendre.leggauss(n)
    g, w = 0.5 * (g + 1.0), 0.5 * w
    area2 = np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
    pts, wts = [], []
    for u, wu in zip(g, w):
        for v, wv in zip(g, w):
            pts.append(P[0] + u * (P[1] - P[0]) + v * (1.0 - u) * (P[2] - P[0]))
            wts.append(wu * wv * (1.0 - u) * area2)
    return np.array(pts), np.array(wts)


def _system(r, nz, L):
    ms = mesh.hierarchy(r, L)
    prm = helmholtz.Params(refinement=r, nlayers=nz)
    nop = nlo.assemble_nlo(ms[0], prm)
    lo = helmholtz.assemble_hierarchy(ms, prm)
    return ms, prm, nop, lo, nlo_mixed.assemble_nlo_mixed(ms[0], prm, nop)


@pytest.fixture(scope="module")
def small():
    return _system(1, 3, 2)


def test_lumped_diagonals_give_the_nlo_operator(small):
    """diag(M2^h), diag(M2^z) are the lumped masses of the NLO operator, and
    M3 + w_c^2 D M2inv D^T with M2inv = 1 / diag(M2~) is exactly its H^."""
    ms, prm, nop, lo, mop = small
    assert np.allclose(mop.Mh.diagonal(), nop.mh, rtol=1e-13, atol=0)
    assert np.allclose(mop.Mz.diagonal(), nop.mz, rtol=1e-13, atol=0)
    Hs = mop.M3 + prm.omega_c ** 2 * (mop.D @ sp.diags(1.0 / mop.m2diag) @ mop.D.T)
    assert abs(Hs - nop.H).max() <= 1e-13 * abs(nop.H).max()


def test_velocity_masses_spd(small):
    ms, prm, nop, lo, mop = small
    for M in (mop.Mh, mop.Mz):
        Md = M.toarray()
        assert np.abs(Md - Md.T).max() <= 1e-14 * np.abs(Md).max()
        assert np.linalg.eigvalsh(Md).min() > 0


def test_velocity_energies_by_prism_quadrature():
    """U^T M2^h U and W^T M2^z W equal the integrals of |u|^2 over the
    physical prisms for random coefficient vectors: the BDFM1 functions
    evaluated on each scaled triangle with the global signs, times the DG1 /
    P2 functions in z (Gauss rules in the plane and in z)."""
    ms = mesh.hierarchy(0, 1)
    m = ms[0]
    prm = helmholtz.Params(refinement=0, nlayers=2)
    nz, dz = prm.nlayers, prm.dz
    Mh, Mz = nlo_mixed.velocity_masses(m, prm)
    owner, nhe, nhf = nlo.horizontal_dofs(m, nz)
    rho = prm.rho()
    g, w = np.polynomial.legendre.leggauss(4)
    zq, zw = 0.5 * (g + 1.0) * dz, 0.5 * w * dz
    psi = lambda z: np.array([1.0 - z / dz, z / dz])
    U = RNG.standard_normal(nhf)
    e = 0.0
    for c in range(m.ncols):
        mine = [(a, base, sgn) for (cc, a, base, sgn) in owner if cc == c]
        for layer in range(nz):
            Pl = m.verts[m.faces[c]] * rho[layer]
            T = nlo.triangle_bdfm(Pl)
            pts, wts = _quad_points(Pl)
            for x, wx in zip(pts, wts):
                lam = _bary(Pl, x)
                vals = [nlo.evaluate(T.basis[a], lam) for (a, _, _) in mine]
                for z, wz in zip(zq, zw):
                    u = sum(sgn * U[base + 2 * layer + b] * vals[q] * psi(z)[b] / dz
                            for q, (a, base, sgn) in enumerate(mine) for b in range(2))
                    e += wx * wz * float(np.dot(u, u))
    assert U @ (Mh @ U) == pytest.approx(e, rel=1e-10)
    nzn = 2 * nz - 1
    W = RNG.standard_normal(Mz.shape[0])
    s_ = lambda z: z / dz
    zeta = lambda z: np.array([(1 - s_(z)) * (1 - 2 * s_(z)), 4 * s_(z) * (1 - s_(z)), s_(z) * (2 * s_(z) - 1)])
    e = 0.0
    for c in range(m.ncols):
        for layer in range(nz):
            Pl = m.verts[m.faces[c]] * rho[layer]
            area = 0.5 * np.linalg.norm(np.cross(Pl[1] - Pl[0], Pl[2] - Pl[0]))
            pts, wts = _quad_points(Pl)
            for x, wx in zip(pts, wts):
                lam = _bary(Pl, x)
                for z, wz in zip(zq, zw):
                    uz = 0.0
                    for kz in range(3):
                        node = 2 * layer + kz
                        if node == 0 or node == 2 * nz:
                            continue
                        for i in range(3):
                            uz += W[(c * 3 + i) * nzn + node - 1] * lam[i] * zeta(z)[kz] / (2 * area)
                    e += wx * wz * uz * uz
    assert W @ (Mz @ W) == pytest.approx(e, rel=1e-10)


def test_schur_factorisation_with_exact_inverses_is_the_inverse():
    ms, prm, nop, lo, mop = _system(0, 2, 1)
    A = mop.A.toarray()
    nu = mop.nu
    Minv = np.linalg.inv(A[:nu, :nu])
    D = mop.D.toarray()
    S = mop.M3.toarray() + mop.a ** 2 * mop.c2 * D @ Minv @ D.T
    n = mop.n
    up, mid, low = np.eye(n), np.zeros((n, n)), np.eye(n)
    up[:nu, nu:] = mop.a * Minv @ D.T
    mid[:nu, :nu] = Minv
    mid[nu:, nu:] = np.linalg.inv(S)
    low[nu:, :nu] = -mop.a * mop.c2 * D @ Minv
    b = RNG.standard_normal(n)
    x_ref = np.linalg.solve(A, b)
    assert np.linalg.norm(up @ mid @ low @ b - x_ref) <= 1e-8 * np.linalg.norm(x_ref)


def test_gmres_with_the_schur_preconditioner_solves_the_system(small):
    """Blocks agree with a sparse direct solve; at the paper's 1e-5 the outer
    GMRES(30) needs about the paper's NLO count (21 iterations, Table
    "SingleNodePerformance")."""
    ms, prm, nop, lo, mop = small
    b = nlo_mixed.assembled_rhs(mop, gi.mixed_rhs(mop.nu, mop.npr))
    x_direct = spla.spsolve(mop.A.tocsc(), b)
    pre = lambda v: nlo_mixed.schur_precondition(mop, nop, lo, v)
    x, info = krylov.fgmres(lambda v: mop.A @ v, pre, b, rtol=1e-11, restart=30)
    assert info.converged
    nu = mop.nu
    for sl in (slice(0, mop.nhf), slice(mop.nhf, nu), slice(nu, None)):
        assert np.linalg.norm(x[sl] - x_direct[sl]) <= 1e-6 * np.linalg.norm(x_direct[sl])
    _, info5 = krylov.fgmres(lambda v: mop.A @ v, pre, b, rtol=1e-5, restart=30)
    assert info5.converged and info5.iterations <= 30


def test_preconditioner_exact_for_a_diagonal_velocity_mass(small, monkeypatch):
    """With the velocity mass replaced by its diagonal and an exact H^ solve
    in place of the V-cycle, the preconditioner inverts the system."""
    ms, prm, nop, lo, mop = small
    Hlu = spla.splu(nop.H.tocsc())
    monkeypatch.setattr(nlo_mixed.nlo, "vcycle", lambda nop_, lo_, r: Hlu.solve(r))
    A_l = sp.bmat([[sp.diags(mop.m2diag), -mop.a * mop.D.T], [mop.a * mop.c2 * mop.D, mop.M3]]).tocsr()
    x = np.concatenate([RNG.standard_normal(mop.nu) * 1e6, RNG.standard_normal(mop.npr)])
    y = nlo_mixed.schur_precondition(mop, nop, lo, A_l @ x)
    nu = mop.nu
    assert np.linalg.norm(y[:nu] - x[:nu]) <= 1e-8 * np.linalg.norm(x[:nu])
    assert np.linalg.norm(y[nu:] - x[nu:]) <= 1e-8 * np.linalg.norm(x[nu:])
