"""Pins of the oracle's smoother, transfers, V-cycle and Krylov solves
(Sec. 3.2, Sec. 4.2.1, Sec. 5, Algorithm 1)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import hmg_inputs as gi
from oracle import helmholtz, krylov, mesh, multigrid

RNG = np.random.default_rng(99)


def _ops(r, nz, L, **kw):
    ms = mesh.hierarchy(r, L)
    prm = helmholtz.Params(refinement=r, nlayers=nz, **kw)
    return ms, prm, helmholtz.assemble_hierarchy(ms, prm)


def test_transfers_are_adjoint_and_preserve_constants():
    nc, nz = 20, 5
    e = RNG.standard_normal(nc * nz)
    r = RNG.standard_normal(4 * nc * nz)
    assert np.dot(multigrid.prolong(e, nc, nz), r) == pytest.approx(np.dot(e, multigrid.restrict(r, nc, nz)), rel=1e-13)
    assert np.all(multigrid.prolong(np.ones(nc * nz), nc, nz) == 1.0)
    assert np.all(multigrid.restrict(np.ones(4 * nc * nz), nc, nz) == 4.0)
    # layer-wise: a coarse value reaches its 4 children in the same layer only
    x = np.zeros(nc * nz)
    x[3 * nz + 2] = 1.0
    y = multigrid.prolong(x, nc, nz).reshape(4 * nc, nz)
    assert set(map(tuple, np.argwhere(y).tolist())) == {(12, 2), (13, 2), (14, 2), (15, 2)}


def test_smoother_solves_decoupled_columns_exactly():
    """Without horizontal couplings (H^ = H^_z) and omega = 1 one line
    relaxation from zero is an exact solve."""
    _, _, ops = _ops(2, 16, 1)
    op = ops[0]
    op.H = op.Hz
    b = RNG.standard_normal(op.ncells)
    u = multigrid.smooth(op, np.zeros_like(b), b, 1.0)
    assert np.linalg.norm(op.Hz @ u - b) / np.linalg.norm(b) < 1e-12


def test_smoother_fixed_point_is_the_solution():
    _, _, ops = _ops(2, 8, 1)
    op = ops[0]
    b = RNG.standard_normal(op.ncells)
    x = spla.spsolve(op.H.tocsc(), b)
    u = multigrid.smooth(op, x, b, 0.8)
    assert np.linalg.norm(u - x) / np.linalg.norm(x) < 1e-11


def test_single_level_cycle_is_two_sweeps():
    _, _, ops = _ops(2, 8, 1)
    b = RNG.standard_normal(ops[0].ncells)
    u = multigrid.smooth(ops[0], np.zeros_like(b), b, 0.8)
    u = multigrid.smooth(ops[0], u, b, 0.8)
    assert np.array_equal(multigrid.vcycle(ops, b), u)


def test_vcycle_linear_symmetric_positive():
    _, _, ops = _ops(3, 8, 3)
    n = ops[0].ncells
    V = lambda v: multigrid.vcycle(ops, v)
    for _ in range(3):
        x, y = RNG.standard_normal((2, n))
        a, c = RNG.standard_normal(2)
        assert np.allclose(V(a * x + c * y), a * V(x) + c * V(y), rtol=1e-11, atol=1e-11 * np.abs(V(x)).max())
        assert np.dot(V(x), y) == pytest.approx(np.dot(x, V(y)), rel=1e-10)
        assert np.dot(x, V(x)) > 0


def _contraction(ops, iters=40):
    """Spectral radius of I - V H^ by power iteration."""
    x = RNG.standard_normal(ops[0].ncells)
    rho = 0.0
    for _ in range(iters):
        y = x - multigrid.vcycle(ops, ops[0].H @ x)
        rho = np.linalg.norm(y) / np.linalg.norm(x)
        x = y / np.linalg.norm(y)
    return rho


def test_vcycle_contraction_bounded_and_level_independent():
    """rho(I - V H^) < 1 and, with the coarsest mesh fixed (refinement 1) and
    the fine grid refined with one more level, unchanged (measured 0.348 at
    r4 / 4 levels and 0.347 at r5 / 5 levels)."""
    rho4 = _contraction(_ops(4, 16, 4)[2])
    rho5 = _contraction(_ops(5, 16, 5)[2])
    assert rho4 < 0.5 and rho5 < 0.5
    assert abs(rho4 - rho5) < 0.05
    # a smaller hierarchy over a coarser coarsest level still contracts
    assert _contraction(_ops(3, 16, 3)[2]) < 0.9


def test_pcg_matches_direct_solve_smallest_workload():
    w = gi.WORKLOADS["r3x16"]
    _, _, ops = _ops(w["refinement"], w["nlayers"], w["nlevels"])
    b = gi.rhs(ops[0].ncells)
    x, info = krylov.pcg(ops[0].H.dot, lambda v: multigrid.vcycle(ops, v), b, rtol=1e-8)
    assert info.converged and info.residuals[-1] < 1e-8
    xs = spla.spsolve(ops[0].H.tocsc(), b)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-7
    # the recursive residual tracks the true one
    true_rel = np.linalg.norm(b - ops[0].H @ x) / np.linalg.norm(b)
    assert true_rel < 2e-8


def test_manufactured_solution():
    _, _, ops = _ops(3, 16, 3)
    ps = gi.pstar(ops[0].ncells)
    b = ops[0].H @ ps
    x, info = krylov.pcg(ops[0].H.dot, lambda v: multigrid.vcycle(ops, v), b, rtol=1e-10)
    assert np.linalg.norm(x - ps) / np.linalg.norm(ps) < 1e-7


def test_grid_independent_iterations_and_multigrid_beats_single_level():
    """Sec. 5.2: at fixed nu_CFL = 8 the iteration count does not grow with
    resolution; Sec. 5.1: the single-level method needs several times more."""
    counts = []
    for r, L in [(2, 2), (3, 3), (4, 4)]:
        _, _, ops = _ops(r, 16, L)
        b = gi.rhs(ops[0].ncells)
        _, info = krylov.pcg(ops[0].H.dot, lambda v: multigrid.vcycle(ops, v), b, rtol=1e-8)
        counts.append(info.iterations)
        if r == 4:
            _, one = krylov.pcg(ops[0].H.dot, lambda v: multigrid.vcycle(ops[:1], v), b, rtol=1e-8, max_iter=1000)
            assert one.iterations > 3 * info.iterations
    # measured 15, 14, 11: no growth with resolution
    assert all(b <= a + 1 for a, b in zip(counts, counts[1:]))


def test_flexible_cg_agrees_with_cg_for_a_linear_preconditioner():
    _, _, ops = _ops(3, 16, 3)
    b = gi.rhs(ops[0].ncells)
    P = lambda v: multigrid.vcycle(ops, v)
    x1, i1 = krylov.pcg(ops[0].H.dot, P, b, rtol=1e-8)
    x2, i2 = krylov.fpcg(ops[0].H.dot, P, b, rtol=1e-8)
    assert abs(i1.iterations - i2.iterations) <= 1
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x1) < 1e-7


def _conjugacy_of_successive_directions(solver, ops, b, max_iter):
    """Run `solver` with a preconditioner that changes between calls (V-cycles
    alternating between 1 and 3 smoothing steps, so not a fixed linear map)
    and return max_k |p_k^T H p_(k-1)| / (||p_k||_H ||p_(k-1)||_H) over the
    search directions p_k, which are exactly the vectors the solver hands to
    the operator."""
    H = ops[0].H
    calls = [0]

    def precond(v):
        nu = 1 if calls[0] % 2 == 0 else 3
        calls[0] += 1
        return multigrid.vcycle(ops, v, nu_pre=nu, nu_post=nu)

    dirs = []

    def apply_A(p):
        dirs.append(p.copy())
        return H.dot(p)

    solver(apply_A, precond, b, rtol=1e-14, max_iter=max_iter)
    worst = 0.0
    for p1, p0 in zip(dirs[1:], dirs[:-1]):
        Hp0 = H.dot(p0)
        den = np.sqrt(np.dot(p1, H.dot(p1)) * np.dot(p0, Hp0))
        worst = max(worst, abs(np.dot(p1, Hp0)) / den)
    return worst, len(dirs)


def test_flexible_cg_keeps_successive_directions_conjugate_for_a_varying_preconditioner():
    """Flexible CG (Polak-Ribiere beta = z_k.(r_k - r_(k-1)) / z_(k-1).r_(k-1)):
    with alpha_(k-1) = z_(k-1).r_(k-1) / p_(k-1).H p_(k-1) and
    r_k - r_(k-1) = -alpha_(k-1) H p_(k-1), beta equals
    -z_k.H p_(k-1) / p_(k-1).H p_(k-1), so p_k = z_k + beta p_(k-1) is
    H-conjugate to p_(k-1) whatever z_k the preconditioner returns.  The
    Fletcher-Reeves beta of plain CG (z_k.r_k / z_(k-1).r_(k-1)) has that
    property only when z_k.r_(k-1) = 0, i.e. for a fixed symmetric
    preconditioner; with the alternating V-cycle it loses it, which the
    second half of the test shows, so a flexible CG that silently used the
    plain-CG beta fails here."""
    _, _, ops = _ops(3, 16, 3)
    b = gi.rhs(ops[0].ncells)
    worst, n = _conjugacy_of_successive_directions(krylov.fpcg, ops, b, 8)
    assert n == 8
    assert worst < 1e-10
    worst_plain, _ = _conjugacy_of_successive_directions(krylov.pcg, ops, b, 8)
    assert worst_plain > 1e-4
