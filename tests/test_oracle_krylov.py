"""Pins of the oracle's restarted flexible GMRES(m) (Sec. 5's outer solver;
Saad, Iterative Methods for Sparse Linear Systems, Sec. 6.5 and Algorithm
9.6) against what the mathematics fixes: the minimal-residual property over
the explicit Krylov space, the closed form of the one-step restart (the
minimal residual iteration), finite termination of full GMRES, and the
solution of H^ p = b with the V-cycle."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import hmg_inputs as gi
from oracle import helmholtz, krylov, mesh, multigrid

RNG = np.random.default_rng(1234)


def _nonsymmetric(n):
    A = RNG.standard_normal((n, n)) + n * np.eye(n)
    M = np.eye(n) + 0.1 * RNG.standard_normal((n, n))   # fixed, nonsymmetric right preconditioner
    return A, M


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_iterate_minimises_the_residual_over_the_krylov_space(k):
    """Right preconditioning: x_k = M y with y in K_k(A M, b), and x_k
    minimises ||b - A x|| there.  Brute force: an orthonormal basis of the
    explicit Krylov matrix [b, AMb, ..., (AM)^(k-1) b] and numpy least squares."""
    n = 24
    A, M = _nonsymmetric(n)
    b = RNG.standard_normal(n)
    AM = A @ M
    K = np.empty((n, k))
    K[:, 0] = b
    for i in range(1, k):
        K[:, i] = AM @ K[:, i - 1]
    Q, _ = np.linalg.qr(K)
    X = M @ Q
    c, *_ = np.linalg.lstsq(A @ X, b, rcond=None)
    x_bf = X @ c
    x, info = krylov.fgmres(A.dot, M.dot, b, rtol=0.0, max_iter=k, restart=max(k, 2))
    assert info.iterations == k and not info.converged
    assert np.linalg.norm(x - x_bf) <= 1e-10 * np.linalg.norm(x_bf)
    # the least-squares estimate is the true residual of the iterate
    true = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert info.residuals[-1] == pytest.approx(true, rel=1e-9)


def test_restart_one_is_the_minimal_residual_iteration():
    """GMRES(1): x <- x + alpha z, z = M r, alpha = (A z . r) / ||A z||^2."""
    n = 16
    A, M = _nonsymmetric(n)
    b = RNG.standard_normal(n)
    x_ref = np.zeros(n)
    for _ in range(5):
        r = b - A @ x_ref
        z = M @ r
        Az = A @ z
        x_ref = x_ref + (np.dot(Az, r) / np.dot(Az, Az)) * z
    x, info = krylov.fgmres(A.dot, M.dot, b, rtol=0.0, max_iter=5, restart=1)
    assert info.iterations == 5
    assert np.linalg.norm(x - x_ref) <= 1e-12 * np.linalg.norm(x_ref)


def test_full_gmres_terminates_in_n_steps():
    n = 12
    A, _ = _nonsymmetric(n)
    b = RNG.standard_normal(n)
    x, info = krylov.fgmres(A.dot, lambda v: v, b, rtol=1e-12, max_iter=n, restart=n)
    assert info.converged and info.iterations <= n
    x_ref = np.linalg.solve(A, b)
    assert np.linalg.norm(x - x_ref) <= 1e-10 * np.linalg.norm(x_ref)


def test_residual_history_is_monotone_within_a_cycle():
    n = 30
    A, M = _nonsymmetric(n)
    b = RNG.standard_normal(n)
    _, info = krylov.fgmres(A.dot, M.dot, b, rtol=1e-10, max_iter=40, restart=8)
    res = np.asarray(info.residuals)
    assert np.all(np.diff(res) <= 1e-15)


def test_vcycle_preconditioned_gmres_solves_helmholtz():
    ms = mesh.hierarchy(3, 3)
    prm = helmholtz.Params(refinement=3, nlayers=16)
    ops = helmholtz.assemble_hierarchy(ms, prm)
    b = gi.rhs(ops[0].ncells)
    x_direct = spla.spsolve(ops[0].H.tocsc(), b)
    x, info = krylov.fgmres(ops[0].H.dot, lambda v: multigrid.vcycle(ops, v), b, rtol=1e-10)
    assert info.converged
    assert np.linalg.norm(b - ops[0].H @ x) / np.linalg.norm(b) < 1.01e-10
    assert np.linalg.norm(x - x_direct) / np.linalg.norm(x_direct) < 1e-8
    # GMRES minimises the residual norm, CG the energy norm: their counts are close
    _, info_cg = krylov.pcg(ops[0].H.dot, lambda v: multigrid.vcycle(ops, v), b, rtol=1e-10)
    assert abs(info.iterations - info_cg.iterations) <= 3
    # restarting every 4 steps still converges, in more steps
    x4, info4 = krylov.fgmres(ops[0].H.dot, lambda v: multigrid.vcycle(ops, v), b, rtol=1e-10, restart=4)
    assert info4.converged and info4.iterations >= info.iterations
    assert np.linalg.norm(x4 - x_direct) / np.linalg.norm(x_direct) < 1e-8
