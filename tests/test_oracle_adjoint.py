"""Pins of the oracle's adjoint gradients (dL/db, dL/dtheta)."""
import numpy as np
import pytest

import hmg_inputs as gi
from oracle import adjoint, helmholtz, krylov, mesh, multigrid

RNG = np.random.default_rng(7)


def _dense_loss(m, prm, theta, b, pt):
    H = helmholtz.assemble(m, prm, theta).H.toarray()
    dtype = np.result_type(H, b)
    p = np.linalg.solve(H.astype(dtype), b.astype(dtype))
    d = p - pt
    return 0.5 * np.sum(d * d)


def test_theta_gradient_matches_complex_step_dense():
    """Complex-step derivative of the dense tiny problem (r0 x 4 layers, 80
    cells): exact to rounding, independent of the adjoint formula."""
    m = mesh.hierarchy(0, 1)[0]
    prm = helmholtz.Params(refinement=0, nlayers=4)
    n = m.ncols * 4
    theta = np.exp(0.3 * RNG.standard_normal(n))
    b = RNG.standard_normal(n)
    op = helmholtz.assemble(m, prm, theta)
    H = op.H.toarray()
    p = np.linalg.solve(H, b)
    pt = p + 0.5 * np.abs(p).max() * RNG.standard_normal(n)
    lam = np.linalg.solve(H, p - pt)
    g = adjoint.theta_gradient(op, prm, m, theta, p, lam)
    h = 1e-30
    for K in [0, 1, 5, 17, 40, 79]:
        tc = theta.astype(complex)
        tc[K] += 1j * h
        cs = _dense_loss(m, prm, tc, b, pt).imag / h
        assert cs != 0.0
        assert g[K] == pytest.approx(cs, rel=1e-9, abs=1e-9 * np.abs(g).max())
    # dL/db = lambda, also by complex step in b
    for K in [3, 50]:
        bc = b.astype(complex)
        bc[K] += 1j * h
        cs = _dense_loss(m, prm, theta, bc, pt).imag / h
        assert cs != 0.0
        assert lam[K] == pytest.approx(cs, rel=1e-9, abs=0.0)


def test_theta_gradient_central_differences_with_multigrid_solves():
    ms = mesh.hierarchy(2, 2)
    prm = helmholtz.Params(refinement=2, nlayers=8)
    n = ms[0].ncols * 8
    theta = gi.theta(n)
    b = gi.rhs(n)
    solve = lambda ops, rhs: krylov.pcg(ops[0].H.dot, lambda v: multigrid.vcycle(ops, v), rhs, rtol=1e-14, max_iter=200)[0]
    ops = helmholtz.assemble_hierarchy(ms, prm, theta)
    p0 = solve(ops, b)
    pt = p0 + 0.1 * np.abs(p0).max() * gi.ptarget(n)
    L, lam, g, _ = adjoint.value_and_grad(ops, prm, ms[0], theta, b, pt, solve)
    h = 1e-6
    for v in gi.directions(n, 3):
        Lp = adjoint.loss(solve(helmholtz.assemble_hierarchy(ms, prm, theta + h * v), b), pt)
        Lm = adjoint.loss(solve(helmholtz.assemble_hierarchy(ms, prm, theta - h * v), b), pt)
        fd = (Lp - Lm) / (2 * h)
        assert np.dot(g, v) == pytest.approx(fd, rel=1e-6)
