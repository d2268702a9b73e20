"""GPU parity of the next-to-lowest-order velocity-pressure system (Eq.
PressureVelocitySystem at NLO) and its GMRES solve with the
Schur-complement preconditioner and the NLO V-cycle, against the oracle
(oracle/nlo_mixed.py).  Unknowns are matched by tests.helpers
(columns by centroid, vertices and edge points by position, signs from
the normal and Whitney orientations).  Tolerances: operator 1e-13 relative
L2 per block; solves: iterations within 1, blocks 1e-9 (rtol 1e-10) or 1e-6
(rtol 1e-5)."""
import numpy as np
import pytest

import hmg_inputs as gi
from oracle import helmholtz, krylov, mesh, nlo, nlo_mixed
from tests.helpers import nlo_mixed_permutation, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1605_00492_gb300 as hmg  # noqa: E402

DEV = "cuda:0"


class Case:
    def __init__(self, r, nz, L):
        self.ms = mesh.hierarchy(r, L)
        self.prm = helmholtz.Params(refinement=r, nlayers=nz)
        self.nop = nlo.assemble_nlo(self.ms[0], self.prm)
        self.lo = helmholtz.assemble_hierarchy(self.ms, self.prm)
        self.mop = nlo_mixed.assemble_nlo_mixed(self.ms[0], self.prm, self.nop)
        self.h = hmg.Hierarchy(r, nz, L)
        self.h.assemble()
        cen, _ = self.h.export_mesh(0)
        self.idx, self.sgn = nlo_mixed_permutation(cen, self.h.export_vertices(0), self.h.export_edges(), self.ms[0],
                                                   nz)
        assert sum(self.h.nlo_mixed_sizes()) == self.mop.n

    def gpu(self, x):
        return torch.tensor(self.sgn * np.asarray(x)[self.idx], dtype=torch.float64, device=DEV)

    def oracle_order(self, t):
        out = np.empty(self.mop.n)
        out[self.idx] = self.sgn * t.cpu().numpy()
        return out

    def blocks(self, x):
        m = self.mop
        return x[:m.nhf], x[m.nhf:m.nu], x[m.nu:]


_CACHE = {}


def case(*a):
    if a not in _CACHE:
        _CACHE[a] = Case(*a)
    return _CACHE[a]


@pytest.mark.parametrize("r,nz,L", [(1, 3, 2), (2, 4, 2), (3, 8, 3)])
def test_nlo_mixed_operator_matches_oracle(r, nz, L):
    c = case(r, nz, L)
    x = np.random.default_rng(12).standard_normal(c.mop.n)
    y = c.oracle_order(c.h.nlo_mixed_apply(c.gpu(x)))
    for got, ref in zip(c.blocks(y), c.blocks(c.mop.A @ x)):
        assert rel_l2(got, ref) < 1e-13


@pytest.mark.parametrize("rtol,orth", [(1e-5, 1), (1e-10, 2)])
def test_nlo_mixed_solve_matches_oracle(rtol, orth):
    c = case(2, 4, 2)
    b = nlo_mixed.assembled_rhs(c.mop, gi.mixed_rhs(c.mop.nu, c.mop.npr))
    x_ref, info_ref = krylov.fgmres(lambda v: c.mop.A @ v,
                                    lambda v: nlo_mixed.schur_precondition(c.mop, c.nop, c.lo, v), b, rtol=rtol,
                                    restart=30)
    x, info = c.h.nlo_mixed_solve(c.gpu(b), rtol=rtol, orth=orth, max_iter=500)
    assert info["converged"] == 1
    assert abs(info["iterations"] - info_ref.iterations) <= 1, (info, info_ref.iterations)
    assert info["true_rel_residual"] < 2 * rtol
    tol = 1e-9 if rtol < 1e-8 else 1e-6
    for got, ref in zip(c.blocks(c.oracle_order(x)), c.blocks(x_ref)):
        assert rel_l2(got, ref) < tol


def test_nlo_mixed_solve_mixed_precision_and_status():
    c = case(2, 4, 2)
    b = nlo_mixed.assembled_rhs(c.mop, gi.mixed_rhs(c.mop.nu, c.mop.npr))
    x_ref, _ = krylov.fgmres(lambda v: c.mop.A @ v, lambda v: nlo_mixed.schur_precondition(c.mop, c.nop, c.lo, v),
                             b, rtol=1e-10, restart=30)
    x, info = c.h.nlo_mixed_solve(c.gpu(b), rtol=1e-10, precision="mixed", max_iter=500)
    assert info["converged"] == 1 and info["true_rel_residual"] < 2e-10
    for got, ref in zip(c.blocks(c.oracle_order(x)), c.blocks(x_ref)):
        assert rel_l2(got, ref) < 1e-8
    _, info = c.h.nlo_mixed_solve(c.gpu(b), rtol=1e-12, max_iter=2, raise_on_failure=False)
    assert info["status"] == "HMG_ERR_NOT_CONVERGED" and info["iterations"] == 2
    with pytest.raises(hmg.HMGError):
        c.h.nlo_mixed_solve(c.gpu(b), restart=0)
