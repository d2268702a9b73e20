"""GPU parity of the next-to-lowest-order path (operator, V-cycle with
p-coarsening, GMRES solve) against the oracle (oracle/nlo.py).

Columns are matched by centroid and the DG1 unknowns of a column by the
position of their vertex.  Tolerances (FP64): operator 1e-13 relative L2
(one rounding per term); V-cycle 1e-11 (the kernels' block L D L^T column
solve and the oracle's sparse LU differ by rounding, amplified by the
condition of the column blocks); solves 1e-9 with the iteration count within
one.
"""
import numpy as np
import pytest

import hmg_inputs as gi
from oracle import helmholtz, krylov, mesh, nlo
from tests.helpers import column_permutation, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1605_00492_gb300 as hmg  # noqa: E402

DEV = "cuda:0"


class NloCase:
    def __init__(self, r, nz, L, **op):
        self.ms = mesh.hierarchy(r, L)
        self.prm = helmholtz.Params(refinement=r, nlayers=nz, **op)
        self.nop = nlo.assemble_nlo(self.ms[0], self.prm)
        self.lo = helmholtz.assemble_hierarchy(self.ms, self.prm)
        self.h = hmg.Hierarchy(r, nz, L)
        self.h.assemble(**{k: v for k, v in op.items() if k in ("c", "N", "nu_cfl", "omega")})
        m = self.ms[0]
        cen, _ = self.h.export_mesh(0)
        perm = column_permutation(cen, m.centroid)
        verts = self.h.export_vertices(0)
        vp = np.empty((m.ncols, 3), dtype=np.int64)
        for c in range(m.ncols):
            d = np.linalg.norm(m.verts[m.faces[perm[c]]][None, :, :] - verts[c][:, None, :], axis=2)
            assert d.min(axis=1).max() < 1e-12
            vp[c] = d.argmin(axis=1)
        u = np.arange(6)
        lay = np.arange(nz)
        # idx[g] = oracle unknown of library unknown g (NLO COLUMN layouts)
        self.idx = (((perm[:, None, None] * nz + lay[None, :, None]) * 3 + vp[:, None, u // 2]) * 2
                    + u % 2).reshape(-1)
        assert self.h.nlo_size() == self.nop.n

    def gpu(self, v):
        return torch.tensor(np.asarray(v)[self.idx], dtype=torch.float64, device=DEV)

    def oracle_order(self, t):
        out = np.empty(self.nop.n)
        out[self.idx] = t.cpu().numpy()
        return out


_CACHE = {}


def case(*a, **k):
    key = (a, tuple(sorted(k.items())))
    if key not in _CACHE:
        _CACHE[key] = NloCase(*a, **k)
    return _CACHE[key]


@pytest.mark.parametrize("r,nz,L", [(1, 3, 2), (2, 4, 2), (3, 16, 3)])
def test_nlo_operator_matches_oracle(r, nz, L):
    c = case(r, nz, L)
    x = np.random.default_rng(3).standard_normal(c.nop.n)
    y = c.oracle_order(c.h.nlo_apply(c.gpu(x)))
    assert rel_l2(y, c.nop.H @ x) < 1e-13


@pytest.mark.parametrize("r,nz,L", [(1, 3, 2), (3, 16, 3)])
def test_nlo_vcycle_matches_oracle(r, nz, L):
    c = case(r, nz, L)
    b = gi.nlo_rhs(c.nop.n)
    z = c.oracle_order(c.h.nlo_vcycle(c.gpu(b)))
    assert rel_l2(z, nlo.vcycle(c.nop, c.lo, b)) < 1e-11
    # one and three sweeps per level
    z = c.oracle_order(c.h.nlo_vcycle(c.gpu(b), nu_pre=1, nu_post=3, n_coarse=1))
    assert rel_l2(z, nlo.vcycle(c.nop, c.lo, b, nu_pre=1, nu_post=3, n_coarse=1)) < 1e-11


def test_nlo_single_level_and_fewer_levels_match_oracle():
    c = case(2, 4, 2)
    b = gi.nlo_rhs(c.nop.n)
    # levels = 1: the NLO smoother alone, n_coarse sweeps from zero
    ref = np.zeros(c.nop.n)
    for _ in range(3):
        ref = nlo.smooth(c.nop, ref, b, 0.8)
    z = c.oracle_order(c.h.nlo_vcycle(c.gpu(b), levels=1, n_coarse=3))
    assert rel_l2(z, ref) < 1e-11
    # levels = 2: the NLO level and one lowest-order level (its coarsest)
    z = c.oracle_order(c.h.nlo_vcycle(c.gpu(b), levels=2))
    assert rel_l2(z, nlo.vcycle(c.nop, c.lo[:1], b)) < 1e-11


_SOLVES = {}


def oracle_solve(c, rtol):
    key = (id(c), rtol)
    if key not in _SOLVES:
        b = gi.nlo_rhs(c.nop.n)
        _SOLVES[key] = krylov.fgmres(lambda v: c.nop.H @ v, lambda v: nlo.vcycle(c.nop, c.lo, v), b, rtol=rtol,
                                     restart=30)
    return _SOLVES[key]


def test_nlo_vcycle_mixed_against_fp64_oracle():
    """The mixed form runs the NLO level and the non-coarsest lowest-order
    levels in FP32: against the FP64 oracle the V-cycle differs by the FP32
    rounding of the column solves (stated bound 1e-4, as for the lowest
    order), and a single-level mixed cycle is the FP64 one."""
    c = case(3, 16, 3)
    b = gi.nlo_rhs(c.nop.n)
    z = c.oracle_order(c.h.nlo_vcycle(c.gpu(b), precision="mixed"))
    assert rel_l2(z, nlo.vcycle(c.nop, c.lo, b)) < 1e-4
    z1 = c.oracle_order(c.h.nlo_vcycle(c.gpu(b), precision="mixed", levels=1))
    ref = nlo.smooth(c.nop, nlo.smooth(c.nop, np.zeros(c.nop.n), b, 0.8), b, 0.8)
    assert rel_l2(z1, ref) < 1e-11


@pytest.mark.parametrize("r,nz,L,rtol,orth", [(2, 8, 2, 1e-8, 1), (3, 16, 3, 1e-10, 2)])
def test_nlo_solve_matches_oracle(r, nz, L, rtol, orth):
    c = case(r, nz, L)
    b = gi.nlo_rhs(c.nop.n)
    x_ref, info_ref = oracle_solve(c, rtol)
    x, info = c.h.nlo_solve(c.gpu(b), rtol=rtol, orth=orth)
    assert info["converged"] == 1
    assert abs(info["iterations"] - info_ref.iterations) <= 1, (info, info_ref.iterations)
    assert info["true_rel_residual"] < 2 * rtol
    assert rel_l2(c.oracle_order(x), x_ref) < (1e-9 if rtol < 1e-9 else 1e-6)


def test_nlo_solve_mixed_precision_and_status():
    c = case(3, 16, 3)
    b = gi.nlo_rhs(c.nop.n)
    x_ref, _ = oracle_solve(c, 1e-10)
    x, info = c.h.nlo_solve(c.gpu(b), rtol=1e-9, precision="mixed")
    assert info["converged"] == 1 and info["true_rel_residual"] < 2e-9
    assert rel_l2(c.oracle_order(x), x_ref) < 1e-6
    _, info = c.h.nlo_solve(c.gpu(b), rtol=1e-12, max_iter=3, raise_on_failure=False)
    assert info["status"] == "HMG_ERR_NOT_CONVERGED" and info["iterations"] == 3
    with pytest.raises(hmg.HMGError):
        c.h.nlo_solve(c.gpu(b), krylov="cg")
    with pytest.raises(hmg.HMGError):
        c.h.nlo_solve(c.gpu(b), levels=5)


def test_nlo_reassembly_refreshes_coefficients():
    c = NloCase(2, 4, 2, nu_cfl=4.0)
    x = np.random.default_rng(5).standard_normal(c.nop.n)
    y4 = c.oracle_order(c.h.nlo_apply(c.gpu(x)))
    assert rel_l2(y4, c.nop.H @ x) < 1e-13
    c.h.assemble(nu_cfl=16.0)
    prm = helmholtz.Params(refinement=2, nlayers=4, nu_cfl=16.0)
    H16 = nlo.assemble_nlo(c.ms[0], prm).H
    assert rel_l2(c.oracle_order(c.h.nlo_apply(c.gpu(x))), H16 @ x) < 1e-13


@pytest.mark.parametrize("r,nz,L", [(0, 2, 1), (1, 128, 2)])
def test_nlo_edge_sizes(r, nz, L):
    """r0 (20 columns: four tiles, one CTA; the lowest-order level below has
    padding columns) with two layers, and 128-layer columns: operator,
    FP64 V-cycle and mixed V-cycle against the oracle."""
    c = case(r, nz, L)
    rng = np.random.default_rng(9)
    x = rng.standard_normal(c.nop.n)
    assert rel_l2(c.oracle_order(c.h.nlo_apply(c.gpu(x))), c.nop.H @ x) < 1e-13
    b = gi.nlo_rhs(c.nop.n)
    z_ref = nlo.vcycle(c.nop, c.lo, b)
    assert rel_l2(c.oracle_order(c.h.nlo_vcycle(c.gpu(b))), z_ref) < 1e-11
    assert rel_l2(c.oracle_order(c.h.nlo_vcycle(c.gpu(b), precision="mixed")), z_ref) < 1e-4


def test_nlo_single_layer_single_level():
    """One layer per column (no vertical coupling inside the column solve):
    the operator and the NLO smoother alone against the oracle."""
    c = case(0, 1, 1)
    x = np.random.default_rng(10).standard_normal(c.nop.n)
    assert rel_l2(c.oracle_order(c.h.nlo_apply(c.gpu(x))), c.nop.H @ x) < 1e-13
    b = gi.nlo_rhs(c.nop.n)
    ref = nlo.smooth(c.nop, nlo.smooth(c.nop, np.zeros(c.nop.n), b, 0.8), b, 0.8)
    assert rel_l2(c.oracle_order(c.h.nlo_vcycle(c.gpu(b), levels=1)), ref) < 1e-11
