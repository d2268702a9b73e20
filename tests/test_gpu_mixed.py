"""GPU parity of the velocity-pressure system (Eq. PressureVelocitySystem)
and its GMRES(30) solve with the Schur-complement preconditioner (Eq.
SchurComplement) against the oracle (oracle/mixed.py).

Columns are matched by centroid as in test_gpu_parity; edges by the matched
column pair, with the flux sign flipped where the two sides orient an edge
differently.  Tolerances: operator 1e-13 relative L2 per block; solves 1e-9
per block with the iteration count within 1.
"""
import numpy as np
import pytest

import hmg_inputs as gi
from oracle import helmholtz, krylov, mesh, mixed
from tests.helpers import column_permutation, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1605_00492_gb300 as hmg  # noqa: E402

DEV = "cuda:0"


class MixedCase:
    def __init__(self, r, nz, L):
        self.ms = mesh.hierarchy(r, L)
        self.prm = helmholtz.Params(refinement=r, nlayers=nz)
        self.ops = helmholtz.assemble_hierarchy(self.ms, self.prm)
        self.mop = mixed.assemble_mixed(self.ms[0], self.prm)
        self.h = hmg.Hierarchy(r, nz, L)
        self.h.assemble()
        m = self.ms[0]
        cen, _ = self.h.export_mesh(0)
        perm = column_permutation(cen, m.centroid)
        nc = m.ncols
        # oracle edge of each (oracle) column pair
        oe = helmholtz.horizontal_faces(m)
        index = {(int(t), int(tn)): e for e, (t, _, tn, _) in enumerate(oe)}
        ge = self.h.export_edges()
        assert ge.shape[0] == oe.shape[0]
        self.eidx = np.empty(ge.shape[0], dtype=np.int64)
        self.esign = np.empty(ge.shape[0])
        for e, (t, _, tn, _) in enumerate(ge):
            a, b = int(perm[t]), int(perm[tn])
            self.eidx[e] = index[(min(a, b), max(a, b))]
            self.esign[e] = 1.0 if a < b else -1.0
        lay = np.arange(nz)
        self.hidx = (self.eidx[:, None] * nz + lay[None, :]).reshape(-1)
        self.hsign = np.repeat(self.esign, nz)
        self.vidx = (perm[:, None] * (nz - 1) + np.arange(nz - 1)[None, :]).reshape(-1)
        self.cidx = (perm[:, None] * nz + lay[None, :]).reshape(-1)
        self.nhf, self.nvf, self.nc3 = self.mop.nhf, self.mop.nvf, nc * nz
        assert self.h.mixed_sizes() == (self.nhf, self.nvf, self.nc3)

    def to_gpu(self, x):
        """Oracle vector (U_h, U_z, P) -> GPU (u, p) tensors."""
        uh = x[:self.nhf][self.hidx] * self.hsign
        uz = x[self.nhf:self.nhf + self.nvf][self.vidx]
        p = x[self.nhf + self.nvf:][self.cidx]
        t = lambda v: torch.tensor(v, dtype=torch.float64, device=DEV)
        return t(np.concatenate([uh, uz])), t(p)

    def to_oracle(self, u, p):
        u = u.cpu().numpy()
        p = p.cpu().numpy()
        x = np.empty(self.nhf + self.nvf + self.nc3)
        x[self.hidx] = u[:self.nhf] * self.hsign
        x[self.nhf + self.vidx] = u[self.nhf:]
        x[self.nhf + self.nvf + self.cidx] = p
        return x


_CACHE = {}


def mcase(*a):
    if a not in _CACHE:
        _CACHE[a] = MixedCase(*a)
    return _CACHE[a]


def _blocks(c, x):
    nu = c.nhf + c.nvf
    return x[:c.nhf], x[c.nhf:nu], x[nu:]


@pytest.mark.parametrize("r,nz,L", [(2, 6, 2), (3, 16, 3), (1, 4, 1)])
def test_mixed_operator_matches_oracle(r, nz, L):
    c = mcase(r, nz, L)
    x = np.random.default_rng(11).standard_normal(c.mop.n)
    y_ref = mixed.apply_mixed(c.mop, x)
    u, p = c.to_gpu(x)
    yu, yp = c.h.mixed_apply(u, p)
    y = c.to_oracle(yu, yp)
    for got, ref in zip(_blocks(c, y), _blocks(c, y_ref)):
        assert rel_l2(got, ref) < 1e-13


@pytest.mark.parametrize("rtol,orth", [(1e-5, 1), (1e-9, 1), (1e-9, 2)])
def test_mixed_solve_matches_oracle(rtol, orth):
    c = mcase(3, 16, 3)
    b = mixed.assembled_rhs(c.mop, gi.mixed_rhs(c.mop.nu, c.mop.M3.size))
    x_ref, info_ref = krylov.fgmres(lambda v: mixed.apply_mixed(c.mop, v),
                                    lambda v: mixed.schur_precondition(c.mop, c.ops, v), b, rtol=rtol, restart=30)
    bu, bp = c.to_gpu(b)
    u, p, info = c.h.mixed_solve(bu, bp, rtol=rtol, restart=30, orth=orth)
    assert info["converged"] == 1
    assert abs(info["iterations"] - info_ref.iterations) <= 1, (info, info_ref.iterations)
    assert info["true_rel_residual"] < 2 * rtol
    x = c.to_oracle(u, p)
    tol = 1e-9 if rtol < 1e-8 else 1e-6
    for got, ref in zip(_blocks(c, x), _blocks(c, x_ref)):
        assert rel_l2(got, ref) < tol


def test_mixed_solve_mixed_precision_cycle_and_status():
    c = mcase(3, 16, 3)
    b = mixed.assembled_rhs(c.mop, gi.mixed_rhs(c.mop.nu, c.mop.M3.size))
    import scipy.sparse.linalg as spla
    x_direct = spla.spsolve(c.mop.A.tocsc(), b)
    bu, bp = c.to_gpu(b)
    u, p, info = c.h.mixed_solve(bu, bp, rtol=1e-8, precision="mixed")
    assert info["converged"] == 1 and info["true_rel_residual"] < 2e-8
    x = c.to_oracle(u, p)
    for got, ref in zip(_blocks(c, x), _blocks(c, x_direct)):
        assert rel_l2(got, ref) < 1e-6
    _, _, info = c.h.mixed_solve(bu, bp, rtol=1e-12, max_iter=2, raise_on_failure=False)
    assert info["status"] == "HMG_ERR_NOT_CONVERGED" and info["iterations"] == 2
    with pytest.raises(hmg.HMGError):
        c.h.mixed_solve(bu, bp, restart=0)
