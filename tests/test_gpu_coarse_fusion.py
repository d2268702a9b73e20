"""The fused coarse end of the V-cycle (one cooperative kernel from the first
level below the finest with at most 160 tiles down to the coarsest and back,
Algorithm 1) against the same cycle run as one kernel per pass
(hmg_set_coarse_fusion).  Both evaluate the same sweeps and residuals in the
same order, so V-cycles and solves agree exactly; the oracle comparisons of
the other GPU tests run with the separate kernels, the default."""
import numpy as np
import pytest

import hmg_inputs as gi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1605_00492_gb300 as hmg  # noqa: E402


def _both(h, fn):
    h.set_coarse_fusion(False)
    a = fn()
    h.set_coarse_fusion(True)
    b = fn()
    return a, b


@pytest.mark.parametrize("r,nz,L", [(3, 16, 3), (2, 8, 2), (4, 64, 4), (5, 128, 5), (3, 5, 4), (1, 3, 2)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nu", [(2, 2, 2), (1, 1, 1), (1, 3, 2), (2, 1, 3)])
def test_fused_vcycle_is_identical(r, nz, L, precision, nu):
    h = hmg.Hierarchy(r, nz, L)
    h.assemble()
    b = torch.tensor(gi.rhs(h.ncells), dtype=torch.float64, device="cuda:0")
    kw = dict(precision=precision, nu_pre=nu[0], nu_post=nu[1], n_coarse=nu[2])
    z0, z1 = _both(h, lambda: h.vcycle(b, **kw))
    assert torch.equal(z0, z1)
    h.close()


@pytest.mark.parametrize("precision,krylov", [("fp64", "cg"), ("mixed", "fcg"), ("fp64", "gmres")])
def test_fused_solve_is_identical(precision, krylov):
    h = hmg.Hierarchy(4, 64, 4)
    h.assemble()
    b = torch.tensor(gi.rhs(h.ncells), dtype=torch.float64, device="cuda:0")
    (x0, i0), (x1, i1) = _both(h, lambda: h.solve(b, precision=precision, krylov=krylov, rtol=1e-8))
    assert i0["iterations"] == i1["iterations"] and i1["converged"] == 1
    assert torch.equal(x0, x1)
    h.close()


def test_fused_nlo_vcycle_is_identical():
    """The NLO V-cycle continues on the lowest-order hierarchy, whose coarse
    end is fused the same way."""
    h = hmg.Hierarchy(3, 8, 3)
    h.assemble()
    n = h.nlo_size()
    b = torch.tensor(gi.nlo_rhs(n), dtype=torch.float64, device="cuda:0")
    for precision in ("fp64", "mixed"):
        z0, z1 = _both(h, lambda: h.nlo_vcycle(b, precision=precision))
        assert torch.equal(z0, z1)
    h.close()


def test_fused_kernel_is_traced_as_one_launch():
    h = hmg.Hierarchy(4, 16, 4)
    h.assemble()
    h.set_coarse_fusion(True)
    b = torch.tensor(gi.rhs(h.ncells), dtype=torch.float64, device="cuda:0")
    h.profile_start()
    h.vcycle(b)
    rec = h.profile_stop()
    # level 1 (refinement 3: 1,280 columns, 40 tiles) is the first fused level
    assert rec[("coarse_cycle", 1)][0] == 1
    assert not any(lev >= 1 and k in ("sweep", "sweep0", "resid_restrict") for (k, lev) in rec)
    h.close()
