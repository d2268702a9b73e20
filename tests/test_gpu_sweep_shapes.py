"""The FP64 sweeps of levels with more tiles than the small-level threshold
(the half-column sweep, two warps per tile, one per half of the column
factorisation twisted at n_z/2) on short and odd columns, against the oracle.

At r5 (640 tiles) the level takes the four-rows-per-batch variant, at r6
(2,560 tiles) the one-row variant; the coarser levels take the twisted tile
sweep.  Layer counts 1, 2 and 3 leave one or both halves of the column
without rows (the twist row is then the only row, or the last one), and 7 is
an odd split.  Tolerances are those of the other FP64 parity tests: a
fixed-iteration V-cycle at 1e-12, a PCG solve at 1e-9 with the iteration
count within 1.
"""
import pytest

import hmg_inputs as gi
from oracle import krylov, multigrid
from tests.helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from tests.test_gpu_parity import case  # noqa: E402


@pytest.mark.parametrize("r,nz,L", [(5, 1, 2), (5, 2, 2), (5, 3, 3), (5, 7, 2), (6, 3, 2)])
def test_vcycle_short_columns(r, nz, L):
    c = case(r, nz, L)
    b = gi.rhs(c.ops[0].ncells)
    z_ref = multigrid.vcycle(c.ops, b)
    z = c.h.vcycle(c.gpu(b))
    assert rel_l2(c.host(z), z_ref[c.idx[0]]) < 1e-12
    # the first relaxation alone (one pre-sweep from zero) exercises the
    # sweep from u = 0 without the later sweeps on top
    z1_ref = multigrid.vcycle(c.ops, b, nu_pre=1, nu_post=1, n_coarse=1)
    z1 = c.h.vcycle(c.gpu(b), nu_pre=1, nu_post=1, n_coarse=1)
    assert rel_l2(c.host(z1), z1_ref[c.idx[0]]) < 1e-12


@pytest.mark.parametrize("r,nz,L", [(5, 3, 3), (5, 7, 2)])
def test_solve_short_columns(r, nz, L):
    """PCG with the fused r.z of the last sweep on a half-column level."""
    c = case(r, nz, L)
    b = gi.rhs(c.ops[0].ncells)
    x_ref, info_ref = krylov.pcg(c.ops[0].H.dot, lambda v: multigrid.vcycle(c.ops, v), b, rtol=1e-8)
    x, info = c.h.solve(c.gpu(b), rtol=1e-8)
    assert info["converged"] == 1
    assert abs(info["iterations"] - info_ref.iterations) <= 1, (info, info_ref.iterations)
    assert rel_l2(c.host(x), x_ref[c.idx[0]]) <= 1e-9
