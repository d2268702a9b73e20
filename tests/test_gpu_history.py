"""The convergence history of the last solve (hmg_residual_history): one
relative residual per iteration, the last equal to the solve's reported
residual, and each equal to the residual a solve stopped after that many
iterations reports (CG from x = 0 is deterministic); the same for GMRES."""
import numpy as np
import pytest

import hmg_inputs as gi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1605_00492_gb300 as hmg  # noqa: E402


@pytest.mark.parametrize("krylov", ["cg", "gmres"])
def test_residual_history(krylov):
    h = hmg.Hierarchy(3, 16, 3)
    h.assemble()
    b = torch.tensor(gi.rhs(h.ncells), dtype=torch.float64, device="cuda:0")
    _, info = h.solve(b, krylov=krylov, rtol=1e-8)
    hist = h.residual_history()
    assert len(hist) == info["iterations"]
    assert hist[-1] == info["rel_residual"] and hist[-1] < 1e-8 <= hist[-2]
    assert hist[0] > hist[-1]
    for k in (1, 3):
        _, ik = h.solve(b, krylov=krylov, rtol=1e-12, max_iter=k, raise_on_failure=False)
        assert ik["iterations"] == k and len(h.residual_history()) == k
        assert ik["rel_residual"] == pytest.approx(hist[k - 1], rel=1e-12)
    h.close()
