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


@pytest.mark.parametrize("precision,krylov", [("fp64", "cg"), ("mixed", "fcg")])
def test_device_loop_matches_host_loop(precision, krylov):
    """CG iterations run as one CUDA graph with a device-side stopping test;
    a traced solve (hmg_profile_start) and a solve allowed more than 1024
    iterations take the host-side loop instead.  All three run the same
    kernels in the same order, so the iterate, the iteration count and the
    residual history agree exactly; a capped solve stops at the same place
    in both loops."""
    h = hmg.Hierarchy(3, 16, 3)
    h.assemble()
    b = torch.tensor(gi.rhs(h.ncells), dtype=torch.float64, device="cuda:0")
    x_dev, i_dev = h.solve(b, precision=precision, krylov=krylov, rtol=1e-8)
    hist_dev = h.residual_history()
    h.profile_start()
    x_host, i_host = h.solve(b, precision=precision, krylov=krylov, rtol=1e-8)
    h.profile_stop()
    hist_host = h.residual_history()
    x_long, i_long = h.solve(b, precision=precision, krylov=krylov, rtol=1e-8, max_iter=5000)
    assert i_dev["iterations"] == i_host["iterations"] == i_long["iterations"]
    hist_long = h.residual_history()
    assert np.array_equal(hist_dev, hist_host) and np.array_equal(hist_dev, hist_long)
    assert torch.equal(x_dev, x_host) and torch.equal(x_dev, x_long)
    assert i_dev["true_rel_residual"] == i_host["true_rel_residual"]
    for k in (1, 2):
        _, a = h.solve(b, precision=precision, krylov=krylov, rtol=1e-12, max_iter=k, raise_on_failure=False)
        h.profile_start()
        _, c = h.solve(b, precision=precision, krylov=krylov, rtol=1e-12, max_iter=k, raise_on_failure=False)
        h.profile_stop()
        assert a["iterations"] == c["iterations"] == k and a["converged"] == c["converged"] == 0
        assert a["rel_residual"] == c["rel_residual"]
    h.close()
