"""The horizontal domain decomposition (Sec. 5: the domain split over
processes, a halo exchange before each parallel loop, the coarsest level on
one process, the Krylov dot products reduced over processes), emulated on
one GPU with K = 2, 3 and 4 parts (hmg_partition), against the same context
unpartitioned.  Each part runs the unpartitioned kernels on its own columns
and reads its neighbours' columns only from its exchanged ghosts, so the
operator and the V-cycle agree to rounding (1e-14 and 1e-12 in FP64, 1e-6 in
the FP32 form) and the solves to the Krylov tolerance (1e-9, iterations within
1).  The multi-process exchange itself is tested on the CPU
(test_partition_host.py)."""
import pytest

import hmg_inputs as gi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1605_00492_gb300 as hmg  # noqa: E402


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


# (6, 8, 3, K): parts of more than 160 tiles take the half-column sweep; with
# K = 3 the level-1 parts hold 213 and 214 tiles (odd tile counts)
@pytest.mark.parametrize("r,nz,L,K", [(3, 16, 3, 2), (3, 16, 3, 4), (4, 64, 4, 3), (5, 64, 5, 4), (2, 8, 2, 10),
                                      (4, 128, 3, 2), (6, 8, 3, 2), (6, 8, 3, 3)])
def test_partitioned_operator_and_vcycle(r, nz, L, K):
    h = hmg.Hierarchy(r, nz, L)
    h.assemble()
    n = h.ncells
    x = torch.tensor(gi.rhs(n, seed=7), dtype=torch.float64, device="cuda:0")
    b = torch.tensor(gi.rhs(n), dtype=torch.float64, device="cuda:0")
    ref = {"apply": h.apply(x), "fp64": h.vcycle(b), "mixed": h.vcycle(b, precision="mixed"),
           "nu1": h.vcycle(b, nu_pre=1, nu_post=1, n_coarse=1)}
    h.partition(K)
    assert _rel(h.apply(x), ref["apply"]) <= 1e-14
    assert _rel(h.vcycle(b), ref["fp64"]) <= 1e-12
    assert _rel(h.vcycle(b, precision="mixed"), ref["mixed"]) <= 1e-6
    assert _rel(h.vcycle(b, nu_pre=1, nu_post=1, n_coarse=1), ref["nu1"]) <= 1e-12
    h.partition(1)
    assert torch.equal(h.vcycle(b), ref["fp64"])
    h.close()


@pytest.mark.parametrize("K", [2, 4])
@pytest.mark.parametrize("precision,krylov", [("fp64", "cg"), ("mixed", "fcg"), ("fp64", "gmres")])
def test_partitioned_solve(K, precision, krylov):
    h = hmg.Hierarchy(4, 64, 4)
    h.assemble()
    b = torch.tensor(gi.rhs(h.ncells), dtype=torch.float64, device="cuda:0")
    kw = dict(precision=precision, krylov=krylov, rtol=1e-8)
    x0, i0 = h.solve(b, **kw)
    h.partition(K)
    x1, i1 = h.solve(b, **kw)
    assert i1["converged"] == 1 and abs(i1["iterations"] - i0["iterations"]) <= 1
    assert i1["true_rel_residual"] < 2e-8
    assert _rel(x1, x0) <= 1e-9
    h.close()


def test_partitioned_single_level_method():
    h = hmg.Hierarchy(3, 16, 3)
    h.assemble()
    b = torch.tensor(gi.rhs(h.ncells), dtype=torch.float64, device="cuda:0")
    x0, i0 = h.solve(b, levels=1, rtol=1e-8, max_iter=1000)
    h.partition(3)
    x1, i1 = h.solve(b, levels=1, rtol=1e-8, max_iter=1000)
    assert abs(i1["iterations"] - i0["iterations"]) <= 1 and _rel(x1, x0) <= 1e-9
    h.close()


def test_partition_rejects_too_many_parts():
    h = hmg.Hierarchy(3, 16, 3)           # level 1: 320 columns = 10 tiles
    h.assemble()
    with pytest.raises(hmg.HMGError) as e:
        h.partition(11)
    assert e.value.name == "HMG_ERR_INVALID_ARG"
    with pytest.raises(hmg.HMGError):
        h.partition(17)
    h.close()


def test_halo_exchange_is_traced():
    h = hmg.Hierarchy(3, 16, 3)
    h.assemble()
    h.partition(2)
    b = torch.tensor(gi.rhs(h.ncells), dtype=torch.float64, device="cuda:0")
    h.profile_start()
    h.vcycle(b)
    rec = h.profile_stop()
    # level 0: one exchange before the second pre-sweep, the residual and each
    # of the two post-sweeps, each a pack and an unpack launch
    assert rec[("halo", 0)][0] == 8
    assert rec[("sweep0", 0)][0] == 2 and rec[("sweep", 0)][0] == 2 * 3
    h.close()
