"""Host-side logic of bench.py (no GPU): byte models, the oracle primitive
decomposition used by the reference arm, and max-over-ranks timing with two
gloo ranks."""
import os

import numpy as np
import pytest

import bench
import hmg_inputs as gi
from oracle import helmholtz, krylov, mesh, multigrid


def test_vcycle_primitives_reproduce_the_oracle_vcycle_bitwise():
    ms = mesh.hierarchy(3, 3)
    prm = helmholtz.Params(refinement=3, nlayers=8)
    ops = helmholtz.assemble_hierarchy(ms, prm)
    r = gi.rhs(ops[0].ncells)
    calls, u = bench.oracle_vcycle_primitives(ops, lambda: r)
    for fn in calls:
        fn()
    assert np.array_equal(u[0], multigrid.vcycle(ops, r))


def test_pcg_primitive_stream_matches_oracle_pcg():
    ms = mesh.hierarchy(2, 2)
    prm = helmholtz.Params(refinement=2, nlayers=8)
    ops = helmholtz.assemble_hierarchy(ms, prm)
    b = gi.rhs(ops[0].ncells)
    state = {}
    stream = bench.oracle_pcg_primitives(ops, b, state)
    _, P, fn = next(stream)
    fn()
    for _ in range(3 * P - 1):
        _, _, fn = next(stream)
        fn()
    x3, info = krylov.pcg(ops[0].H.dot, lambda v: multigrid.vcycle(ops, v), b, rtol=1e-30, max_iter=3)
    assert info.iterations == 3
    assert np.array_equal(state["x"], x3)


def test_vcycle_byte_model_paper_scale():
    nz = 64
    lv = [81920 * 64 // 4 ** k for k in range(5)]
    fp64 = bench.vcycle_bytes(lv, nz, mixed=False)
    mixed = bench.vcycle_bytes(lv, nz, mixed=True)
    # finest-level sweep: b, u, lo, w read, u' written, plus per-column data
    assert bench.kernel_bytes_per_cell("sweep", 8, 64) == pytest.approx(40 + 48 / 64)
    assert 1.3e9 < fp64 < 1.6e9
    assert 0.45 < mixed / fp64 < 0.55


def _ranks_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    v = bench.max_over_ranks(10.0 + rank, world, "cpu")
    bench.barrier(world)
    out.put((rank, v))
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    import multiprocessing as mp
    import socket
    ctx = mp.get_context("spawn")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    q = ctx.Queue()
    procs = [ctx.Process(target=_ranks_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert res == {0: 11.0, 1: 11.0}


def test_useful_bandwidth_from_a_breakdown():
    """Model bytes and FP64 flops of each kernel class over its traced time."""
    br = {("sweep", 0): (3, 0.3), ("apply", 0): (1, 0.08), ("dot", 0): (1, 0.02), ("sweep0", 1): (2, 0.04)}
    cells = [5_242_880, 1_310_720]
    ub = bench.useful_bandwidth(br, cells, 64, 6795.5)
    assert set(ub) == {"sweep@0", "apply@0", "sweep0@1"}          # kernels without a byte model are left out
    per_cell = bench.kernel_bytes_per_cell("sweep", 8, 64)
    assert ub["sweep@0"]["GB_s"] == pytest.approx(per_cell * cells[0] * 3 / 0.3e-3 / 1e9, rel=1e-3)
    assert ub["sweep@0"]["us_per_launch"] == pytest.approx(100.0)
    assert ub["apply@0"]["TFLOP_s"] == pytest.approx(11 * cells[0] / 0.08e-3 / 1e12, rel=1e-3)
    assert 0 < ub["sweep0@1"]["frac_hbm"] < 1


def test_cpu_baseline_runs_one_oracle_copy_per_core():
    """The CPU baseline runs single-threaded copies of the oracle side by
    side and sums their solves/s; each copy times the same bounded sample."""
    d = bench.cpu_baseline_subprocess("r3x16", 1, copies=2)
    assert d["kind"] == "oracle" and d["cores"] == 2 and d["unit"] == bench.UNIT
    lo, hi = d["seconds_per_solve_min_max"]
    assert 0 < lo <= hi
    assert 2 / hi - 1e-9 <= d["value"] <= 2 / lo + 1e-9
