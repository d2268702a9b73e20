"""The horizontal domain decomposition's host logic (Sec. 5: domain split
over processes, halo exchange before each parallel loop, Krylov dot products
reduced over processes): the library's partition tables (hmg_partition_*)
checked against the unpartitioned neighbour table, and the halo exchange and
scalar reduction of paper_1605_00492_gb300.distributed run by two gloo ranks
on the CPU.  No GPU is used."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
hmg = pytest.importorskip("paper_1605_00492_gb300")

CASES = [(3, 3, 2), (3, 3, 4), (3, 3, 10), (4, 4, 3), (2, 1, 2), (2, 2, 3), (5, 5, 7)]


def _global_nbr(r, L, level):
    """The unpartitioned table: one part owns everything and has no ghosts."""
    t = hmg.partition_tables(r, L, 1, 0, level)
    assert t["col_begin"] == 0 and len(t["ghost_col"]) == 0 and len(t["send_col"]) == 0
    return t["local_nbr"]


@pytest.mark.parametrize("r,L,K", CASES)
def test_partition_tables(r, L, K):
    P = L - 1 if L > 1 else 1
    prev = None
    for level in range(P):
        nbr = _global_nbr(r, L, level)
        nc = len(nbr)
        assert nc == 20 * 4 ** (r - level)
        # the unpartitioned table is a valid adjacency: 3 distinct neighbours, symmetric
        assert np.all(nbr != np.arange(nc)[:, None])
        assert np.all(np.sort(nbr, axis=1)[:, 1:] != np.sort(nbr, axis=1)[:, :-1])
        assert all(c in nbr[n] for c in range(nc) for n in nbr[c])
        parts = [hmg.partition_tables(r, L, K, p, level) for p in range(K)]
        # owned ranges tile the level in order
        assert parts[0]["col_begin"] == 0 and parts[-1]["col_end"] == nc
        for a, b in zip(parts, parts[1:]):
            assert a["col_end"] == b["col_begin"]
        if prev is not None:   # coarse levels inherit the partition: children 4C..4C+3 stay with C
            for p in range(K):
                assert parts[p]["col_begin"] * 4 == prev[p]["col_begin"]
                assert parts[p]["col_end"] * 4 == prev[p]["col_end"]
        for p, t in enumerate(parts):
            b0, e0, npad = t["col_begin"], t["col_end"], t["ncols_padded"]
            assert npad % 32 == 0 and e0 - b0 <= npad < e0 - b0 + 32
            assert b0 % 32 == 0    # whole tiles of the level
            # local neighbours map back to the global table
            loc = t["local_nbr"]
            glob = np.where(loc < npad, loc + b0, t["ghost_col"][np.clip(loc - npad, 0, None)]
                            if len(t["ghost_col"]) else loc + b0)
            assert np.array_equal(glob, nbr[b0:e0])
            # ghosts: outside the range, unique, sorted by (owner, column), owners right
            g, go, gl = t["ghost_col"], t["ghost_owner"], t["ghost_owner_local"]
            assert np.all((g < b0) | (g >= e0))
            assert len(np.unique(g)) == len(g)
            assert np.all(np.lexsort((g, go)) == np.arange(len(g)))
            for col, q, j in zip(g, go, gl):
                assert parts[q]["col_begin"] <= col < parts[q]["col_end"]
                assert j == col - parts[q]["col_begin"]
            # every ghost is some owned column's neighbour
            assert set(g.tolist()) == set(nbr[b0:e0].ravel().tolist()) - set(range(b0, e0))
        # send lists match the receivers' ghost lists, in order
        for p, t in enumerate(parts):
            for q in range(K):
                want = parts[q]["ghost_col"][parts[q]["ghost_owner"] == p] if q != p else np.zeros(0, np.int32)
                assert np.array_equal(t["send_col"][t["send_to"] == q], want)
            assert np.all(np.diff(t["send_to"]) >= 0)
        prev = parts


def test_partition_rejects_bad_arguments():
    with pytest.raises(hmg.HMGError):
        hmg.partition_tables(2, 2, 11, 0, 0)     # level 0 of refinement 2: 320 columns = 10 tiles < 11 parts
    with pytest.raises(hmg.HMGError):
        hmg.partition_tables(3, 3, 2, 2, 0)      # part out of range
    with pytest.raises(hmg.HMGError):
        hmg.partition_tables(3, 3, 2, 0, 2)      # the coarsest level is not partitioned
    with pytest.raises(hmg.HMGError):
        hmg.partition_tables(1, 2, 4, 0, 0)      # 80 columns = 3 tiles < 4 parts


def _rank_main(rank, world, port, r, L, nz, out):
    import torch.distributed as dist

    from paper_1605_00492_gb300.distributed import HaloPlan, allreduce_sum, exchange_halo
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = []
        for level in range(max(1, L - 1)):
            plan = HaloPlan(r, L, world, rank, level)
            nc = 20 * 4 ** (r - level)
            rng = np.random.default_rng(100 + level)        # the same global fields on every rank
            F = torch.tensor(rng.standard_normal((nc, nz)))
            G = torch.tensor(rng.standard_normal((nc, nz)))
            owned = F[plan.col_begin:plan.col_end].clone()
            ghosts = torch.full((plan.n_ghost, nz), float("nan"), dtype=torch.float64)
            exchange_halo(plan, owned, ghosts)
            ok_halo = bool(torch.equal(ghosts, F[torch.as_tensor(plan.ghost_col, dtype=torch.int64)]))
            part = torch.tensor([float(torch.sum(owned * G[plan.col_begin:plan.col_end])), float(owned.numel())],
                                dtype=torch.float64)
            allreduce_sum(part)
            full = float(torch.sum(F * G))
            res.append((level, ok_halo, abs(float(part[0]) - full) / abs(full), float(part[1]) == F.numel()))
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,r,L", [(2, 3, 3), (3, 4, 3)])
def test_halo_exchange_and_scalar_reduction_gloo(world, r, L):
    ctx = mp.get_context("spawn")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(k, world, port, r, L, 5, q)) for k in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert sorted(res) == list(range(world))
    for rank, rows in res.items():
        assert len(rows) == max(1, L - 1)
        for level, ok_halo, rel, count_ok in rows:
            assert ok_halo, (rank, level)
            assert rel < 1e-13 and count_ok
