"""Halo exchange and scalar reduction between processes for the horizontal
domain decomposition (Sec. 5: the paper splits the horizontal domain over MPI
processes, exchanges the halo before each parallel loop and reduces the
Krylov dot products over processes).

The tables come from the library's host partition (hmg_partition_tables):
part p owns a contiguous range of columns on each partitioned level; its
ghosts are the columns its stencils read that other parts own, ordered by
(owner, column); its send list holds, grouped by receiver and in the
receiver's ghost order, the owned columns other parts read.  So one exchange
is: pack the send list, one send/recv pair per neighbouring part (NCCL for
CUDA tensors, gloo for CPU tensors, through torch.distributed), unpack into
the ghost rows in order.  Values are per column: a row of nz layers.
"""
import numpy as np
import torch

from . import partition_tables


class HaloPlan:
    """The exchange of one part (this rank) on one partitioned level."""

    def __init__(self, refinement, nlevels, nparts, part, level):
        t = partition_tables(refinement, nlevels, nparts, part, level)
        self.part, self.nparts = part, nparts
        self.col_begin, self.col_end = t["col_begin"], t["col_end"]
        self.ncols_padded = t["ncols_padded"]
        self.ghost_col = t["ghost_col"]
        self.local_nbr = t["local_nbr"]
        # send segments: receiver -> owned local rows, in the receiver's ghost order
        self.send = {}
        for q in np.unique(t["send_to"]):
            cols = t["send_col"][t["send_to"] == q]
            self.send[int(q)] = torch.as_tensor(cols - self.col_begin, dtype=torch.int64)
        # receive segments: owner -> ghost positions (contiguous, ghosts are grouped by owner)
        self.recv = {}
        for q in np.unique(t["ghost_owner"]):
            idx = np.nonzero(t["ghost_owner"] == q)[0]
            self.recv[int(q)] = (int(idx[0]), int(idx[-1]) + 1)

    @property
    def n_own(self):
        return self.col_end - self.col_begin

    @property
    def n_ghost(self):
        return len(self.ghost_col)


def exchange_halo(plan, owned, ghosts, group=None):
    """Fill ghosts (n_ghost, nz) from the other parts' owned rows; owned is
    this part's (n_own, nz) block.  Every rank of the group calls it with the
    plan of its own part."""
    import torch.distributed as dist
    reqs = []
    bufs = {}
    for q, (a, b) in sorted(plan.recv.items()):
        bufs[q] = torch.empty((b - a,) + tuple(owned.shape[1:]), dtype=owned.dtype, device=owned.device)
        reqs.append(dist.irecv(bufs[q], src=q, group=group))
    for q, rows in sorted(plan.send.items()):
        payload = owned.index_select(0, rows.to(owned.device)).contiguous()
        reqs.append(dist.isend(payload, dst=q, group=group))
    for r in reqs:
        r.wait()
    for q, (a, b) in plan.recv.items():
        ghosts[a:b] = bufs[q]
    return ghosts


def allreduce_sum(values, group=None):
    """Sum a small FP64 tensor of partial dot products over all parts (the
    2-3 Krylov scalars of an iteration)."""
    import torch.distributed as dist
    dist.all_reduce(values, op=dist.ReduceOp.SUM, group=group)
    return values
