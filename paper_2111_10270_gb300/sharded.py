"""One instance split over several ranks (one process and one GPU per rank).

Host side of the library's shard calls (fdog_shard_* in fastdog.h): the
rows are split into blocks by their smallest variable (fdog_shard_plan),
each rank builds an ordinary instance of its block's rows, and every pass of
Alg. 1 ends with an
all-reduce of one float per variable whose copies lie in several shards (the
partial sums of its multipliers, from which each shard forms the deferred
term of Eq. 5), every iteration with an all-reduce of the lower bound.  The
kernels and the sums run in the library; this module slices the ILP and
moves the exchanged buffers through ``torch.distributed``: in place on the
device with NCCL, through host memory with any other backend (gloo).
"""
from __future__ import annotations

import numpy as np

from . import capi


def shard_rows(ilp, row_shard, copies, rank: int):
    """The ILP a rank builds: every variable, the rows of its block, and the
    cost of a variable only where some row of the block holds it (its target
    of Prop. 1), or on rank 0 for a variable no row holds.  Returns
    (n_vars, cost, row_ptr, col, coef, sense, rhs, rows) with rows the
    original indices of the block's rows."""
    rows = np.nonzero(np.asarray(row_shard) == rank)[0]
    rp = np.asarray(ilp.row_ptr, np.int64)
    lens = rp[rows + 1] - rp[rows]
    row_ptr = np.zeros(len(rows) + 1, np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    take = np.concatenate([np.arange(rp[j], rp[j + 1]) for j in rows]) if len(rows) else np.zeros(0, np.int64)
    col = np.asarray(ilp.col, np.int32)[take]
    coef = np.asarray(ilp.coef, np.int32)[take]
    held = np.zeros(ilp.n_vars, bool)
    held[col[coef != 0]] = True
    if rank == 0:
        held |= np.asarray(copies) == 0
    cost = np.where(held, np.asarray(ilp.cost, np.float64), 0.0)
    return (ilp.n_vars, cost, row_ptr, col, coef, np.asarray(ilp.sense, np.int8)[rows],
            np.asarray(ilp.rhs, np.int64)[rows], rows)


def allreduce_sum(t, group=None):
    """Sum of `t` over the group's ranks, in place; device tensors go through
    host memory unless the backend is NCCL."""
    import torch.distributed as dist

    if t.is_cuda and dist.get_backend(group) != "nccl":
        h = t.cpu()
        dist.all_reduce(h, group=group)
        t.copy_(h)
    else:
        dist.all_reduce(t, group=group)
    return t


class ShardedInstance:
    """This rank's shard of `ilp` (every rank passes the same ILP), built on
    `device` with torch's current stream of that device, so that the
    all-reduces are ordered between the library's passes."""

    def __init__(self, ilp, rank: int, world: int, device: int = 0, group=None, **params):
        import torch

        self.rank, self.world, self.device, self.group = rank, world, device, group
        self.row_shard, self.copies, self.shared = capi.shard_plan(ilp.n_vars, ilp.row_ptr, ilp.col, ilp.coef,
                                                                   world)
        n, cost, rp, col, coef, sense, rhs, self.rows = shard_rows(ilp, self.row_shard, self.copies, rank)
        self.inst = capi.Instance(n, cost, rp, col, coef, sense, rhs, **params)
        self.inst.shard_setup(self.shared, self.copies)
        self.n_shared = self.inst.shard_info()
        self.stream = torch.cuda.current_stream(device)
        self.inst.build(device, self.stream)
        self.sums = torch.zeros(max(self.n_shared, 1), dtype=torch.float32, device=f"cuda:{device}")
        self.trace = []  # the bound of the whole instance after each iteration
        self._pending = False  # iterations ran since the last finalize

    def _pass(self, descending: bool):
        ptr = self.sums.data_ptr()
        self.inst.shard_pass(descending, ptr)
        if self.n_shared > 0:
            allreduce_sum(self.sums, self.group)
            self.inst.shard_apply(ptr)

    def iterate(self, k: int):
        """Up to k iterations of Alg. 1 over all shards (every rank calls it
        with the same k); returns (iterations run, bound of the whole
        instance after the last one)."""
        import torch

        done = 0
        for _ in range(k):
            self._pass(False)
            self._pass(True)
            part = torch.tensor([self.inst.shard_bound()], dtype=torch.float64,
                                device=f"cuda:{self.device}")
            lb = float(allreduce_sum(part, self.group)[0])
            stop = self.inst.shard_commit(lb)
            self.trace.append(lb)
            done += 1
            self._pending = True
            if stop:
                break
        return done, (self.trace[-1] if self.trace else None)

    def finalize(self):
        self.inst.finalize()
        self._pending = False

    def lower_bound(self):
        """(running, feasible) bounds of the whole instance.  The feasible
        bound (and the running one at a finalised state) is each shard's FP64
        evaluation summed over the ranks; after iterations the running bound
        is the last committed one."""
        import torch

        run, fea = self.inst.lower_bound()
        parts = torch.tensor([0.0 if self._pending else run, fea], dtype=torch.float64,
                             device=f"cuda:{self.device}")
        allreduce_sum(parts, self.group)
        return (self.trace[-1] if self._pending else float(parts[0])), float(parts[1])

    def multipliers(self):
        """This shard's slots: (variable, original row, lambda)."""
        var, row, lam = self.inst.multipliers()
        return var, self.rows[row], lam

    def min_marginals(self):
        var, row, m0, m1 = self.inst.min_marginals()
        return var, self.rows[row], m0, m1

    def close(self):
        self.inst.close()
