"""Mode-1 row partition of a problem across processes (one per GPU) and the partitioned
epoch: the host side of the multi-GPU path.

Every process holds a contiguous range of mode-1 rows with the tensor entries and the
mode-1 coupled entries of those rows; coupled entries of matrices on other modes are dealt
round-robin.  G, U^(2..N) and every V are replicated; U^(1) rows are only ever changed by
their owner, so they never conflict.  A partitioned epoch is one step of the minibatch rule
whose group is the whole epoch (the sync interval): each process computes its part's share
of the whole gradient (s3_gradient, with the whole problem's row counts set by
s3_set_counts), the shares are summed by one all-reduce (the path's only exchange), and
every process applies the same step (s3_apply_gradient), which leaves identical replicas.
The result equals the single-process minibatch epoch with one batch holding every item.

The arithmetic runs in the library's kernels; this module splits the data, computes the
whole problem's row counts (integer bookkeeping) and calls torch.distributed.
"""
from __future__ import annotations

import copy

import numpy as np


def mode1_ranges(counts1, world):
    """Contiguous mode-1 row ranges [lo, hi) of about equal tensor-entry counts."""
    csum = np.concatenate([[0], np.cumsum(np.asarray(counts1, dtype=np.int64))])
    total = csum[-1]
    bounds = [0]
    for r in range(1, world):
        bounds.append(int(np.searchsorted(csum, total * r / world, side="left")))
    bounds.append(len(counts1))
    bounds = np.maximum.accumulate(np.array(bounds))
    return [(int(bounds[r]), int(bounds[r + 1])) for r in range(world)]


def whole_counts(prob):
    """The whole problem's row counts: |Omega^{n,i}| for every tensor factor row, then
    |Omega_Y^{2,k}| for every coupled factor row (int64 arrays), and |Omega|."""
    idx = np.asarray(prob.train_idx)
    counts = [np.bincount(idx[n], minlength=prob.dims[n]).astype(np.int64) for n in range(len(prob.dims))]
    counts += [np.bincount(np.asarray(c.cols), minlength=c.K).astype(np.int64) for c in prob.coupled]
    return counts, int(idx.shape[1])


def mode1_part(prob, world, rank):
    """The part of `prob` that process `rank` of `world` holds: the tensor entries whose
    mode-1 index lies in its row range, the entries of coupled matrices on mode 1 whose row
    does, and every world-th entry (from rank) of coupled matrices on other modes.  Returns
    (part, (lo, hi)); the part keeps the problem's dimensions, ranks and hyper-parameters."""
    idx = np.asarray(prob.train_idx)
    counts1 = np.bincount(idx[0], minlength=prob.dims[0])
    lo, hi = mode1_ranges(counts1, world)[rank]
    keep = (idx[0] >= lo) & (idx[0] < hi)
    part = copy.copy(prob)
    part.train_idx = idx[:, keep]
    part.train_val = np.asarray(prob.train_val)[keep]
    cpl = []
    for c in prob.coupled:
        rows = np.asarray(c.rows)
        if c.mode == 0:
            k = (rows >= lo) & (rows < hi)
        else:
            k = (np.arange(rows.shape[0]) % world) == rank
        cc = copy.copy(c)
        cc.rows, cc.cols = rows[k], np.asarray(c.cols)[k]
        cc.vals = None if c.vals is None else np.asarray(c.vals)[k]
        cpl.append(cc)
    part.coupled = cpl
    return part, (lo, hi)


def allreduce_sum(tensors, group=None):
    """Sum every tensor over the processes of the group, in place (one all-reduce each)."""
    import torch.distributed as dist
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return tensors


class PartitionedModel:
    """One process's share of a mode-1 partitioned problem on its GPU.

    prob: the whole problem (every process passes the same one); the process keeps its part.
    Every process starts from the library's seeded initial parameters (identical on all) or
    from parameters given to set_params."""

    def __init__(self, prob, world, rank, group=None, device=None, **hp):
        from .model import S3CMTF
        self.world, self.rank, self.group = world, rank, group
        part, self.rows = mode1_part(prob, world, rank)
        counts, nnz_total = whole_counts(prob)
        hp = dict(prob.hparams, **hp)
        hp["row_rule"] = "sum"
        self.model = S3CMTF.from_problem(part, device=device, **hp)
        self.model.set_counts(counts, nnz_total)
        self.nnz_total = nnz_total

    def set_params(self, G, U, V):
        self.model.set_params(G, U, V)

    def get_params(self):
        return self.model.get_params()

    def epoch(self):
        """One partitioned epoch: this part's gradient share, the all-reduce, the step."""
        dG, dU, dV = self.model.gradient()
        allreduce_sum([dG, *dU, *dV], self.group)
        self.model.apply_gradient(dG, dU, dV)

    def close(self):
        self.model.close()
