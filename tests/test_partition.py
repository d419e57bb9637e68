"""The mode-1 partition of the multi-GPU path on the CPU: the host logic (data split, the
whole problem's row counts, the all-reduce) with the FP64 oracle as each part's gradient
engine.  Each part's gradient, with the whole problem's counts, summed over the parts is
the whole problem's gradient (Eq. (8) summed over every entry); the step every process then
applies is the single-process minibatch rule with one batch holding the whole epoch.  The
two-process case runs as world_size-2 gloo groups over 127.0.0.1."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1708_08640_gb300 import partition
from tests.oracle_cases import random_problem

HP = dict(lr0=0.05, mu=0.0, lambda_reg=0.3, lambda_m=1.7, core_scale=2.0, batch=1)


def _problem():
    prob, params = random_problem((12, 9, 7), (3, 2, 3), nnz=160, n_coupled=2, seed=31,
                                  coupled_nnz=40)
    return prob, params


def _part_gradient(prob, params, world, rank):
    part, _ = partition.mode1_part(prob, world, rank)
    counts, nnz_total = partition.whole_counts(prob)
    o = oracle.Oracle(part, counts=counts, nnz_total=nnz_total, **HP)
    o.set_params(*params)
    return o.full_gradient(), part


@pytest.mark.parametrize("world", [2, 3])
def test_parts_cover_every_item_once(world):
    prob, _ = _problem()
    parts = [partition.mode1_part(prob, world, r)[0] for r in range(world)]
    assert sum(p.train_val.shape[0] for p in parts) == prob.train_val.shape[0]
    for m in range(len(prob.coupled)):
        assert sum(p.coupled[m].rows.shape[0] for p in parts) == prob.coupled[m].rows.shape[0]
    # mode-1 rows are disjoint across the parts, and mode-1 coupled entries follow their row
    ranges = [partition.mode1_part(prob, world, r)[1] for r in range(world)]
    for (lo, hi), p in zip(ranges, parts):
        assert np.all((p.train_idx[0] >= lo) & (p.train_idx[0] < hi))
        for c in p.coupled:
            if c.mode == 0:
                assert np.all((c.rows >= lo) & (c.rows < hi))


@pytest.mark.parametrize("world", [2, 3])
def test_sum_of_part_gradients_is_the_whole_gradient(world):
    prob, params = _problem()
    whole = oracle.Oracle(prob, **HP)
    whole.set_params(*params)
    gG, gU, gV = whole.full_gradient()
    sG, sU, sV = np.zeros_like(gG), [np.zeros_like(u) for u in gU], [np.zeros_like(v) for v in gV]
    for r in range(world):
        (pG, pU, pV), _ = _part_gradient(prob, params, world, r)
        sG += pG
        for a, b in zip(sU, pU):
            a += b
        for a, b in zip(sV, pV):
            a += b
    np.testing.assert_allclose(sG, gG, rtol=1e-12, atol=1e-12)
    for a, b in zip(sU, gU):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)
    for a, b in zip(sV, gV):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob, params = _problem()
    (pG, pU, pV), _ = _part_gradient(prob, params, world, rank)
    ts = [torch.from_numpy(np.ascontiguousarray(a)) for a in [pG, *pU, *pV]]
    partition.allreduce_sum(ts)
    q.put((rank, [t.numpy() for t in ts]))
    dist.barrier()
    dist.destroy_process_group()


def test_partitioned_epoch_equals_the_full_batch_minibatch_rule_with_gloo():
    """Two processes (gloo): each part's gradient, summed by partition.allreduce_sum, is the
    whole gradient on both; the step of the minibatch rule taken from it (rows -eta sum,
    core -eta core_scale mean over the tensor entries) is the oracle's minibatch epoch with
    one batch of every item."""
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    prob, params = _problem()
    whole = oracle.Oracle(prob, **HP)
    whole.set_params(*params)
    gG, gU, gV = whole.full_gradient()
    ref = [gG, *gU, *gV]
    for rank in range(world):
        for a, b in zip(out[rank], ref):
            np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)
    # the step every process applies, against the single-process rule
    G0, U0, V0 = params
    eta = HP["lr0"]
    n_t = prob.train_val.shape[0]
    stepped = [G0 - eta * HP["core_scale"] * gG / n_t, *[u - eta * g for u, g in zip(U0, gU)],
               *[v - eta * g for v, g in zip(V0, gV)]]
    n_union = n_t + sum(c.rows.shape[0] for c in prob.coupled)
    whole.epoch_minibatch(0, np.arange(n_union), batch=n_union)
    G1, U1, V1 = whole.get_params()
    for a, b in zip(stepped, [G1, *U1, *V1]):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)
