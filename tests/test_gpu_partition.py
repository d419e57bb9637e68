"""The mode-1 partitioned epoch through the C ABI on one GPU: the parts of a problem as
separate contexts (run one after another: no kernel of one waits for another), each with the
whole problem's row counts (s3_set_counts).  Their gradient shares summed (the all-reduce of
the multi-GPU path, done here by the test) are the whole gradient, and the step every part
applies from it (s3_apply_gradient) equals the single-context minibatch epoch with one batch
of every item, leaving bit-identical replicas.  Tolerance 1e-5 relative (FP32, compensated
sums), as in the other parity tests."""
import numpy as np
import pytest
import torch

import oracle
from paper_1708_08640_gb300 import partition, synth
from tests.gpu_common import assert_close_blocks, assert_step_close, fp32_params, fp32_problem

pytestmark = pytest.mark.gpu


def as_np(t):
    return t.detach().cpu().double().numpy()


@pytest.mark.parametrize("name,world", [("cfg1_tiny", 2), ("cfg3_tiny", 3)])
def test_partitioned_epoch_matches_full_batch_minibatch(cuda_lib, name, world):
    from paper_1708_08640_gb300.model import S3CMTF
    p = fp32_problem(synth.make_problem(name))
    params = fp32_params(synth.init_params(p, 1))
    counts, nnz_total = partition.whole_counts(p)
    hp = dict(p.hparams, row_rule="sum")
    parts = []
    for r in range(world):
        part, _ = partition.mode1_part(p, world, r)
        m = S3CMTF.from_problem(part, **hp)
        m.set_counts(counts, nnz_total)
        m.set_params(*params)
        parts.append(m)
    grads = [m.gradient() for m in parts]
    dG = sum(g[0] for g in grads)
    dU = [sum(g[1][n] for g in grads) for n in range(p.N)]
    dV = [sum(g[2][k] for g in grads) for k in range(len(p.coupled))]
    # the whole gradient, from the oracle over every entry
    orc = oracle.Oracle(p, **{k: v for k, v in hp.items()
                             if k in ("lr0", "mu", "lambda_reg", "lambda_m", "core_scale")})
    orc.set_params(*params)
    gG, gU, gV = orc.full_gradient()
    assert_close_blocks(as_np(dG), gG, 1e-5, 1e-6, "summed dG")
    for n in range(p.N):
        assert_close_blocks(as_np(dU[n]), gU[n], 1e-5, 1e-6, f"summed dU{n}")
    for k in range(len(p.coupled)):
        assert_close_blocks(as_np(dV[k]), gV[k], 1e-5, 1e-6, f"summed dV{k}")
    for m in parts:
        m.apply_gradient(dG, dU, dV)
    after = [m.get_params() for m in parts]
    for other in after[1:]:            # identical replicas
        assert torch.equal(other[0], after[0][0])
        assert all(torch.equal(x, y) for x, y in zip(other[1], after[0][1]))
        assert all(torch.equal(x, y) for x, y in zip(other[2], after[0][2]))
    # the single-process minibatch rule with one batch holding every item
    n_union = p.nnz + sum(c.nnz for c in p.coupled)
    orc.epoch_minibatch(0, np.arange(n_union), batch=n_union)
    G0, U0, V0 = params
    G1, U1, V1 = after[0]
    assert_step_close(as_np(G1), orc.G, G0, 1e-5, "G step")
    for n in range(p.N):
        assert_step_close(as_np(U1[n]), orc.U[n], U0[n], 1e-5, f"U{n} step")
    for k in range(len(p.coupled)):
        assert_step_close(as_np(V1[k]), orc.V[k], V0[k], 1e-5, f"V{k} step")
    for m in parts:
        assert m.epoch_count == 1
        m.close()


def test_set_counts_rejects_counts_below_the_parts_own(cuda_lib):
    from paper_1708_08640_gb300 import _lib as L
    from paper_1708_08640_gb300.model import S3CMTF
    p = synth.make_problem("cfg0")
    part, _ = partition.mode1_part(p, 2, 0)
    m = S3CMTF.from_problem(part)
    counts, nnz_total = partition.whole_counts(p)
    bad = [c.copy() for c in counts]
    row = int(part.train_idx[1][0])
    bad[1][row] = 0
    with pytest.raises(L.S3Error) as ei:
        m.set_counts(bad, nnz_total)
    assert ei.value.status == L.S3_ERR_ARG
    m.set_counts(counts, nnz_total)       # the context is still usable
    assert np.isfinite(m.loss()[0])
    m.close()
