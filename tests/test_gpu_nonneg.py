"""The non-negative form (hp.nonneg = 1: projected SGD, Section 5) on the GPU against the
oracle's nonneg = 1 path: a HOGWILD epoch that fits one tile is one projected group step
(FP32, BF16 and S3CMTF-CP kernels), the deterministic minibatch epochs reproduce the
oracle's, and on the cfg1 rating tensor every parameter stays non-negative in every form
while the BF16 form's test RMSE tracks the FP32 form's.

Tolerances as in the plain form's tests: FP32 steps within 1e-5 (rows) and 1e-4 (core)
plus FP32 storage rounding; BF16 steps within 3e-2 relative; minibatch epochs within 1e-4."""
import numpy as np
import pytest

import oracle
from paper_1708_08640_gb300 import synth
from tests.gpu_common import assert_step_close, f32, fp32_params, make_pair, rel
from tests.oracle_cases import random_problem

pytestmark = pytest.mark.gpu


def as_np(t):
    return t.detach().cpu().double().numpy()


def tile_problem(J, cp, seed=6, nnz=120):
    """One tile's worth of entries (120 <= 128) whose values sit below every prediction, so
    that the step drives rows below zero and the projection binds."""
    prob, (G, U, V) = random_problem((30, 20, 10), (J, J, J), nnz=nnz, n_coupled=1, seed=seed,
                                     coupled_nnz=nnz // 3, K=9)
    prob.train_val = f32(prob.train_val - 5.0)
    for c in prob.coupled:
        c.vals = f32(c.vals - 3.0)
    G = G * np.sqrt(27.0 / J ** 3)
    if cp:
        D = np.zeros_like(G)
        D[(np.arange(J),) * 3] = G[(np.arange(J),) * 3]
        G = D
    return prob, fp32_params((G, U, V))


@pytest.mark.parametrize("precision,J,cp", [("fp32", 5, 0), ("fp32", 16, 0), ("bf16", 16, 0),
                                            ("bf16", 20, 0), ("fp32", 8, 1)])
def test_nonneg_hogwild_single_tile_is_projected_group_step(cuda_lib, precision, J, cp):
    from paper_1708_08640_gb300.model import S3CMTF
    prob, params = tile_problem(J, cp)
    hp = dict(lr0=0.01, mu=0.0, lambda_reg=0.1, lambda_m=2.0, core_scale=1.0, cp=cp)
    cpl = [(c.mode, c.K, c.rows, c.cols, c.vals) for c in prob.coupled]
    gpu = S3CMTF(prob.dims, prob.J, prob.train_idx, prob.train_val, cpl, hog_staleness=-1.0,
                 hog_tile=128, hog_ctas=1, nonneg=1, **hp)
    gpu.set_params(*params)
    gpu.epoch("hogwild", precision)
    G, U, V = gpu.get_params()
    gpu.close()
    n_union = prob.train_val.shape[0] + sum(c.rows.shape[0] for c in prob.coupled)
    orc = oracle.Oracle(prob, nonneg=1, **hp)
    orc.set_params(*params)
    orc.epoch_minibatch(0, np.arange(n_union), batch=n_union)
    plain = oracle.Oracle(prob, **hp)
    plain.set_params(*params)
    plain.epoch_minibatch(0, np.arange(n_union), batch=n_union)
    # the example exercises the projection on rows, coupled rows and core
    assert np.any(plain.U[0] < 0) and np.any(plain.V[0] < 0) and np.any(plain.G < 0)
    G0, U0, V0 = params
    got = [("G", as_np(G), orc.G, G0)] + [(f"U{n}", as_np(U[n]), orc.U[n], U0[n]) for n in range(3)] \
        + [("V", as_np(V[0]), orc.V[0], V0[0])]
    for name, g, r, _ in got:
        assert g.min() >= 0.0, (name, g.min())
    if precision == "fp32":
        for name, g, r, old in got:
            assert_step_close(g, r, old, 1e-4 if name == "G" else 1e-5, name)
    else:
        errs = {name: rel(g - old, r - old) for name, g, r, old in got}
        print("BF16 projected step relative error per parameter block:", errs)
        assert max(errs.values()) < 3e-2, errs


@pytest.mark.parametrize("name", ["cfg0", "cfg3_tiny"])
def test_nonneg_minibatch_epochs_track_oracle(cuda_lib, name):
    p = synth.make_problem(name)
    gpu, orc, q, order = make_pair(p, batch=256, nonneg=1, row_rule="mean")
    for t in range(3):
        gpu.epoch("minibatch")
        orc.epoch_minibatch(t, order)
        assert rel(gpu.rmse(q.test_idx, q.test_val), orc.rmse(q.test_idx, q.test_val)) <= 1e-4
    G, U, V = gpu.get_params()
    assert rel(as_np(G), orc.G) <= 1e-4
    assert as_np(G).min() >= 0.0 and orc.G.min() >= 0.0
    for n in range(p.N):
        assert rel(as_np(U[n]), orc.U[n]) <= 1e-4
        assert as_np(U[n]).min() >= 0.0
    for m in range(len(V)):
        assert rel(as_np(V[m]), orc.V[m]) <= 1e-4
        assert as_np(V[m]).min() >= 0.0
    gpu.close()


def test_nonneg_forms_on_rating_tensor(cuda_lib, rating_tensor):
    """cfg1 at J = 16: FP32 and BF16 HOGWILD epochs and the S3CMTF-CP epoch of the
    non-negative form leave every parameter non-negative and lower the test RMSE; the BF16
    form's test RMSE per epoch is within 1% of the FP32 form's."""
    from paper_1708_08640_gb300.model import S3CMTF
    q = synth.with_rank(rating_tensor, (16, 16, 16))
    init = synth.init_params(q, 1)
    order = synth.union_order(q, 2)
    curves = {}
    for form in ("fp32", "bf16", "cp"):
        m = S3CMTF.from_problem(q, order=order, nonneg=1, cp=int(form == "cp"))
        G0, U0, V0 = init
        if form == "cp":
            D = np.zeros_like(G0)
            D[(np.arange(16),) * 3] = np.abs(G0[(np.arange(16),) * 3])
            G0 = D
        m.set_params(G0, U0, V0)
        m.set_test(q.test_idx, q.test_val)
        out = [m.rmse()]
        for t in range(3):
            m.epoch("hogwild", "bf16" if form == "bf16" else "fp32")
            out.append(m.rmse())
        G, U, V = m.get_params()
        m.close()
        assert np.all(np.isfinite(out)) and out[-1] < out[0], (form, out)
        for name, x in [("G", G)] + [(f"U{n}", u) for n, u in enumerate(U)] + [("V", V[0])]:
            assert as_np(x).min() >= 0.0, (form, name, as_np(x).min())
        curves[form] = out[1:]
    print("non-negative form, test RMSE per epoch:", curves)
    for x, y in zip(curves["fp32"], curves["bf16"]):
        assert abs(y - x) / x <= 0.01
