"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded
inputs.  Tolerances: loss, gradient and one deterministic step within 1e-5 relative
(FP32 form, compensated reductions)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1708_08640_gb300 import synth
from tests.gpu_common import (assert_close_blocks, assert_step_close, f32, fp32_params,
                              fp32_problem, make_pair, rel)

pytestmark = pytest.mark.gpu

CASES = ["cfg0", "cfg1_tiny", "cfg3_tiny"]


@pytest.fixture(scope="module")
def problems():
    return {name: synth.make_problem(name) for name in CASES}


def as_np(t):
    return t.detach().cpu().double().numpy()


@pytest.mark.parametrize("name", CASES)
def test_loss_and_rmse(cuda_lib, problems, name):
    p = problems[name]
    gpu, orc, q, _ = make_pair(p)
    f, tr = gpu.loss()
    fo, se, _ = orc.loss()
    assert rel(f, fo) <= 1e-5
    assert rel(tr, np.sqrt(se / q.nnz)) <= 1e-5
    r_gpu = gpu.rmse(q.test_idx, q.test_val)
    assert rel(r_gpu, orc.rmse(q.test_idx, q.test_val)) <= 1e-5
    gpu.set_test(q.test_idx, q.test_val)
    assert gpu.rmse() == pytest.approx(r_gpu, rel=1e-12)


@pytest.mark.parametrize("name", CASES)
def test_gradient(cuda_lib, problems, name):
    p = problems[name]
    gpu, orc, q, _ = make_pair(p)
    dG, dU, dV = gpu.gradient()
    gG, gU, gV = orc.full_gradient()
    assert_close_blocks(as_np(dG), gG, 1e-5, 1e-6, "dG")
    for n in range(p.N):
        assert_close_blocks(as_np(dU[n]), gU[n], 1e-5, 1e-6, f"dU{n}")
    for m in range(len(p.coupled)):
        assert_close_blocks(as_np(dV[m]), gV[m], 1e-5, 1e-6, f"dV{m}")


@pytest.mark.parametrize("name", ["cfg0", "cfg3_tiny"])
def test_predict(cuda_lib, problems, name):
    p = problems[name]
    gpu, orc, q, _ = make_pair(p)
    rng = np.random.default_rng(0)
    n = 1000 + 77                                    # ragged against the 256-entry tile
    idx = np.stack([rng.integers(0, d, n) for d in p.dims]).astype(np.int32)
    got = gpu.predict(idx).cpu().double().numpy()
    ref = orc.predict(idx)
    assert_close_blocks(got, ref, 1e-5, 1e-6, "predict")


@pytest.mark.parametrize("name,batch", [("cfg0", None), ("cfg1_tiny", None), ("cfg3_tiny", None)])
def test_one_deterministic_step(cuda_lib, problems, name, batch):
    """One minibatch step that covers every item: parameter deltas within 1e-5 relative,
    plus the FP32 rounding of the stored parameters."""
    p = problems[name]
    B = p.n_union
    gpu, orc, q, order = make_pair(p, batch=B)
    G0, U0, V0 = fp32_params(synth.init_params(p, 1))
    gpu.epoch("minibatch")
    orc.epoch_minibatch(0, order)
    G, U, V = gpu.get_params()
    assert_step_close(as_np(G), orc.G, G0, 1e-5, "dG step")
    for n in range(p.N):
        assert_step_close(as_np(U[n]), orc.U[n], U0[n], 1e-5, f"dU{n} step")
    for m in range(len(p.coupled)):
        assert_step_close(as_np(V[m]), orc.V[m], V0[m], 1e-5, f"dV{m} step")


@pytest.mark.parametrize("row_rule", ["sum", "mean"])
def test_minibatch_epochs_track_oracle(cuda_lib, problems, row_rule):
    """Several epochs of 256-item batches on cfg0 (ragged last batch): parameters within
    1e-4 of the FP64 oracle after 3 epochs; test RMSE within 1e-4 relative."""
    p = problems["cfg0"]
    gpu, orc, q, order = make_pair(p, batch=256, row_rule=row_rule)
    for t in range(3):
        gpu.epoch("minibatch")
        orc.epoch_minibatch(t, order)
        assert rel(gpu.rmse(q.test_idx, q.test_val), orc.rmse(q.test_idx, q.test_val)) <= 1e-4
    G, U, V = gpu.get_params()
    assert rel(as_np(G), orc.G) <= 1e-4
    for n in range(p.N):
        assert rel(as_np(U[n]), orc.U[n]) <= 1e-4


@pytest.mark.parametrize("row_rule", ["sum", "mean"])
def test_minibatch_epochs_track_oracle_4way(cuda_lib, problems, row_rule):
    """The deterministic epoch on the 4-way cfg3_tiny data (two coupled matrices, batches of
    1024 items, both row rules): test RMSE within 1e-4 relative of the FP64 oracle's after
    each of 3 epochs, parameters within 1e-4."""
    p = problems["cfg3_tiny"]
    gpu, orc, q, order = make_pair(p, batch=1024, row_rule=row_rule)
    for t in range(3):
        gpu.epoch("minibatch")
        orc.epoch_minibatch(t, order)
        a, b = gpu.rmse(q.test_idx, q.test_val), orc.rmse(q.test_idx, q.test_val)
        assert np.isfinite(b)
        assert abs(a - b) / b <= 1e-4, (t, a, b)
    G, U, V = gpu.get_params()
    assert rel(as_np(G), orc.G) <= 1e-4
    for n in range(p.N):
        assert rel(as_np(U[n]), orc.U[n]) <= 1e-4
    for m in range(len(p.coupled)):
        assert rel(as_np(V[m]), orc.V[m]) <= 1e-4


def test_minibatch_curve_cfg1_tiny(cuda_lib, problems):
    p = problems["cfg1_tiny"]
    gpu, orc, q, order = make_pair(p)
    for t in range(4):
        gpu.epoch("minibatch")
        orc.epoch_minibatch(t, order)
        a, b = gpu.rmse(q.test_idx, q.test_val), orc.rmse(q.test_idx, q.test_val)
        assert abs(a - b) / b <= 1e-3, (t, a, b)


def test_hogwild_runs_and_decreases_rmse(cuda_lib, problems):
    p = problems["cfg1_tiny"]
    gpu, orc, q, order = make_pair(p)
    r0 = gpu.rmse(q.test_idx, q.test_val)
    hist = []
    for t in range(4):
        gpu.epoch("hogwild")
        hist.append(gpu.rmse(q.test_idx, q.test_val))
    assert np.all(np.isfinite(hist))
    assert hist[-1] < r0


def test_init_params_from_seed(cuda_lib):
    """The library's own initial parameters follow the counter-based generator
    (splitmix64) written out here from its published definition."""
    from paper_1708_08640_gb300.model import S3CMTF
    p = synth.make_problem("cfg0")
    gpu = S3CMTF.from_problem(p, seed=1234)
    G, U, V = gpu.get_params()
    M64 = (1 << 64) - 1

    def mix(z):
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        return z ^ (z >> 31)

    def unif(stream, k):
        z = mix((1234 + 0x9E3779B97F4A7C15 * ((stream << 40) + k + 1)) & M64)
        return (z >> 11) * 2.0 ** -53

    U1 = U[1].cpu().numpy()
    for (i, j) in [(0, 0), (3, 4), (99, 2)]:
        assert U1[i, j] == np.float32(unif(2, i * 5 + j))
    V0 = V[0].cpu().numpy()
    assert V0[7, 3] == np.float32(unif(1 + 3, 7 * 5 + 3))
    sigma = np.sqrt(27 / 125)
    Gn = G.cpu().numpy().ravel()
    for l in [0, 17, 124]:
        u1 = 1.0 - unif(0, 2 * l)
        u2 = unif(0, 2 * l + 1)
        g = sigma * np.sqrt(-2 * np.log(u1)) * np.cos(2 * np.pi * u2)
        assert Gn[l] == pytest.approx(g, rel=1e-6)


def test_params_roundtrip_and_epoch_counter(cuda_lib, problems):
    p = problems["cfg0"]
    gpu, orc, q, order = make_pair(p)
    G0, U0, V0 = fp32_params(synth.init_params(p, 1))
    G, U, V = gpu.get_params()
    assert np.array_equal(as_np(G), G0)
    assert all(np.array_equal(as_np(a), b) for a, b in zip(U, U0))
    assert gpu.epoch_count == 0
    gpu.epoch("minibatch")
    assert gpu.epoch_count == 1
    gpu.epoch_count = 5
    assert gpu.epoch_count == 5


def test_resume_equals_uninterrupted(cuda_lib, problems):
    p = problems["cfg0"]
    a, _, _, _ = make_pair(p, batch=512)
    b, _, _, _ = make_pair(p, batch=512)
    for _ in range(3):
        a.epoch("minibatch")
    b.epoch("minibatch")
    G, U, V = b.get_params()
    t = b.epoch_count
    c, _, _, _ = make_pair(p, batch=512)
    c.set_params(G, U, V)
    c.epoch_count = t
    for _ in range(2):
        c.epoch("minibatch")
    Ga, Ua, _ = a.get_params()
    Gc, Uc, _ = c.get_params()
    assert torch.equal(Ga, Gc) and all(torch.equal(x, y) for x, y in zip(Ua, Uc))


def test_update_values(cuda_lib, problems):
    p = problems["cfg0"]
    gpu, orc, q, order = make_pair(p)
    rng = np.random.default_rng(9)
    newx = f32(rng.normal(size=q.nnz) + 1.0)
    newy = f32(rng.normal(size=q.coupled[0].nnz))
    gpu.update_values(newx.astype(np.float32), [newy.astype(np.float32)])
    q2 = fp32_problem(p)
    q2.train_val = newx
    q2.coupled[0].vals = newy
    o2 = oracle.Oracle(q2, **p.hparams)
    o2.set_params(*fp32_params(synth.init_params(p, 1)))
    assert rel(gpu.loss()[0], o2.loss()[0]) <= 1e-5


def test_update_values_reach_every_layout(cuda_lib, problems):
    """s3_update_values stages the values once; each layout takes them when a call next reads
    it.  After two updates (the second without coupled values, which keep the first's): the
    loss and the gradient equal the oracle's on those values (1e-5), a minibatch epoch its
    epoch (1e-4, the multi-epoch bound), and a HOGWILD epoch on one CTA the epoch of a
    context built with them (1e-5)."""
    from paper_1708_08640_gb300.model import S3CMTF
    p = problems["cfg0"]
    gpu, _, q, order = make_pair(p, batch=256)
    rng = np.random.default_rng(10)
    y1 = f32(rng.normal(size=q.coupled[0].nnz))
    x2 = f32(rng.normal(size=q.nnz) + 2.0)
    gpu.update_values(f32(rng.normal(size=q.nnz)).astype(np.float32), [y1.astype(np.float32)])
    gpu.update_values(x2.astype(np.float32))
    q2 = fp32_problem(p)
    q2.train_val = x2
    q2.coupled[0].vals = y1
    params = fp32_params(synth.init_params(p, 1))
    hp = {k: v for k, v in p.hparams.items() if k in ("lr0", "mu", "lambda_reg", "lambda_m", "core_scale")}
    o2 = oracle.Oracle(q2, batch=256, **hp)
    o2.set_params(*params)
    assert rel(gpu.loss()[0], o2.loss()[0]) <= 1e-5
    dG, dU, dV = gpu.gradient()
    gG, gU, gV = o2.full_gradient()
    assert rel(as_np(dG), gG) <= 1e-5
    assert all(rel(as_np(a), b) <= 1e-5 for a, b in zip(dU, gU))
    gpu.epoch("minibatch")
    o2.epoch_minibatch(0, order)
    G, U, _ = gpu.get_params()
    assert rel(as_np(G), o2.G) <= 1e-4
    assert all(rel(as_np(a), b) <= 1e-4 for a, b in zip(U, o2.U))
    # HOGWILD on one CTA: this context (values updated) against one built with them
    h = dict(p.hparams, hog_ctas=1)
    a = S3CMTF.from_problem(q, order=order, **h)
    b = S3CMTF.from_problem(q2, order=order, **h)
    for m in (a, b):
        m.set_params(*params)
    a.update_values(x2.astype(np.float32), [y1.astype(np.float32)])
    a.epoch("hogwild")
    b.epoch("hogwild")
    Ga, Ua, _ = a.get_params()
    Gb, Ub, _ = b.get_params()
    assert rel(as_np(Ga), as_np(Gb)) <= 1e-5
    assert all(rel(as_np(x), as_np(y)) <= 1e-5 for x, y in zip(Ua, Ub))
    for m in (gpu, a, b):
        m.close()


def test_no_coupled_small_rank_and_ragged(cuda_lib):
    """J = 1 and J = 3 (padded ranks), no coupled matrix, nnz not a multiple of 256, rows
    without entries."""
    from tests.oracle_cases import random_problem
    for dims, J in [((40, 30, 20), (1, 1, 1)), ((40, 30, 20), (3, 2, 3))]:
        prob, params = random_problem(dims, J, nnz=1234, n_coupled=0, seed=3)
        prob.train_val = f32(prob.train_val)
        params = fp32_params(params)
        from paper_1708_08640_gb300.model import S3CMTF
        gpu = S3CMTF(dims, J, prob.train_idx, prob.train_val, (), lr0=0.01, lambda_reg=0.1,
                     batch=100)
        gpu.set_params(*params)
        orc = oracle.Oracle(prob, lr0=0.01, lambda_reg=0.1, batch=100)
        orc.set_params(*params)
        assert rel(gpu.loss()[0], orc.loss()[0]) <= 1e-5
        dG, dU, _ = gpu.gradient()
        gG, gU, _ = orc.full_gradient()
        assert_close_blocks(as_np(dG), gG, 1e-5, 1e-6, "dG")
        for n in range(3):
            assert_close_blocks(as_np(dU[n]), gU[n], 1e-5, 1e-6, f"dU{n}")
        order = np.arange(1234)
        gpu2 = S3CMTF(dims, J, prob.train_idx, prob.train_val, (), lr0=0.01, lambda_reg=0.1,
                      batch=100, order=order)
        gpu2.set_params(*params)
        gpu2.epoch("minibatch")
        orc.epoch_minibatch(0, order)
        G, U, _ = gpu2.get_params()
        assert rel(as_np(G), orc.G) <= 1e-5
        for n in range(3):
            assert rel(as_np(U[n]), orc.U[n]) <= 1e-5


def test_divergence_is_reported(cuda_lib, problems):
    from paper_1708_08640_gb300 import _lib as L
    p = problems["cfg0"]
    gpu, _, _, _ = make_pair(p, lr0=1e6, mu=0.0)
    with pytest.raises(L.S3Error) as ei:
        for _ in range(5):
            gpu.epoch("minibatch")
    assert ei.value.status == L.S3_ERR_DIVERGED


def test_autograd_function_matches_oracle(cuda_lib, problems):
    from paper_1708_08640_gb300.autograd import s3_loss
    p = problems["cfg3_tiny"]
    gpu, orc, q, _ = make_pair(p)
    G0, U0, V0 = fp32_params(synth.init_params(p, 1))
    G = torch.tensor(G0, dtype=torch.float32, device="cuda", requires_grad=True)
    U = [torch.tensor(u, dtype=torch.float32, device="cuda", requires_grad=True) for u in U0]
    V = [torch.tensor(v, dtype=torch.float32, device="cuda", requires_grad=True) for v in V0]
    f = s3_loss(gpu, G, U, V)
    (2.5 * f).backward()
    gG, gU, gV = orc.full_gradient()
    assert rel(f.item(), orc.loss()[0]) <= 1e-5
    assert_close_blocks(as_np(G.grad), 2.5 * gG, 1e-5, 1e-6, "G.grad")
    for n in range(4):
        assert_close_blocks(as_np(U[n].grad), 2.5 * gU[n], 1e-5, 1e-6, f"U{n}.grad")
    for m in range(2):
        assert_close_blocks(as_np(V[m].grad), 2.5 * gV[m], 1e-5, 1e-6, f"V{m}.grad")
