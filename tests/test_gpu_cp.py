"""S3CMTF-CP (Section 4.2: the method with a hyper-diagonal core) on the GPU against the
oracle's CP mode: one HOGWILD tile (a deterministic group step), deterministic minibatch
epochs, the full gradient, and a HOGWILD run on a rating tensor."""
import numpy as np
import pytest

from paper_1708_08640_gb300 import synth
from tests.gpu_common import assert_close_blocks, assert_step_close, f32, fp32_params, make_pair, rel
from tests.oracle_cases import random_problem

pytestmark = pytest.mark.gpu


def as_np(t):
    return t.detach().cpu().double().numpy()


def diagonal(G):
    J = G.shape[0]
    D = np.zeros_like(G)
    idx = (np.arange(J),) * G.ndim
    D[idx] = G[idx]
    return D


def cp_params(p, seed=1):
    G, U, V = fp32_params(synth.init_params(p, seed))
    J = G.shape[0]
    lam = f32(np.random.default_rng(seed).normal(size=J))
    G = np.zeros_like(G)
    G[(np.arange(J),) * G.ndim] = lam
    return G, U, V


def test_cp_hogwild_single_tile_is_group_step(cuda_lib):
    """120 entries on one CTA and one 128-entry tile: the HOGWILD CP epoch is one group step,
    which the oracle's minibatch rule with a single batch computes (cp = 1)."""
    import oracle
    from paper_1708_08640_gb300.model import S3CMTF
    prob, (G, U, V) = random_problem((30, 20, 10), (6, 6, 6), nnz=120, n_coupled=1, seed=4,
                                     coupled_nnz=40, K=9)
    prob.train_val = f32(prob.train_val + 2.0)
    for c in prob.coupled:
        c.vals = f32(c.vals)
    G, U, V = fp32_params((diagonal(G) * 0.5, U, V))
    hp = dict(lr0=0.01, mu=0.0, lambda_reg=0.1, lambda_m=2.0, core_scale=1.0)
    cpl = [(c.mode, c.K, c.rows, c.cols, c.vals) for c in prob.coupled]
    gpu = S3CMTF(prob.dims, prob.J, prob.train_idx, prob.train_val, cpl, hog_staleness=-1.0,
                 hog_tile=128, hog_ctas=1, cp=1, **hp)
    gpu.set_params(G, U, V)
    gpu.epoch("hogwild")
    G1, U1, V1 = gpu.get_params()
    orc = oracle.Oracle(prob, cp=1, **hp)
    orc.set_params(G, U, V)
    n_union = prob.train_val.shape[0] + sum(c.rows.shape[0] for c in prob.coupled)
    orc.epoch_minibatch(0, np.arange(n_union), batch=n_union)
    assert_step_close(as_np(G1), orc.G, G, 1e-4, "G")
    assert np.all(as_np(G1) == diagonal(as_np(G1)))
    for n in range(3):
        assert_step_close(as_np(U1[n]), orc.U[n], U[n], 1e-5, f"U{n}")
    assert_step_close(as_np(V1[0]), orc.V[0], V[0], 1e-5, "V")
    gpu.close()


@pytest.mark.parametrize("name", ["cfg0", "cfg3_tiny"])
def test_cp_minibatch_epochs_and_gradient_track_oracle(cuda_lib, name):
    p = synth.make_problem(name)
    gpu, orc, q, order = make_pair(p, batch=256, cp=1)
    params = cp_params(p)
    gpu.set_params(*params)
    orc.set_params(*params)
    dG, dU, dV = gpu.gradient()
    gG, gU, gV = orc.full_gradient()
    assert_close_blocks(as_np(dG), gG, 1e-5, 1e-6, "dG")
    assert np.all(as_np(dG) == diagonal(as_np(dG)))
    for n in range(p.N):
        assert_close_blocks(as_np(dU[n]), gU[n], 1e-5, 1e-6, f"dU{n}")
    for t in range(2):
        gpu.epoch("minibatch")
        orc.epoch_minibatch(t, order)
        assert rel(gpu.rmse(q.test_idx, q.test_val), orc.rmse(q.test_idx, q.test_val)) <= 1e-4
    G, U, V = gpu.get_params()
    assert rel(as_np(G), orc.G) <= 1e-4
    assert np.all(as_np(G) == diagonal(as_np(G)))
    for n in range(p.N):
        assert rel(as_np(U[n]), orc.U[n]) <= 1e-4
    gpu.close()


def test_cp_hogwild_on_rating_tensor_decreases_rmse(cuda_lib):
    from paper_1708_08640_gb300.model import S3CMTF
    p = synth.make_problem("cfg1_small")
    m = S3CMTF.from_problem(p, order=synth.union_order(p, 2), cp=1)
    m.set_params(*cp_params(p))
    m.set_test(p.test_idx, p.test_val)
    hist = [m.rmse()]
    for t in range(4):
        m.epoch("hogwild")
        hist.append(m.rmse())
    G = as_np(m.get_params()[0])
    assert np.all(np.isfinite(hist)) and hist[-1] < hist[0]
    assert np.all(G == diagonal(G))
    m.close()


def test_cp_rejects_unequal_ranks_and_bf16(cuda_lib):
    from paper_1708_08640_gb300._lib import S3Error
    from paper_1708_08640_gb300.model import S3CMTF
    prob, _ = random_problem((30, 20, 10), (4, 3, 4), nnz=50, n_coupled=0, seed=2)
    with pytest.raises(S3Error):
        S3CMTF(prob.dims, prob.J, prob.train_idx, prob.train_val, [], cp=1)
    p = synth.make_problem("cfg0")
    m = S3CMTF.from_problem(p, cp=1)
    with pytest.raises(S3Error):
        m.epoch("hogwild", "bf16")
    m.close()
