"""Edge cases of the CUDA path: a single tensor entry, a single coupled entry, an empty
test set and prediction batch, the largest tile and a one-entry tile, one batch holding the
whole epoch, an empty train tensor and out-of-range indices (rejected before any device
work)."""
import numpy as np
import pytest

import oracle
from tests.gpu_common import f32, fp32_params, rel
from tests.oracle_cases import random_problem

pytestmark = pytest.mark.gpu


def as_np(t):
    return t.detach().cpu().double().numpy()


def _pair(prob, params, **hp):
    from paper_1708_08640_gb300.model import S3CMTF
    prob.train_val = f32(prob.train_val)
    for c in prob.coupled:
        c.vals = f32(c.vals)
    params = fp32_params(params)
    cpl = [(c.mode, c.K, c.rows, c.cols, c.vals) for c in prob.coupled]
    gpu = S3CMTF(prob.dims, prob.J, prob.train_idx, prob.train_val, cpl, **hp)
    gpu.set_params(*params)
    orc = oracle.Oracle(prob, **{k: v for k, v in hp.items()
                                 if k in ("lr0", "mu", "lambda_reg", "lambda_m", "batch",
                                          "core_scale")})
    orc.set_params(*params)
    return gpu, orc


def test_single_tensor_entry_and_single_coupled_entry():
    """One tensor entry, one coupled entry: a minibatch epoch of batch 1 is Algorithm 1."""
    prob, params = random_problem((3, 4, 5), (2, 2, 2), nnz=1, n_coupled=1, seed=21,
                                  coupled_nnz=1)
    gpu, orc = _pair(prob, params, lr0=0.05, lambda_reg=0.1, lambda_m=2.0, batch=1,
                     order=np.arange(2))
    gpu.epoch("minibatch")
    orc.epoch_sequential(0, np.arange(2))
    G, U, V = gpu.get_params()
    assert rel(as_np(G), orc.G) <= 1e-5
    for n in range(3):
        assert rel(as_np(U[n]), orc.U[n]) <= 1e-5
    assert rel(as_np(V[0]), orc.V[0]) <= 1e-5
    gpu.epoch("hogwild")                        # one tile of one entry: runs and stays finite
    assert np.isfinite(gpu.loss()[0])
    gpu.close()


def test_empty_test_set_and_prediction_batch():
    prob, params = random_problem((10, 9, 8), (2, 3, 2), nnz=50, n_coupled=0, seed=22)
    gpu, _ = _pair(prob, params)
    empty = np.zeros((3, 0), dtype=np.int32)
    assert gpu.rmse(empty, np.zeros(0, dtype=np.float32)) == 0.0
    assert gpu.predict(empty).numel() == 0
    gpu.close()


@pytest.mark.parametrize("tile", [1, 128])
def test_one_entry_tiles_and_the_largest_tile(tile):
    """HOGWILD with tiles of 1 entry (four lanes) and of 128 (two lanes, the largest),
    one CTA, no staleness scaling: the epoch is a sequence of group steps of that size,
    which the oracle's minibatch rule computes with batch = the tile's items."""
    prob, params = random_problem((30, 20, 10), (4, 4, 4), nnz=128, n_coupled=0, seed=23)
    hp = dict(lr0=0.01, mu=0.0, lambda_reg=0.1, core_scale=1.0)
    n = prob.train_val.shape[0]
    gpu, orc = _pair(prob, params, hog_tile=tile, hog_ctas=1, hog_staleness=-1.0,
                     order=np.arange(n), **hp)
    gpu.epoch("hogwild")
    orc.epoch_minibatch(0, np.arange(n), batch=tile)
    G, U, _ = gpu.get_params()
    assert rel(as_np(G), orc.G) <= 1e-4
    for k in range(3):
        assert rel(as_np(U[k]), orc.U[k]) <= 1e-5
    gpu.close()


def test_one_batch_holds_the_whole_epoch():
    prob, params = random_problem((30, 20, 10), (3, 3, 3), nnz=400, n_coupled=1, seed=24,
                                  coupled_nnz=100)
    hp = dict(lr0=0.005, lambda_reg=0.1, lambda_m=1.0, batch=500)
    gpu, orc = _pair(prob, params, order=np.arange(500), **hp)
    gpu.epoch("minibatch")
    orc.epoch_minibatch(0, np.arange(500))
    G, U, V = gpu.get_params()
    assert rel(as_np(G), orc.G) <= 1e-5
    for n in range(3):
        assert rel(as_np(U[n]), orc.U[n]) <= 1e-5
    gpu.close()


def test_empty_train_and_bad_indices_are_rejected():
    from paper_1708_08640_gb300._lib import S3Error
    from paper_1708_08640_gb300.model import S3CMTF
    with pytest.raises(S3Error):
        S3CMTF((5, 5, 5), (2, 2, 2), np.zeros((3, 0), np.int32), np.zeros(0, np.float32), ())
    idx = np.array([[0, 1], [0, 5], [0, 1]], np.int32)      # 5 is outside mode 2's 5 rows
    with pytest.raises(S3Error):
        S3CMTF((5, 5, 5), (2, 2, 2), idx, np.ones(2, np.float32), ())
