"""The GPU epochs against the oracle's stored test-RMSE curves on the cfg1 workloads
(tests/golden/curve_*.json, written by tests/golden/make_golden.py from oracle/ alone):
the HOGWILD epoch, in both precision forms, tracks the sequential Algorithm 1 (P = 1) curve
within 1% per epoch (rank 10, and rank 16 for cfg2; rank 32 is an open miss, asserted as an
expected failure), and the deterministic minibatch epoch reproduces the oracle's minibatch
curve; the same two checks for the non-negative form (projected SGD, Section 5)."""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_1708_08640_gb300 import synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name, mode):
    return json.load(open(os.path.join(GOLDEN, f"curve_{name}_{mode}.json")))


def fingerprint(p):
    """The stored curve's input fingerprint (the same hash make_golden.py records)."""
    h = hashlib.sha256()
    for a in (p.train_idx, p.train_val, p.test_idx, p.test_val):
        h.update(np.ascontiguousarray(a).tobytes())
    for c in p.coupled:
        for a in (c.rows, c.cols, c.vals):
            h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()[:16]


def gpu_curve(p, rec, mode, precision="fp32", **kw):
    from paper_1708_08640_gb300.model import S3CMTF
    hp = dict(p.hparams)
    hp.update(rec["hparams"])
    if rec.get("minibatch"):
        mb = rec["minibatch"]
        hp.update(batch=mb["batch"], core_scale=mb["core_scale"], row_rule="mean" if mb["row_mean"] else "sum")
    m = S3CMTF.from_problem(p, order=synth.union_order(p, rec["order_seed"]), **hp, **kw)
    m.set_params(*synth.init_params(p, rec["init_seed"]))
    m.set_test(p.test_idx, p.test_val)
    out = []
    for _ in range(rec["epochs"]):
        m.epoch(mode, precision)
        out.append(m.rmse())
    m.close()
    return np.array(out)


def test_hogwild_tracks_algorithm1_on_cfg1(cuda_lib, rating_tensor):
    """cfg1, J = 10, the default launch (29 184 tensor entries in flight): the HOGWILD
    test RMSE after each of 10 epochs within 1% of Algorithm 1's (Section 3.3's lock-free
    scheme against the sequential one, same data, start and visiting order)."""
    rec = golden("cfg1", "sequential")
    assert fingerprint(rating_tensor) == rec["fingerprint"]
    got = gpu_curve(rating_tensor, rec, "hogwild")
    ref = np.array(rec["test_rmse"])
    dev = np.abs(got - ref) / ref
    print("HOGWILD vs Algorithm 1, relative deviation per epoch:", np.round(dev, 5).tolist())
    assert np.all(dev <= 0.01), dev


def test_bf16_hogwild_tracks_algorithm1_on_cfg1(cuda_lib, rating_tensor):
    """The BF16 tensor-core form of the same epoch (rank 10 computed on the 16 x 16 pair
    grid, the same 29 184 entries in flight): within 1% of Algorithm 1 after each of 10
    epochs, like the FP32 form."""
    rec = golden("cfg1", "sequential")
    assert fingerprint(rating_tensor) == rec["fingerprint"]
    got = gpu_curve(rating_tensor, rec, "hogwild", "bf16")
    ref = np.array(rec["test_rmse"])
    dev = np.abs(got - ref) / ref
    print("BF16 HOGWILD vs Algorithm 1, relative deviation per epoch:", np.round(dev, 5).tolist())
    assert np.all(dev <= 0.01), dev


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_hogwild_tracks_algorithm1_at_rank16_on_cfg1(cuda_lib, rating_tensor, precision):
    """cfg2's rank: the cfg1 data fitted at J = (16, 16, 16) (core step scale of that rank),
    the default launch (about 22 000 entries in flight at rank 16), both precision forms:
    test RMSE within 1% of the oracle's Algorithm 1 curve after each stored epoch."""
    from paper_1708_08640_gb300 import synth
    rec = golden("cfg1_j16", "sequential")
    q = synth.with_rank(rating_tensor, (16, 16, 16))
    assert rec["rank"] == [16, 16, 16]
    assert fingerprint(q) == rec["fingerprint"]
    got = gpu_curve(q, rec, "hogwild", precision)
    ref = np.array(rec["test_rmse"])
    dev = np.abs(got - ref) / ref
    print(f"{precision} HOGWILD vs Algorithm 1 at rank 16, relative deviation per epoch:",
          np.round((got - ref) / ref, 5).tolist())
    assert np.all(dev <= 0.01), dev


@pytest.mark.xfail(strict=True, reason="open: at rank 32 the HOGWILD curve leaves the 1% band "
                   "(cfg1, FP32: 1.0% below Algorithm 1 after the first epoch, 3.0% and 4.3% "
                   "above it after the second and third); no hot-row threshold holds them all")
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_hogwild_tracks_algorithm1_at_rank32_on_cfg1(cuda_lib, rating_tensor, precision):
    """cfg2's larger rank: the cfg1 data fitted at J = (32, 32, 32), the default launch
    (9 728 entries in flight: the FP32 form's tiles of 64, one CTA per SM; the BF16 form
    the same): test RMSE within 1% of the oracle's Algorithm 1 curve after each stored
    epoch, both precision forms.  A known miss, asserted at the 1% bound and expected to
    fail until it is closed."""
    from paper_1708_08640_gb300 import synth
    rec = golden("cfg1_j32", "sequential")
    q = synth.with_rank(rating_tensor, (32, 32, 32))
    assert rec["rank"] == [32, 32, 32]
    assert fingerprint(q) == rec["fingerprint"]
    got = gpu_curve(q, rec, "hogwild", precision)
    ref = np.array(rec["test_rmse"])
    dev = np.abs(got - ref) / ref
    print(f"{precision} HOGWILD vs Algorithm 1 at rank 32, relative deviation per epoch:",
          np.round((got - ref) / ref, 5).tolist())
    assert np.all(dev <= 0.01), dev


def test_minibatch_reproduces_oracle_curve_on_cfg1(cuda_lib, rating_tensor):
    """cfg1, J = 10: the deterministic minibatch epoch (B = 4096, row sum, core_scale 32)
    against the oracle's FP64 curve of the same rule over 10 epochs."""
    rec = golden("cfg1", "minibatch")
    assert fingerprint(rating_tensor) == rec["fingerprint"]
    got = gpu_curve(rating_tensor, rec, "minibatch")
    ref = np.array(rec["test_rmse"])
    dev = np.abs(got - ref) / ref
    print("minibatch vs oracle, relative deviation per epoch:", np.round(dev, 8).tolist())
    assert np.all(dev <= 1e-4), dev


def test_nonneg_hogwild_tracks_projected_algorithm1_on_cfg1(cuda_lib, rating_tensor):
    """The non-negative form (projected SGD, Section 5) on cfg1, J = 10, with this form's
    default launch (21 888 entries in flight, hot-row damping threshold 200): the HOGWILD
    test RMSE after each of 10 epochs within 1% of the oracle's projected Algorithm 1 curve.
    The kernels' arithmetic is pinned separately: one tile is exactly the oracle's projected
    group step, and the minibatch form reproduces the oracle's projected curve."""
    rec = golden("cfg1", "sequential_nonneg")
    assert rec["hparams"].get("nonneg") == 1
    assert fingerprint(rating_tensor) == rec["fingerprint"]
    got = gpu_curve(rating_tensor, rec, "hogwild")
    ref = np.array(rec["test_rmse"])
    dev = np.abs(got - ref) / ref
    print("non-negative HOGWILD vs projected Algorithm 1, relative deviation per epoch:",
          np.round((got - ref) / ref, 5).tolist())
    assert np.all(dev <= 0.01), dev


def test_nonneg_minibatch_reproduces_oracle_curve_on_cfg1(cuda_lib, rating_tensor):
    """The non-negative form's deterministic minibatch epoch (B = 4096, row sum,
    core_scale 32) against the oracle's FP64 curve of the same projected rule."""
    rec = golden("cfg1", "minibatch_nonneg")
    assert rec["hparams"].get("nonneg") == 1
    assert fingerprint(rating_tensor) == rec["fingerprint"]
    got = gpu_curve(rating_tensor, rec, "minibatch")
    ref = np.array(rec["test_rmse"])
    dev = np.abs(got - ref) / ref
    print("non-negative minibatch vs oracle, relative deviation per epoch:", np.round(dev, 8).tolist())
    assert np.all(dev <= 1e-4), dev
