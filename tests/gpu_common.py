"""Helpers shared by the GPU tests: the same seeded inputs for the CUDA path and the
oracle, with the inputs rounded to FP32 once (the CUDA path stores FP32) so both sides
start from identical numbers."""
import copy

import numpy as np

from paper_1708_08640_gb300 import synth


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def fp32_problem(p):
    q = copy.copy(p)
    q.train_val = f32(p.train_val)
    q.test_val = f32(p.test_val)
    q.coupled = [synth.Coupled(c.mode, c.K, c.rows, c.cols, f32(c.vals)) for c in p.coupled]
    return q


def fp32_params(params):
    G, U, V = params
    return f32(G), [f32(u) for u in U], [f32(v) for v in V]


def make_pair(p, init_seed=1, order_seed=2, **hp):
    """(GPU model, oracle) on the same data, parameters and visiting order."""
    import oracle
    from paper_1708_08640_gb300.model import S3CMTF
    q = fp32_problem(p)
    params = fp32_params(synth.init_params(p, init_seed))
    order = synth.union_order(p, order_seed)
    h = dict(p.hparams)
    h.update(hp)
    gpu = S3CMTF.from_problem(q, order=order, **h)
    gpu.set_params(*params)
    orc = oracle.Oracle(q, **{k: v for k, v in h.items()
                             if k in ("lr0", "mu", "lambda_reg", "lambda_m", "batch",
                                      "core_scale", "cp", "nonneg")},
                        row_mean=1 if h.get("row_rule", "sum") == "mean" else 0)
    orc.set_params(*params)
    return gpu, orc, q, order


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = np.linalg.norm(a - b)
    n = np.linalg.norm(b)
    return d / n if n > 0 else d


def assert_close_blocks(got, ref, rtol, floor, what=""):
    """norm-wise rel <= rtol and |got - ref| <= rtol*|ref| + floor*max|ref| elementwise"""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    r = rel(got, ref)
    assert r <= rtol, f"{what}: norm-wise relative error {r:.3e} > {rtol}"
    scale = np.abs(ref).max() if ref.size else 0.0
    bad = np.abs(got - ref) > rtol * np.abs(ref) + floor * scale
    assert not bad.any(), (f"{what}: {int(bad.sum())} elements off, worst "
                           f"{np.abs(got - ref).max():.3e} (scale {scale:.3e})")


def assert_step_close(new, ref_new, old, rtol, what=""):
    """A step computed in FP32 and stored as FP32: the delta new - old may differ from the
    oracle's by rtol relative plus the storage rounding of the new parameter (half an FP32
    ulp, 2^-24 |p|, twice for safety), elementwise and in norm."""
    new = np.asarray(new, dtype=np.float64)
    ref_new = np.asarray(ref_new, dtype=np.float64)
    old = np.asarray(old, dtype=np.float64)
    dg, dr = new - old, ref_new - old
    store = 2.0 ** -23 * np.abs(ref_new)
    err = np.abs(dg - dr)
    assert np.linalg.norm(dg - dr) <= rtol * np.linalg.norm(dr) + np.linalg.norm(store), (
        f"{what}: norm-wise {np.linalg.norm(dg - dr):.3e} vs |d| {np.linalg.norm(dr):.3e}")
    bad = err > rtol * np.abs(dr) + store + 1e-6 * (np.abs(dr).max() if dr.size else 0.0)
    assert not bad.any(), f"{what}: {int(bad.sum())} elements off, worst {err.max():.3e}"
