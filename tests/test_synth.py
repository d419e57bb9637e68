"""The seeded input generator: shapes, uniqueness, laws and determinism (CPU)."""
import numpy as np
import pytest

from paper_1708_08640_gb300 import synth


def test_cfg0_shapes_and_ranges():
    p = synth.make_problem("cfg0")
    assert p.dims == (100, 100, 20) and p.J == (5, 5, 5)
    assert p.nnz == 9000 and p.test_val.shape[0] == 1000
    allc = np.concatenate([p.train_idx, p.test_idx], axis=1)
    keys = np.ravel_multi_index(tuple(allc), p.dims)
    assert np.unique(keys).shape[0] == 10000
    for n in range(3):
        assert allc[n].min() >= 0 and allc[n].max() < p.dims[n]
    c = p.coupled[0]
    assert c.mode == 0 and c.K == 50 and c.nnz == 1000
    assert np.unique(c.rows.astype(np.int64) * 50 + c.cols).shape[0] == 1000


def test_deterministic():
    a = synth.make_problem("cfg1_tiny", seed=3)
    b = synth.make_problem("cfg1_tiny", seed=3)
    np.testing.assert_array_equal(a.train_idx, b.train_idx)
    np.testing.assert_array_equal(a.train_val, b.train_val)
    np.testing.assert_array_equal(a.coupled[0].rows, b.coupled[0].rows)
    np.testing.assert_array_equal(synth.union_order(a, 5), synth.union_order(b, 5))


def test_rating_tensor_laws():
    p = synth.make_problem("cfg1_tiny")
    assert set(np.unique(p.train_val)) <= {1.0, 2.0, 3.0, 4.0, 5.0}
    f = [np.bincount(p.train_idx[n], minlength=p.dims[n]).max() / p.nnz for n in range(3)]
    assert f[0] > 0.05 and f[1] > 0.05          # Zipf(1.1) modes have a hot row
    assert f[2] < 3.0 / p.dims[2]                # the time mode is uniform
    c = p.coupled[0]
    assert np.all(c.vals == 1.0)
    assert np.all(c.rows != c.cols)
    fwd = set(zip(c.rows.tolist(), c.cols.tolist()))
    assert fwd == set(zip(c.cols.tolist(), c.rows.tolist()))
    assert len(fwd) == c.nnz


def test_zipf_sampler_frequencies():
    rng = np.random.default_rng(0)
    ids = synth.zipf_sample(rng, 400_000, 50, 1.1)
    cnt = np.sort(np.bincount(ids, minlength=50))[::-1] / 400_000
    p = np.arange(1, 51) ** -1.1
    p /= p.sum()
    np.testing.assert_allclose(cnt[:5], p[:5], rtol=0.03)


def test_init_params_and_order():
    p = synth.make_problem("cfg0")
    G, U, V = synth.init_params(p, 1)
    assert G.shape == (5, 5, 5)
    assert abs(G.std() - np.sqrt(27 / 125)) < 0.1
    assert all(u.min() >= 0 and u.max() < 1 for u in U + V)
    o = synth.union_order(p, 2)
    np.testing.assert_array_equal(np.sort(o), np.arange(p.n_union))


def test_fourway_and_scalability_presets():
    p = synth.make_problem("scal:300:3000")
    assert p.dims == (300, 300, 300) and p.nnz == 2700
    assert p.coupled[0].nnz == 300
    with pytest.raises(ValueError):
        synth.unique_coords(np.random.default_rng(0), 10, (2, 2), ("uniform", "uniform"))


def test_incremental_unique_merge_equals_numpy_unique():
    """The generators' redraw loop keeps the sorted distinct coordinates by inserting each
    redraw's new keys; the result is numpy.unique of everything drawn so far."""
    rng = np.random.default_rng(5)
    keys = np.empty(0, dtype=np.int64)
    seen = np.empty(0, dtype=np.int64)
    for _ in range(50):
        new = rng.integers(0, 400, size=int(rng.integers(0, 60)))
        keys = synth._merge_unique(keys, new)
        seen = np.concatenate([seen, new])
        assert np.array_equal(keys, np.unique(seen))


def test_planted_values_do_not_depend_on_slicing():
    """The planted model is evaluated in slices on host threads; every slice is computed
    alone, so any slice size gives the same values bit for bit."""
    rng = np.random.default_rng(6)
    dims, J = (40, 30, 20), (3, 4, 5)
    G = rng.standard_normal(J)
    U = [rng.random((d, j)) for d, j in zip(dims, J)]
    idx = np.stack([rng.integers(0, d, size=5000) for d in dims])
    a = synth._planted_values(G, U, idx, chunk=1 << 17)
    b = synth._planted_values(G, U, idx, chunk=97)
    assert np.array_equal(a, b)
    ref = np.einsum("abc,ea,eb,ec->e", G, U[0][idx[0]], U[1][idx[1]], U[2][idx[2]])
    assert np.allclose(a, ref, rtol=1e-12, atol=1e-12)
