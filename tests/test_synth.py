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
