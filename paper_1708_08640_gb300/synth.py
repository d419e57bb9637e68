"""Seeded synthetic inputs shaped like the paper's rating-tensor workloads.

The paper evaluates on MovieLens, Netflix and Yelp (Section 4.1, Table 4), which are not
available here.  This module draws stand-ins with the same structure: a sparse N-way
tensor of observed entries with power-law (Zipf) or uniform coordinates, values from a
planted Tucker model plus noise (optionally turned into integer ratings 1..5), and sparse
coupled matrices sharing one tensor mode (Section 2.3, Definition 1).

This module is input generation only.  It holds none of the factorisation method's
arithmetic (no loss, no gradient, no update): the planted values are produced by a chain
of numpy tensordot/einsum contractions of the planted core and factor rows, which is the
data-generating process the workloads name.  Everything is driven by
``numpy.random.default_rng(seed)``.  The random numbers the method itself draws (the
initial parameters and the visiting order of Algorithm 1) are drawn here too and passed to
both the CUDA path and the oracle as inputs.
"""
from __future__ import annotations

import os
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Coupled", "Problem", "make_problem", "init_params", "union_order", "PRESETS",
    "zipf_sample", "unique_coords",
]


@dataclass
class Coupled:
    """A sparse matrix Y (I_c x K) coupled to tensor mode ``mode`` (0-based)."""
    mode: int
    K: int
    rows: np.ndarray   # int32 [nnz], index into I_c
    cols: np.ndarray   # int32 [nnz], index into K
    vals: np.ndarray   # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.rows.shape[0])


@dataclass
class Problem:
    name: str
    dims: tuple
    J: tuple
    train_idx: np.ndarray    # int32 [N, nnz_train]
    train_val: np.ndarray    # float64 [nnz_train]
    test_idx: np.ndarray     # int32 [N, nnz_test]
    test_val: np.ndarray     # float64 [nnz_test]
    coupled: list = field(default_factory=list)
    hparams: dict = field(default_factory=dict)
    recipe: str = ""

    @property
    def N(self) -> int:
        return len(self.dims)

    @property
    def nnz(self) -> int:
        return int(self.train_val.shape[0])

    @property
    def n_union(self) -> int:
        return self.nnz + sum(c.nnz for c in self.coupled)


# ----------------------------------------------------------------------------- samplers

def _in_slices(n, fn, chunk=1 << 22):
    """fn(slice) over [0, n) in slices of `chunk`, on a pool of host threads for large n
    (numpy releases the interpreter lock in these loops). Every slice is computed as it
    would be alone, so the results do not depend on the thread count."""
    slices = [slice(s, min(n, s + chunk)) for s in range(0, n, chunk)]
    workers = min(len(slices), os.cpu_count() or 1)
    if workers <= 1:
        for sl in slices:
            fn(sl)
        return
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(workers) as pool:
        list(pool.map(fn, slices))


def _zipf_ranks(cdf, u):
    """Ranks of the uniform draws u under the CDF cdf (searchsorted, clipped), by slices."""
    rank = np.empty(u.shape[0], dtype=np.int64)

    def one(sl):
        r = np.searchsorted(cdf, u[sl], side="right")
        np.minimum(r, cdf.shape[0] - 1, out=r)
        rank[sl] = r
    _in_slices(u.shape[0], one)
    return rank


def zipf_sample(rng, n, support, s):
    """Draw ``n`` ids from a finite Zipf law p_k ~ k^-s over ranks 1..support.

    Ranks are mapped to ids through a seeded permutation so that hot ids are not
    the small ones.  Returns int64 ids in [0, support).
    """
    w = np.arange(1, support + 1, dtype=np.float64) ** (-float(s))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    rank = _zipf_ranks(cdf, rng.random(n))
    perm = rng.permutation(support)
    return perm[rank].astype(np.int64)


def _merge_unique(keys, new):
    """Sorted distinct values of keys (sorted, distinct) together with new: the same result
    as numpy.unique(numpy.concatenate([keys, new])), by sorting only the new values and
    inserting those not present at their positions."""
    new = np.sort(new)
    if new.shape[0] > 1:
        first = np.empty(new.shape[0], dtype=bool)
        first[0] = True
        np.not_equal(new[1:], new[:-1], out=first[1:])
        new = new[first]
    if keys.shape[0] == 0:
        return new
    pos = np.searchsorted(keys, new)
    present = keys[np.minimum(pos, keys.shape[0] - 1)] == new
    present &= pos < keys.shape[0]
    keep = ~present
    return np.insert(keys, pos[keep], new[keep])


def _draw_coords(rng, n, dims, laws, perms):
    cols = []
    for d, law, perm in zip(dims, laws, perms):
        if law == "uniform":
            cols.append(rng.integers(0, d, size=n, dtype=np.int64))
        else:
            s = float(law[4:])
            w = np.arange(1, d + 1, dtype=np.float64) ** (-s)
            cdf = np.cumsum(w)
            cdf /= cdf[-1]
            rank = _zipf_ranks(cdf, rng.random(n))
            ids = np.empty(n, dtype=np.int64)

            def gather(sl, ids=ids, rank=rank, perm=perm):
                ids[sl] = perm[rank[sl]]
            _in_slices(n, gather)
            cols.append(ids)
    return cols


def unique_coords(rng, n, dims, laws):
    """Exactly ``n`` distinct coordinates; each mode follows its law ('uniform' or
    'zipfS').  Duplicates are dropped and the deficit redrawn until n remain; the
    result is in random order.  Returns int64 [len(dims), n]."""
    dims = tuple(int(d) for d in dims)
    total = 1
    for d in dims:
        total *= d
    if n > total:
        raise ValueError("more unique coordinates requested than cells")
    if total >= 1 << 62:
        return _unique_coords_wide(rng, n, dims, laws)
    # one rank->id permutation per Zipf mode, fixed across redraws
    perms = [rng.permutation(d) if law != "uniform" else None for d, law in zip(dims, laws)]
    keys = np.empty(0, dtype=np.int64)
    need = n
    while need > 0:
        draw = int(need * 1.15) + 64
        cols = _draw_coords(rng, draw, dims, laws, perms)
        k = np.ravel_multi_index(tuple(cols), dims).astype(np.int64)
        keys = _merge_unique(keys, k)
        need = n - keys.shape[0]
    if keys.shape[0] > n:
        keys = rng.choice(keys, size=n, replace=False)
    keys = keys[rng.permutation(keys.shape[0])]
    return np.stack(np.unravel_index(keys, dims)).astype(np.int64)


def _unique_coords_wide(rng, n, dims, laws):
    """unique_coords for index spaces beyond 64-bit linear keys: duplicates found by a
    lexicographic sort of the coordinate columns."""
    perms = [rng.permutation(d) if law != "uniform" else None for d, law in zip(dims, laws)]
    cols = np.empty((len(dims), 0), dtype=np.int64)
    need = n
    while need > 0:
        draw = int(need * 1.15) + 64
        new = np.stack(_draw_coords(rng, draw, dims, laws, perms)).astype(np.int64)
        cols = np.concatenate([cols, new], axis=1)
        order = np.lexsort(cols[::-1])
        srt = cols[:, order]
        keep = np.ones(srt.shape[1], dtype=bool)
        keep[1:] = np.any(srt[:, 1:] != srt[:, :-1], axis=0)
        cols = srt[:, keep]
        need = n - cols.shape[1]
    if cols.shape[1] > n:
        cols = cols[:, rng.choice(cols.shape[1], size=n, replace=False)]
    return cols[:, rng.permutation(cols.shape[1])]


def _planted_values(G, U, idx, chunk=1 << 17):
    """Planted model evaluated at coordinates idx (data synthesis; numpy contractions)."""
    N = len(U)
    # contract the last mode against every row of U[N-1] once
    T = np.tensordot(U[N - 1], G, axes=([1], [N - 1]))      # (I_N, J_1..J_{N-1})
    out = np.empty(idx.shape[1], dtype=np.float64)

    def one(e):
        t = T[idx[N - 1, e]]
        for n in range(N - 2, -1, -1):
            t = np.einsum("c...j,cj->c...", t, U[n][idx[n, e]])
        out[e] = t
    _in_slices(idx.shape[1], one, chunk)
    return out


def _split(rng, idx, val, test_frac):
    n = idx.shape[1]
    n_test = int(round(n * test_frac))
    perm = rng.permutation(n)
    te, tr = perm[:n_test], perm[n_test:]
    return (idx[:, tr].astype(np.int32), val[tr].copy(),
            idx[:, te].astype(np.int32), val[te].copy())


def _binary_symmetric(rng, n_entries, I, law):
    """Symmetric 0/1 matrix with n_entries stored entries (n_entries/2 undirected
    edges), endpoints from ``law``, no self loops, no duplicate edges."""
    n_edges = n_entries // 2
    perm = rng.permutation(I) if law != "uniform" else None
    keys = np.empty(0, dtype=np.int64)
    need = n_edges
    while need > 0:
        draw = int(need * 1.2) + 64
        a, b = _draw_coords(rng, draw, (I, I), (law, law), (perm, perm))
        keep = a != b
        lo, hi = np.minimum(a, b)[keep], np.maximum(a, b)[keep]
        keys = _merge_unique(keys, lo * I + hi)
        need = n_edges - keys.shape[0]
    if keys.shape[0] > n_edges:
        keys = rng.choice(keys, size=n_edges, replace=False)
    lo, hi = keys // I, keys % I
    r = np.concatenate([lo, hi])
    c = np.concatenate([hi, lo])
    p = rng.permutation(r.shape[0])
    return r[p].astype(np.int32), c[p].astype(np.int32), np.ones(r.shape[0])


def _sparse_matrix(rng, n_entries, I, K, law_r="uniform", law_c="uniform"):
    rc = unique_coords(rng, n_entries, (I, K), (law_r, law_c))
    return rc[0].astype(np.int32), rc[1].astype(np.int32)


# ----------------------------------------------------------------------------- presets

def _tensor(rng, dims, nnz, laws, Jp, value_mode, noise):
    N = len(dims)
    coords = unique_coords(rng, nnz, dims, laws)
    Gp = rng.standard_normal(Jp)
    Up = [rng.random((d, j)) for d, j in zip(dims, Jp)]
    raw = _planted_values(Gp, Up, coords)
    if value_mode == "rating":
        z = (raw - raw.mean()) / raw.std()
        v = 3.0 + z + rng.normal(0.0, noise, size=raw.shape)
        v = np.clip(np.rint(v), 1.0, 5.0)
    else:
        v = raw + rng.normal(0.0, noise, size=raw.shape)
    assert coords.shape[0] == N
    return coords, v, Gp, Up


def _cfg0(rng, noise=0.1):
    dims, J = (100, 100, 20), (5, 5, 5)
    coords, v, Gp, Up = _tensor(rng, dims, 10_000, ("uniform",) * 3, J, "real", noise)
    tr_i, tr_v, te_i, te_v = _split(rng, coords, v, 0.10)
    W = rng.random((50, 5))
    r, c = _sparse_matrix(rng, 1_000, 100, 50)
    y = np.einsum("ej,ej->e", Up[0][r], W[c]) + rng.normal(0.0, noise, size=r.shape[0])
    cpl = [Coupled(0, 50, r, c, y)]
    hp = dict(lr0=0.01, mu=0.1, lambda_reg=0.01, lambda_m=10.0, batch=4096, core_scale=1.0)
    rec = ("3-way 100x100x20, 10k unique uniform coordinates, planted core 5x5x5 ~ N(0,1), "
           "factors ~ U(0,1), + N(0,0.1^2), 90/10 split; coupled 100x50 on mode 1, 1k unique "
           "uniform entries = U1 W^T + N(0,0.1^2), W 50x5 ~ U(0,1)")
    return dims, J, tr_i, tr_v, te_i, te_v, cpl, hp, rec


def rating_core_scale(J):
    """Core step scale of the rating workloads: 32 at ranks (10, 10, 10), times (10^3 / prod J)
    at other ranks.  With factors ~ U(0,1) the outer products a1 o a2 o a3 share a mean
    direction of squared norm prod(J_n / 4), which sets the curvature of a mean core step; the
    scaling keeps eta * core_scale * prod(J_n / 4) at its rank-10 value (0.5 at eta 0.001),
    where rank 32 with core_scale 32 diverges."""
    return 32.0 * 1000.0 / float(np.prod(J))


def with_rank(prob, J):
    """A copy of a rating-workload problem at ranks J (cfg2: the cfg1 data at J = 16, 32),
    with the core step scale of that rank."""
    import copy
    q = copy.copy(prob)
    q.J = tuple(int(j) for j in J)
    q.hparams = dict(prob.hparams, core_scale=rating_core_scale(q.J))
    return q


def _rating_like(rng, dims, nnz, J, n_cpl, zipf="zipf1.1"):
    coords, v, _, _ = _tensor(rng, dims, nnz, (zipf, zipf, "uniform"), (10, 10, 10),
                              "rating", 0.2)
    tr_i, tr_v, te_i, te_v = _split(rng, coords, v, 0.10)
    r, c, y = _binary_symmetric(rng, n_cpl, dims[0], zipf)
    cpl = [Coupled(0, dims[0], r, c, y)]
    hp = dict(lr0=0.001, mu=0.1, lambda_reg=0.1, lambda_m=10.0, batch=4096,
              core_scale=rating_core_scale(J))
    rec = (f"3-way {dims[0]}x{dims[1]}x{dims[2]}, {nnz} unique coordinates, modes 1-2 "
           f"{zipf}, mode 3 uniform; planted rank-(10,10,10) core ~ N(0,1), factors ~ U(0,1), "
           "standardised to mean 3 std 1, + N(0,0.2^2), rounded half-even, clipped to 1..5; "
           f"90/10 split; coupled binary symmetric {dims[0]}x{dims[0]} on mode 1 with "
           f"{n_cpl} entries, {zipf} endpoints, no self loops or duplicates")
    return dims, J, tr_i, tr_v, te_i, te_v, cpl, hp, rec


def _cfg1(rng, J=(10, 10, 10)):
    return _rating_like(rng, (100_000, 50_000, 1_000), 10_000_000, J, 5_000_000)


def _cfg1_small(rng, J=(10, 10, 10)):
    return _rating_like(rng, (20_000, 10_000, 200), 1_000_000, J, 500_000)


def _cfg1_tiny(rng, J=(10, 10, 10)):
    return _rating_like(rng, (2_000, 1_000, 50), 60_000, J, 30_000)


def _cfg4(rng, scale=1, J=(20, 20, 20)):
    """Config 4 (scale): 3-way 10^7 x 10^6 x 1000 with 5*10^8 entries, Zipf(1.1) on modes
    1-2, uniform mode 3, ratings 1..5 from a planted rank-(20,20,20) Tucker model + noise;
    coupled: binary symmetric 10^7 x 10^7 on mode 1 (10^8 entries, Zipf(1.1) endpoints),
    10^6 x 500 on mode 2 (5*10^7 entries ~ U(0,1)), 1000 x 64 dense on mode 3.  `scale`
    divides modes 1-2, the tensor and the two sparse coupled matrices."""
    I1, I2, I3 = 10_000_000 // scale, 1_000_000 // scale, 1000
    nnz = 500_000_000 // scale
    coords, v, _, _ = _tensor(rng, (I1, I2, I3), nnz, ("zipf1.1", "zipf1.1", "uniform"),
                              (20, 20, 20), "rating", 0.2)
    tr_i, tr_v, te_i, te_v = _split(rng, coords, v, 0.10)
    del coords, v
    r, c, y = _binary_symmetric(rng, 100_000_000 // scale, I1, "zipf1.1")
    r2, c2 = _sparse_matrix(rng, 50_000_000 // scale, I2, 500)
    r3, c3 = np.meshgrid(np.arange(I3, dtype=np.int32), np.arange(64, dtype=np.int32), indexing="ij")
    cpl = [Coupled(0, I1, r, c, y),
           Coupled(1, 500, r2, c2, rng.random(r2.shape[0])),
           Coupled(2, 64, r3.ravel(), c3.ravel(), rng.random(I3 * 64))]
    hp = dict(lr0=0.001, mu=0.1, lambda_reg=0.1, lambda_m=10.0, batch=4096,
              core_scale=rating_core_scale(J))
    rec = (f"3-way {I1}x{I2}x{I3}, {nnz} unique coordinates, modes 1-2 Zipf(1.1), mode 3 "
           "uniform; planted rank-(20,20,20) core ~ N(0,1), factors ~ U(0,1), standardised to "
           "mean 3 std 1, + N(0,0.2^2), rounded half-even, clipped to 1..5; 90/10 split; coupled "
           f"binary symmetric {I1}x{I1} on mode 1 ({100_000_000 // scale} entries, Zipf(1.1) "
           f"endpoints), {I2}x500 on mode 2 ({50_000_000 // scale} entries ~ U(0,1)), "
           f"{I3}x64 dense on mode 3")
    return (I1, I2, I3), J, tr_i, tr_v, te_i, te_v, cpl, hp, rec


def _fourway(rng, dims, nnz, nA, nB):
    J = (8, 8, 8, 8)
    coords, v, _, _ = _tensor(rng, dims, nnz, ("zipf1.05",) * 4, J, "real", 0.1)
    tr_i, tr_v, te_i, te_v = _split(rng, coords, v, 0.10)
    ra, ca = _sparse_matrix(rng, nA, dims[0], 200)
    ya = rng.standard_normal(ra.shape[0])
    rb, cb = _sparse_matrix(rng, nB, dims[1], 1000)
    yb = np.ones(rb.shape[0])
    cpl = [Coupled(0, 200, ra, ca, ya), Coupled(1, 1000, rb, cb, yb)]
    hp = dict(lr0=0.001, mu=0.1, lambda_reg=0.1, lambda_m=10.0, batch=4096, core_scale=32.0)
    rec = (f"4-way {'x'.join(map(str, dims))}, {nnz} unique Zipf(1.05) coordinates on all "
           "modes, planted rank-(8,8,8,8) + N(0,0.1^2); coupled A on mode 1 (x200) with "
           f"{nA} N(0,1) entries, coupled B binary on mode 2 (x1000) with {nB} entries")
    return dims, J, tr_i, tr_v, te_i, te_v, cpl, hp, rec


def _cfg3(rng):
    return _fourway(rng, (1_000_000, 500_000, 100, 24), 50_000_000, 20_000_000, 2_000_000)


def _cfg3_small(rng):
    return _fourway(rng, (20_000, 10_000, 50, 24), 500_000, 200_000, 20_000)


def _cfg3_tiny(rng):
    return _fourway(rng, (2_000, 1_000, 20, 24), 30_000, 12_000, 1_200)


def _scal(rng, I, nnz):
    """Synthetic scalability workload of Section 4.3: 3-way I x I x I uniform, coupled
    I x I matrix with |Omega_Y| = |Omega_X| / 10."""
    dims = (I, I, I)
    coords = unique_coords(rng, nnz, dims, ("uniform",) * 3)
    v = rng.random(nnz) * 4.0 + 1.0
    tr_i, tr_v, te_i, te_v = _split(rng, coords, v, 0.10)
    r, c = _sparse_matrix(rng, max(1, nnz // 10), I, I)
    cpl = [Coupled(0, I, r, c, rng.random(r.shape[0]))]
    hp = dict(lr0=0.001, mu=0.1, lambda_reg=0.1, lambda_m=1.0)
    return dims, (10, 10, 10), tr_i, tr_v, te_i, te_v, cpl, hp, f"scalability I={I} nnz={nnz}"


PRESETS = {
    "cfg0": _cfg0,
    "cfg1": _cfg1,
    "cfg1_small": _cfg1_small,
    "cfg1_tiny": _cfg1_tiny,
    "cfg2_j16": lambda rng: _cfg1(rng, (16, 16, 16)),
    "cfg2_j32": lambda rng: _cfg1(rng, (32, 32, 32)),
    "cfg2_small_j16": lambda rng: _cfg1_small(rng, (16, 16, 16)),
    "cfg2_small_j32": lambda rng: _cfg1_small(rng, (32, 32, 32)),
    "cfg2_tiny_j16": lambda rng: _cfg1_tiny(rng, (16, 16, 16)),
    "cfg3": _cfg3,
    "cfg4": _cfg4,
    "cfg4_small": lambda rng: _cfg4(rng, 10),
    "cfg4_tiny": lambda rng: _cfg4(rng, 1000),
    "cfg3_small": _cfg3_small,
    "cfg3_tiny": _cfg3_tiny,
}


def make_problem(name, seed=0, **kw):
    """Build a named synthetic problem.  ``scal:I:nnz`` gives the Section 4.3 workload."""
    rng = np.random.default_rng(seed)
    if name.startswith("scal:"):
        _, I, nnz = name.split(":")
        out = _scal(rng, int(I), int(nnz))
    else:
        out = PRESETS[name](rng, **kw)
    dims, J, tr_i, tr_v, te_i, te_v, cpl, hp, rec = out
    return Problem(name, tuple(int(d) for d in dims), tuple(int(j) for j in J),
                   tr_i, tr_v, te_i, te_v, cpl, hp, rec)


# ----------------------------------------------------------------------------- method draws

def init_params(prob, seed=1):
    """Random initial parameters (Algorithm 1 initialises "randomly"): factors and coupled
    factors ~ U(0,1); core ~ N(0, 3^N / prod J) so that a prediction has unit variance."""
    rng = np.random.default_rng(seed)
    N = prob.N
    J = prob.J
    sigma = np.sqrt(3.0 ** N / float(np.prod(J)))
    G = rng.standard_normal(J) * sigma
    U = [rng.random((d, j)) for d, j in zip(prob.dims, J)]
    V = [rng.random((c.K, J[c.mode])) for c in prob.coupled]
    return G, U, V


def union_order(prob, seed=2):
    """A seeded visiting order of the union of tensor train entries and coupled entries
    (Algorithm 1 visits them "in random order").  Items 0..nnz-1 are tensor entries;
    then the entries of each coupled matrix in turn."""
    rng = np.random.default_rng(seed)
    return rng.permutation(prob.n_union).astype(np.int64)
