"""Small seeded problems for the oracle pins (plain numpy; no method arithmetic)."""
import numpy as np


class Cpl:
    def __init__(self, mode, K, rows, cols, vals):
        self.mode, self.K, self.rows, self.cols, self.vals = mode, K, rows, cols, vals


class Prob:
    def __init__(self, dims, J, idx, val, coupled, hparams=None):
        self.dims, self.J = tuple(dims), tuple(J)
        self.train_idx, self.train_val = idx, val
        self.coupled = coupled
        self.hparams = hparams or {}


def random_problem(dims, J, nnz, n_coupled=1, seed=0, zero_free=False, coupled_nnz=None,
                   coupled_mode=0, K=7):
    rng = np.random.default_rng(seed)
    cells = int(np.prod(dims))
    flat = rng.choice(cells, size=nnz, replace=False)
    idx = np.stack(np.unravel_index(flat, dims)).astype(np.int32)
    val = rng.normal(size=nnz) + 2.0
    cpl = []
    for m in range(n_coupled):
        cn = coupled_nnz or max(1, nnz // 2)
        mode = (coupled_mode + m) % len(dims)
        f = rng.choice(dims[mode] * K, size=min(cn, dims[mode] * K), replace=False)
        r, c = np.unravel_index(f, (dims[mode], K))
        cpl.append(Cpl(mode, K, r.astype(np.int32), c.astype(np.int32), rng.normal(size=r.shape[0])))
    G = rng.normal(size=J)
    U = [rng.random((d, j)) + (0.1 if zero_free else 0.0) for d, j in zip(dims, J)]
    V = [rng.random((c.K, J[c.mode])) + (0.1 if zero_free else 0.0) for c in cpl]
    if zero_free:
        G = np.where(np.abs(G) < 0.05, 0.05, G)
    return Prob(dims, J, idx, val, cpl), (G, U, V)


def dense_tucker(G, U):
    """G x_1 U1 x_2 U2 ... x_N UN by successive mode products (numpy tensordot)."""
    X = G
    for n, u in enumerate(U):
        X = np.moveaxis(np.tensordot(u, X, axes=([1], [n])), 0, n)
    return X
