"""Pins of the FP64 oracle against things other than itself: a dense reconstruction by
mode products, special cases that reduce to matrix algebra, symbolic differentiation,
central finite differences, algebraic identities between its routes, and recovery of a
planted model to its noise floor.  CPU only."""
import numpy as np
import pytest

import oracle
from tests.oracle_cases import Cpl, Prob, dense_tucker, random_problem


def make(prob, params, **hp):
    o = oracle.Oracle(prob, **hp)
    o.set_params(*params)
    return o


# ------------------------------------------------------------------ Eq. (4): prediction
@pytest.mark.parametrize("dims,J", [((7, 6, 5), (2, 3, 4)), ((5, 4, 3, 3), (2, 2, 3, 2))])
def test_predict_equals_dense_reconstruction(dims, J):
    prob, params = random_problem(dims, J, nnz=20, seed=1)
    o = make(prob, params)
    G, U, _ = params
    X = dense_tucker(G, U)                      # Tucker model of Section 2.2, matrix form
    cells = np.stack(np.unravel_index(np.arange(X.size), dims)).astype(np.int32)
    np.testing.assert_allclose(o.predict(cells), X.ravel(), rtol=1e-12, atol=1e-12)


def test_predict_cfg0_all_cells():
    """Brute force over all 200k cells of a 100x100x20 tensor with a 5x5x5 core."""
    prob, params = random_problem((100, 100, 20), (5, 5, 5), nnz=50, seed=2)
    o = make(prob, params)
    X = dense_tucker(params[0], params[1])
    cells = np.stack(np.unravel_index(np.arange(X.size), X.shape)).astype(np.int32)
    np.testing.assert_allclose(o.predict(cells), X.ravel(), rtol=1e-12, atol=1e-12)


def test_predict_order2_is_bilinear_form():
    rng = np.random.default_rng(3)
    dims, J = (9, 8), (3, 4)
    idx = np.stack(np.unravel_index(np.arange(72), dims)).astype(np.int32)
    prob = Prob(dims, J, idx, np.zeros(72), [])
    G = rng.normal(size=J)
    U = [rng.random((9, 3)), rng.random((8, 4))]
    o = make(prob, (G, U, []))
    expect = U[0] @ G @ U[1].T                 # x~_{i1 i2} = u1^T G u2
    np.testing.assert_allclose(o.predict(idx), expect.ravel(), rtol=1e-12)


def test_predict_hyperdiagonal_core_is_cp():
    """Section 2.2: a hyper-diagonal core with equal ranks gives the CP model."""
    rng = np.random.default_rng(4)
    dims, R = (6, 5, 4), 3
    G = np.zeros((R, R, R))
    lam = rng.normal(size=R)
    for r in range(R):
        G[r, r, r] = lam[r]
    U = [rng.random((d, R)) for d in dims]
    idx = np.stack(np.unravel_index(np.arange(120), dims)).astype(np.int32)
    o = make(Prob(dims, (R,) * 3, idx, np.zeros(120), []), (G, U, []))
    cp = np.einsum("r,ir,jr,kr->ijk", lam, *U)
    np.testing.assert_allclose(o.predict(idx), cp.ravel(), rtol=1e-12)


# ------------------------------------------------------------------ Eq. (3): partial products
def test_partials_are_derivatives_of_prediction():
    """G x_{-n} {u} is the derivative of the (multilinear) prediction w.r.t. row n, and
    its dot product with row n gives the prediction back."""
    prob, params = random_problem((5, 4, 3, 3), (2, 3, 2, 3), nnz=10, seed=5)
    o = make(prob, params)
    alpha = np.array([1, 2, 0, 2], dtype=np.int32)
    parts = o.partials(alpha)
    xt = o.predict(alpha.reshape(4, 1))[0]
    G, U, V = params
    for n in range(4):
        assert np.dot(parts[n], U[n][alpha[n]]) == pytest.approx(xt, rel=1e-12)
        for k in range(prob.J[n]):
            Up = [u.copy() for u in U]
            Um = [u.copy() for u in U]
            h = 1e-4
            Up[n][alpha[n], k] += h
            Um[n][alpha[n], k] -= h
            o.set_params(G, Up, V)
            fp = o.predict(alpha.reshape(4, 1))[0]
            o.set_params(G, Um, V)
            fm = o.predict(alpha.reshape(4, 1))[0]
            assert (fp - fm) / (2 * h) == pytest.approx(parts[n][k], rel=1e-9, abs=1e-12)
        o.set_params(G, U, V)


# ------------------------------------------------------------------ Eq. (7): the objective
def test_loss_forms_agree_and_match_numpy():
    prob, params = random_problem((8, 7, 6), (3, 2, 4), nnz=60, seed=6)
    hp = dict(lambda_reg=0.3, lambda_m=2.5)
    o = make(prob, params, **hp)
    f, se, sy = o.loss()
    assert o.loss_rowform() == pytest.approx(f, rel=1e-12)
    # the same number from a dense reconstruction and plain norms
    G, U, V = params
    X = dense_tucker(G, U)
    pred = X[tuple(prob.train_idx)]
    se_np = np.sum((prob.train_val - pred) ** 2)
    assert se == pytest.approx(se_np, rel=1e-12)
    reg = np.sum(G ** 2)
    for n in range(3):
        touched = np.unique(prob.train_idx[n])
        reg += np.sum(U[n][touched] ** 2)
    c = prob.coupled[0]
    e_y = c.vals - np.sum(U[c.mode][c.rows] * V[0][c.cols], axis=1)
    rv = np.sum(V[0][np.unique(c.cols)] ** 2)
    f_np = 0.5 * se_np + 0.5 * hp["lambda_reg"] * reg + 0.5 * hp["lambda_m"] * (
        np.sum(e_y ** 2) + hp["lambda_reg"] * rv)
    assert f == pytest.approx(f_np, rel=1e-12)
    assert sy[0] == pytest.approx(np.sum(e_y ** 2), rel=1e-12)


def test_rmse_definition():
    prob, params = random_problem((6, 6, 6), (2, 2, 2), nnz=30, seed=7)
    o = make(prob, params)
    X = dense_tucker(params[0], params[1])
    rng = np.random.default_rng(0)
    idx = rng.integers(0, 6, size=(3, 40)).astype(np.int32)
    val = rng.normal(size=40)
    expect = np.sqrt(np.mean((val - X[tuple(idx)]) ** 2))
    assert o.rmse(idx, val) == pytest.approx(expect, rel=1e-12)


# ------------------------------------------------------------------ Eq. (8): gradients
@pytest.mark.parametrize("dims,J,ncpl", [((6, 5, 4), (2, 3, 2), 1), ((5, 4, 3, 3), (2, 2, 3, 2), 2),
                                        ((7, 5, 4), (3, 3, 3), 0)])
def test_full_gradient_central_differences(dims, J, ncpl):
    prob, params = random_problem(dims, J, nnz=35, n_coupled=ncpl, seed=8, coupled_nnz=15)
    hp = dict(lambda_reg=0.2, lambda_m=1.7)
    o = make(prob, params, **hp)
    gG, gU, gV = o.full_gradient()
    G, U, V = params
    rng = np.random.default_rng(1)

    def f_at(G_, U_, V_):
        o.set_params(G_, U_, V_)
        return o.loss()[0]

    checks = []
    for l in rng.choice(G.size, size=min(G.size, 10), replace=False):
        checks.append(("G", None, np.unravel_index(l, G.shape)))
    for n in range(len(dims)):
        for _ in range(6):
            checks.append(("U", n, (rng.integers(dims[n]), rng.integers(J[n]))))
    for m in range(ncpl):
        for _ in range(6):
            checks.append(("V", m, (rng.integers(V[m].shape[0]), rng.integers(V[m].shape[1]))))
    for kind, k, pos in checks:
        Gp, Up, Vp = G.copy(), [u.copy() for u in U], [v.copy() for v in V]
        Gm, Um, Vm = G.copy(), [u.copy() for u in U], [v.copy() for v in V]
        tgt_p = Gp if kind == "G" else (Up[k] if kind == "U" else Vp[k])
        tgt_m = Gm if kind == "G" else (Um[k] if kind == "U" else Vm[k])
        x = tgt_p[pos]
        h = 1e-6 * max(1.0, abs(x))
        tgt_p[pos] += h
        tgt_m[pos] -= h
        fd = (f_at(Gp, Up, Vp) - f_at(Gm, Um, Vm)) / (2 * h)
        an = gG[pos] if kind == "G" else (gU[k][pos] if kind == "U" else gV[k][pos])
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-7), (kind, k, pos)


@pytest.mark.parametrize("dims,J,ncpl", [((6, 5, 4), (2, 3, 2), 1), ((5, 4, 3, 3), (2, 2, 3, 2), 2)])
def test_weighted_gradient_central_differences(dims, J, ncpl):
    """Per-entry weights w in place of -e: the gradient of
    F = sum_alpha w_alpha x~_alpha + (f - 1/2 sum_alpha e_alpha^2), i.e. the data term made
    linear in the predictions with the regularisers and coupled terms of Eq. (7) kept; F is
    evaluated from the pinned prediction and loss routines.  With w = -e it is the gradient
    of f itself."""
    prob, params = random_problem(dims, J, nnz=35, n_coupled=ncpl, seed=18, coupled_nnz=15)
    hp = dict(lambda_reg=0.3, lambda_m=1.3)
    o = make(prob, params, **hp)
    rng = np.random.default_rng(5)
    w = rng.normal(size=prob.train_val.shape[0])
    gG, gU, gV = o.full_gradient(w=w)
    G, U, V = params
    idx, x = prob.train_idx.astype(np.int32), prob.train_val

    def F_at(G_, U_, V_):
        o.set_params(G_, U_, V_)
        xt = o.predict(idx)
        return float(np.dot(w, xt) + o.loss()[0] - 0.5 * np.sum((x - xt) ** 2))

    checks = [("G", None, np.unravel_index(l, G.shape))
              for l in rng.choice(G.size, size=min(G.size, 8), replace=False)]
    for n in range(len(dims)):
        for _ in range(5):
            checks.append(("U", n, (rng.integers(dims[n]), rng.integers(J[n]))))
    for m in range(ncpl):
        for _ in range(5):
            checks.append(("V", m, (rng.integers(V[m].shape[0]), rng.integers(V[m].shape[1]))))
    for kind, k, pos in checks:
        Gp, Up, Vp = G.copy(), [u.copy() for u in U], [v.copy() for v in V]
        Gm, Um, Vm = G.copy(), [u.copy() for u in U], [v.copy() for v in V]
        tgt_p = Gp if kind == "G" else (Up[k] if kind == "U" else Vp[k])
        tgt_m = Gm if kind == "G" else (Um[k] if kind == "U" else Vm[k])
        h = 1e-6 * max(1.0, abs(tgt_p[pos]))
        tgt_p[pos] += h
        tgt_m[pos] -= h
        fd = (F_at(Gp, Up, Vp) - F_at(Gm, Um, Vm)) / (2 * h)
        an = gG[pos] if kind == "G" else (gU[k][pos] if kind == "U" else gV[k][pos])
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-7), (kind, k, pos)
    # w = -e reproduces the gradient of f
    o.set_params(*params)
    e = x - o.predict(idx)
    for a, b in zip([*o.full_gradient(w=-e)], [*o.full_gradient()]):
        for u, v in zip(a if isinstance(a, list) else [a], b if isinstance(b, list) else [b]):
            np.testing.assert_allclose(u, v, rtol=1e-12, atol=1e-13)


def test_untouched_rows_have_zero_gradient():
    prob, params = random_problem((10, 4, 4), (2, 2, 2), nnz=6, n_coupled=0, seed=9)
    o = make(prob, params, lambda_reg=0.5)
    _, gU, _ = o.full_gradient()
    untouched = np.setdiff1d(np.arange(10), prob.train_idx[0])
    assert untouched.size > 0
    assert np.all(gU[0][untouched] == 0.0)


def test_entry_gradients_sum_to_full_gradient():
    prob, params = random_problem((6, 5, 4), (2, 3, 2), nnz=25, n_coupled=0, seed=10)
    o = make(prob, params, lambda_reg=0.4)
    gG, gU, _ = o.full_gradient()
    sG = np.zeros_like(gG)
    sU = [np.zeros_like(u) for u in gU]
    for e in range(25):
        _, gu, g = o.entry_gradient(e)
        sG += g
        for n in range(3):
            sU[n][prob.train_idx[n][e]] += gu[n]
    np.testing.assert_allclose(sG, gG, rtol=1e-12, atol=1e-12)
    for n in range(3):
        np.testing.assert_allclose(sU[n], gU[n], rtol=1e-12, atol=1e-12)


def test_opt_route_equals_naive_route():
    """Lemma 2 / Lemma 3 (Section 3.5): S, Collapse and element-wise division give the
    same per-entry gradients as Eq. (8) on inputs without zeros."""
    prob, params = random_problem((6, 5, 4, 3), (2, 3, 2, 2), nnz=12, n_coupled=0, seed=11,
                                  zero_free=True)
    o = make(prob, params, lambda_reg=0.3)
    for e in range(12):
        e1, gu1, gG1 = o.entry_gradient(e)
        e2, gu2, gG2 = o.entry_gradient_opt(e)
        assert e1 == pytest.approx(e2, rel=1e-12)
        for a, b in zip(gu1, gu2):
            np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(gG1, gG2, rtol=1e-10, atol=1e-12)


def test_rank_one_sgd_step_by_symbolic_differentiation():
    """J = 1: one sequential step over a tensor entry then a coupled entry, with the
    gradients obtained by sympy from the scalar per-entry objective."""
    sympy = pytest.importorskip("sympy")
    g, a, b, c, w = sympy.symbols("g a b c w")
    x, y, lam, lm, eta = 3.1, -0.7, 0.3, 2.0, 0.05
    vals = {g: 0.9, a: 0.4, b: -1.3, c: 0.8, w: 0.6}
    # per-entry terms of f (Eq. (7)); |Omega| = 1 and every count is 1
    f_alpha = sympy.Rational(1, 2) * ((x - g * a * b * c) ** 2 + lam * g ** 2 + lam * (a ** 2 + b ** 2 + c ** 2))
    f_beta = lm / 2 * ((y - a * w) ** 2 + lam * w ** 2)
    step1 = {s: float(vals[s] - eta * sympy.diff(f_alpha, s).subs(vals)) for s in (g, a, b, c)}
    step1[w] = vals[w]
    step2 = dict(step1)
    for s in (a, w):
        step2[s] = float(step1[s] - eta * sympy.diff(f_beta, s).subs(step1))
    idx = np.zeros((3, 1), dtype=np.int32)
    prob = Prob((1, 1, 1), (1, 1, 1), idx, np.array([x]),
                [Cpl(0, 1, np.zeros(1, np.int32), np.zeros(1, np.int32), np.array([y]))])
    o = make(prob, (np.array([[[0.9]]]), [np.array([[0.4]]), np.array([[-1.3]]), np.array([[0.8]])],
                    [np.array([[0.6]])]), lambda_reg=lam, lambda_m=lm, lr0=eta, mu=0.0)
    o.epoch_sequential(0, np.array([0, 1]))
    G, U, V = o.get_params()
    assert G.ravel()[0] == pytest.approx(step2[g], rel=1e-13)
    assert U[0][0, 0] == pytest.approx(step2[a], rel=1e-13)
    assert U[1][0, 0] == pytest.approx(step2[b], rel=1e-13)
    assert U[2][0, 0] == pytest.approx(step2[c], rel=1e-13)
    assert V[0][0, 0] == pytest.approx(step2[w], rel=1e-13)


# ------------------------------------------------------------------ Alg. 1 and the minibatch rule
def test_learning_rate_schedule():
    prob, params = random_problem((3, 3, 3), (1, 1, 1), nnz=3, n_coupled=0)
    o = make(prob, params, lr0=0.02, mu=0.1)
    assert o.learning_rate(0) == pytest.approx(0.02)
    assert o.learning_rate(5) == pytest.approx(0.02 / 1.5)


def test_minibatch_of_one_is_sequential():
    prob, params = random_problem((6, 5, 4), (2, 3, 2), nnz=40, n_coupled=1, seed=12,
                                  coupled_nnz=20)
    order = np.random.default_rng(0).permutation(60)
    a = make(prob, params, lr0=0.05, mu=0.1, lambda_reg=0.2, lambda_m=1.5)
    b = make(prob, params, lr0=0.05, mu=0.1, lambda_reg=0.2, lambda_m=1.5, batch=1)
    for t in range(2):
        a.epoch_sequential(t, order)
        b.epoch_minibatch(t, order)
    for x, y in zip([a.G] + a.U + a.V, [b.G] + b.U + b.V):
        np.testing.assert_allclose(x, y, rtol=1e-13, atol=1e-14)


def test_full_batch_is_a_gradient_step():
    prob, params = random_problem((6, 5, 4), (2, 3, 2), nnz=40, n_coupled=1, seed=13,
                                  coupled_nnz=20)
    hp = dict(lr0=0.03, mu=0.0, lambda_reg=0.2, lambda_m=1.5, core_scale=2.0)
    o = make(prob, params, **hp)
    gG, gU, gV = o.full_gradient()
    o.epoch_minibatch(0, np.arange(60), batch=60)
    G, U, V = params
    np.testing.assert_allclose(o.G, G - 0.03 * 2.0 * gG / 40, rtol=1e-12, atol=1e-14)
    for n in range(3):
        np.testing.assert_allclose(o.U[n], U[n] - 0.03 * gU[n], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(o.V[0], V[0] - 0.03 * gV[0], rtol=1e-12, atol=1e-14)


def test_minibatch_mean_rule_divides_by_row_hits():
    prob, params = random_problem((3, 3, 3), (2, 2, 2), nnz=12, n_coupled=0, seed=14)
    o = make(prob, params, lr0=0.03, mu=0.0, lambda_reg=0.1)
    _, gU, _ = o.full_gradient()
    o.epoch_minibatch(0, np.arange(12), batch=12, row_mean=1)
    hits = np.bincount(prob.train_idx[0], minlength=3)
    U0 = params[1][0]
    expect = U0 - 0.03 * gU[0] / np.maximum(hits, 1)[:, None]
    np.testing.assert_allclose(o.U[0], expect, rtol=1e-12, atol=1e-14)


def test_order_outside_union_is_rejected():
    prob, params = random_problem((3, 3, 3), (1, 1, 1), nnz=3, n_coupled=0)
    o = make(prob, params)
    with pytest.raises(ValueError):
        o.epoch_sequential(0, np.array([0, 1, 7]))


# ------------------------------------------------------------------ planted recovery
def test_recovers_planted_model_to_noise_floor():
    from paper_1708_08640_gb300 import synth
    p = synth.make_problem("cfg0")                   # noise sigma = 0.1
    o = oracle.Oracle(p, lr0=0.02, mu=0.0, lambda_reg=0.01, lambda_m=1.0)
    o.set_params(*synth.init_params(p, 1))
    order = synth.union_order(p, 2)
    for t in range(40):
        o.epoch_sequential(t, order)
    assert o.rmse(p.test_idx, p.test_val) <= 1.3 * 0.1


def test_noiseless_planted_model_train_error_goes_to_zero():
    from paper_1708_08640_gb300 import synth
    p = synth.make_problem("cfg0", noise=0.0)
    o = oracle.Oracle(p, lr0=0.02, mu=0.0, lambda_reg=0.0, lambda_m=1.0)
    o.set_params(*synth.init_params(p, 1))
    order = synth.union_order(p, 2)
    hist = []
    for t in range(50):
        o.epoch_sequential(t, order)
        hist.append(o.rmse(p.train_idx, p.train_val))
    assert np.all(np.diff(hist[15:]) < 0)
    assert hist[-1] < 0.01


# ------------------------------------------------------------------ Alg. 1: final QR step
@pytest.mark.parametrize("dims,J,ncpl", [((30, 20, 10), (4, 3, 2), 2), ((9, 8, 7, 6), (3, 2, 3, 2), 2)])
def test_finalize_qr_keeps_every_prediction(dims, J, ncpl):
    """Section 3.4: replacing U by Q, G by G x_n R and V by V R^T is the same factorisation:
    every tensor cell of the dense reconstruction and every coupled entry is unchanged."""
    prob, params = random_problem(dims, J, nnz=60, n_coupled=ncpl, seed=7)
    o = make(prob, params)
    X0 = dense_tucker(params[0], params[1])
    cpl0 = [o.predict_coupled(m, c.rows, c.cols) for m, c in enumerate(prob.coupled)]
    o.finalize_qr()
    G1, U1, _ = o.get_params()
    np.testing.assert_allclose(dense_tucker(G1, U1), X0, rtol=1e-11, atol=1e-12)
    for m, c in enumerate(prob.coupled):
        np.testing.assert_allclose(o.predict_coupled(m, c.rows, c.cols), cpl0[m], rtol=1e-11,
                                   atol=1e-12)


def test_finalize_qr_is_the_thin_qr_with_positive_diagonal():
    """U_old = Q R with Q^T Q = I and R upper triangular, diag(R) > 0: the same Q and R as
    numpy's (LAPACK) QR after its signs are made positive."""
    prob, params = random_problem((40, 25, 12), (5, 4, 3), nnz=50, n_coupled=1, seed=8)
    o = make(prob, params)
    Rs = o.finalize_qr()
    _, U1, _ = o.get_params()
    for n, (u0, q, r) in enumerate(zip(params[1], U1, Rs)):
        np.testing.assert_allclose(q.T @ q, np.eye(q.shape[1]), atol=1e-13)
        np.testing.assert_allclose(q @ r, u0, rtol=1e-12, atol=1e-13)
        assert np.all(np.tril(r, -1) == 0.0) and np.all(np.diag(r) > 0)
        ql, rl = np.linalg.qr(u0)
        s = np.sign(np.diag(rl))
        np.testing.assert_allclose(q, ql * s, atol=1e-12)
        np.testing.assert_allclose(r, s[:, None] * rl, atol=1e-12)


def test_finalize_qr_rank_one_by_hand():
    """J = 1: Q = u / |u|, R = |u|, so G becomes G |u1| |u2| |u3| and V becomes V |u_c|."""
    prob, params = random_problem((6, 5, 4), (1, 1, 1), nnz=10, n_coupled=1, seed=9)
    o = make(prob, params)
    G, U, V = params
    norms = [np.linalg.norm(u[:, 0]) for u in U]
    o.finalize_qr()
    G1, U1, V1 = o.get_params()
    np.testing.assert_allclose(G1.ravel(), G.ravel() * np.prod(norms), rtol=1e-13)
    for u, u1, nm in zip(U, U1, norms):
        np.testing.assert_allclose(u1[:, 0], u[:, 0] / nm, rtol=1e-13)
    np.testing.assert_allclose(V1[0], V[0] * norms[prob.coupled[0].mode], rtol=1e-13)


def test_finalize_qr_is_idempotent_and_rejects_rank_deficiency():
    prob, params = random_problem((20, 15, 10), (3, 3, 2), nnz=30, n_coupled=1, seed=10)
    o = make(prob, params)
    o.finalize_qr()
    p1 = o.get_params()
    for r in o.finalize_qr():                 # orthonormal factors: R = I
        np.testing.assert_allclose(r, np.eye(r.shape[0]), atol=1e-13)
    p2 = o.get_params()
    np.testing.assert_allclose(p2[0], p1[0], atol=1e-13)
    G, U, V = params
    U = [u.copy() for u in U]
    U[1][:, 2] = U[1][:, 0]                   # dependent columns
    o2 = make(prob, (G, U, V))
    with pytest.raises(ValueError):
        o2.finalize_qr()


# ------------------------------------------------------------------ S3CMTF-CP (Section 4.2)
def _cp_problem(seed=11, J=3):
    prob, (G, U, V) = random_problem((12, 10, 8), (J, J, J), nnz=40, n_coupled=1, seed=seed,
                                     coupled_nnz=20)
    lam = np.random.default_rng(seed).normal(size=J)
    G = np.zeros((J, J, J))
    G[np.arange(J), np.arange(J), np.arange(J)] = lam
    return prob, (G, U, V), lam


@pytest.mark.parametrize("nonneg", [0, 1])
def test_cp_sequential_epoch_follows_the_cp_formulas(nonneg):
    """S3CMTF-CP (hyper-diagonal core, Section 4.2): Algorithm 1 with the CP model written
    out directly in numpy: x~ = sum_j l_j prod_n a_n[j]; du_n = -e l o prod_{m!=n} a_m +
    (lambda_reg / c_n) a_n; dl = -e prod_n a_n + (lambda_reg / |Omega|) l; coupled as Eq. (8).
    nonneg = 1: each updated row and the diagonal then take max(0, .) (Section 5)."""
    prob, params, lam = _cp_problem()
    hp = dict(lr0=0.05, mu=0.0, lambda_reg=0.3, lambda_m=1.5, cp=1, nonneg=nonneg)
    proj = (lambda v: np.maximum(0.0, v)) if nonneg else (lambda v: v)
    clipped = 0
    o = make(prob, params, **hp)
    n_union = prob.train_val.shape[0] + prob.coupled[0].rows.shape[0]
    order = np.random.default_rng(5).permutation(n_union)
    o.epoch_sequential(0, order)
    G1, U1, V1 = o.get_params()
    # numpy CP reference
    _, U, V = params
    U = [u.copy() for u in U]
    V = [v.copy() for v in V]
    lam = lam.copy()
    idx, x = prob.train_idx, prob.train_val
    nnz = x.shape[0]
    cnt = [np.bincount(idx[n], minlength=prob.dims[n]) for n in range(3)]
    c = prob.coupled[0]
    cntY = np.bincount(c.cols, minlength=c.K)
    eta, lr, lm = hp["lr0"], hp["lambda_reg"], hp["lambda_m"]
    for it in order:
        if it < nnz:
            a = [U[n][idx[n, it]].copy() for n in range(3)]
            e = x[it] - np.sum(lam * a[0] * a[1] * a[2])
            for n in range(3):
                others = np.prod([a[m] for m in range(3) if m != n], axis=0)
                step = U[n][idx[n, it]] - eta * (-e * lam * others + lr / cnt[n][idx[n, it]] * a[n])
                clipped += int(np.sum(step < 0))
                U[n][idx[n, it]] = proj(step)
            step = lam - eta * (-e * a[0] * a[1] * a[2] + lr / nnz * lam)
            clipped += int(np.sum(step < 0))
            lam = proj(step)
        else:
            b = it - nnz
            u, v = U[c.mode][c.rows[b]].copy(), V[0][c.cols[b]].copy()
            e = c.vals[b] - u @ v
            su = U[c.mode][c.rows[b]] - eta * (-lm * e * v)
            sv = V[0][c.cols[b]] - eta * (-lm * e * u + lm * lr / cntY[c.cols[b]] * v)
            clipped += int(np.sum(su < 0) + np.sum(sv < 0))
            U[c.mode][c.rows[b]] = proj(su)
            V[0][c.cols[b]] = proj(sv)
    J = lam.shape[0]
    np.testing.assert_allclose(G1[np.arange(J), np.arange(J), np.arange(J)], lam, rtol=1e-12, atol=1e-14)
    off = G1.copy()
    off[np.arange(J), np.arange(J), np.arange(J)] = 0.0
    assert np.all(off == 0.0)
    for n in range(3):
        np.testing.assert_allclose(U1[n], U[n], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(V1[0], V[0], rtol=1e-12, atol=1e-14)
    if nonneg:
        assert clipped > 0 and min(G1.min(), V1[0].min(), *(u.min() for u in U1)) >= 0.0


def test_cp_full_gradient_is_the_diagonal_of_central_differences():
    prob, params, lam = _cp_problem(seed=12)
    o = make(prob, params, lambda_reg=0.2, lambda_m=1.3, cp=1)
    gG, _, _ = o.full_gradient()
    G, U, V = params
    J = lam.shape[0]
    for j in range(J):
        Gp, Gm = G.copy(), G.copy()
        h = 1e-6 * max(1.0, abs(G[j, j, j]))
        Gp[j, j, j] += h
        Gm[j, j, j] -= h
        o.set_params(Gp, U, V)
        fp = o.loss()[0]
        o.set_params(Gm, U, V)
        fm = o.loss()[0]
        assert gG[j, j, j] == pytest.approx((fp - fm) / (2 * h), rel=1e-6, abs=1e-7)
    off = gG.copy()
    off[np.arange(J), np.arange(J), np.arange(J)] = 0.0
    assert np.all(off == 0.0)


def test_cp_minibatch_keeps_the_core_hyperdiagonal():
    prob, params, lam = _cp_problem(seed=13)
    o = make(prob, params, lr0=0.02, lambda_reg=0.1, lambda_m=1.0, batch=16, core_scale=2.0, cp=1)
    n_union = prob.train_val.shape[0] + prob.coupled[0].rows.shape[0]
    for t in range(3):
        o.epoch_minibatch(t, np.arange(n_union))
    G1 = o.get_params()[0]
    J = lam.shape[0]
    diag = G1[np.arange(J), np.arange(J), np.arange(J)].copy()
    G1[np.arange(J), np.arange(J), np.arange(J)] = 0.0
    assert np.all(G1 == 0.0) and np.all(diag != lam)


# ------------------------------------------------------------------ non-negative form (Section 5)
# Section 5 fits a non-negative factorisation with the projected gradient method (Lin
# 2007): a gradient step followed by the projection onto the non-negative orthant,
# max(0, .) element by element.  These pins tie the oracle's nonneg = 1 path to sympy
# derivatives, to the pinned full gradient, and to the plain path where no projection binds.

def test_nonneg_rank_one_step_by_symbolic_differentiation():
    """J = 1: a tensor step that drives b below zero, then a coupled step that drives w
    below zero; each step is the sympy gradient step followed by max(0, .)."""
    sympy = pytest.importorskip("sympy")
    g, a, b, c, w = sympy.symbols("g a b c w")
    x, y, lam, lm, eta = -3.0, -2.0, 0.3, 2.0, 0.2
    vals = {g: 0.9, a: 0.4, b: 0.05, c: 0.8, w: 0.2}
    f_alpha = sympy.Rational(1, 2) * ((x - g * a * b * c) ** 2 + lam * g ** 2 + lam * (a ** 2 + b ** 2 + c ** 2))
    f_beta = lm / 2 * ((y - a * w) ** 2 + lam * w ** 2)
    raw1 = {s: float(vals[s] - eta * sympy.diff(f_alpha, s).subs(vals)) for s in (g, a, b, c)}
    step1 = {s: max(0.0, v) for s, v in raw1.items()}
    step1[w] = vals[w]
    raw2 = {s: float(step1[s] - eta * sympy.diff(f_beta, s).subs(step1)) for s in (a, w)}
    step2 = dict(step1)
    step2.update({s: max(0.0, v) for s, v in raw2.items()})
    # the example exercises both projections and leaves the other parameters inside
    assert raw1[b] < 0 and raw2[w] < 0
    assert min(raw1[g], raw1[a], raw1[c], raw2[a]) > 0
    idx = np.zeros((3, 1), dtype=np.int32)
    prob = Prob((1, 1, 1), (1, 1, 1), idx, np.array([x]),
                [Cpl(0, 1, np.zeros(1, np.int32), np.zeros(1, np.int32), np.array([y]))])
    o = make(prob, (np.array([[[0.9]]]), [np.array([[0.4]]), np.array([[0.05]]), np.array([[0.8]])],
                    [np.array([[0.2]])]), lambda_reg=lam, lambda_m=lm, lr0=eta, mu=0.0, nonneg=1)
    o.epoch_sequential(0, np.array([0, 1]))
    G, U, V = o.get_params()
    assert G.ravel()[0] == pytest.approx(step2[g], rel=1e-13)
    assert U[0][0, 0] == pytest.approx(step2[a], rel=1e-13)
    assert U[1][0, 0] == 0.0
    assert U[2][0, 0] == pytest.approx(step2[c], rel=1e-13)
    assert V[0][0, 0] == 0.0


@pytest.mark.parametrize("dims,J,ncpl", [((6, 5, 4), (2, 3, 2), 1), ((5, 4, 3, 3), (2, 2, 3, 2), 2)])
def test_nonneg_full_batch_is_a_projected_gradient_step(dims, J, ncpl):
    """One batch holding every item: each touched row and the core take max(0, theta -
    step * full gradient); rows no item touches keep their values (3-way with one coupled
    matrix, 4-way with two)."""
    prob, params = random_problem(dims, J, nnz=40, n_coupled=ncpl, seed=13, coupled_nnz=20)
    n_union = 40 + 20 * ncpl
    hp = dict(lr0=0.5, mu=0.0, lambda_reg=0.2, lambda_m=1.5, core_scale=2.0)
    o = make(prob, params, nonneg=1, **hp)
    gG, gU, gV = make(prob, params, **hp).full_gradient()
    o.epoch_minibatch(0, np.arange(n_union), batch=n_union)
    G, U, V = params
    eG = np.maximum(0.0, G - 0.5 * 2.0 * gG / 40)
    assert np.any(G - 0.5 * 2.0 * gG / 40 < 0) and np.any(eG > 0)
    np.testing.assert_allclose(o.G, eG, rtol=1e-12, atol=1e-14)
    clipped = 0
    for n in range(len(dims)):
        touched = np.zeros(prob.dims[n], bool)
        touched[prob.train_idx[n]] = True
        for c in prob.coupled:
            if n == c.mode:
                touched[c.rows] = True
        step = U[n] - 0.5 * gU[n]
        clipped += int(np.sum(step[touched] < 0))
        expect = np.where(touched[:, None], np.maximum(0.0, step), U[n])
        np.testing.assert_allclose(o.U[n], expect, rtol=1e-12, atol=1e-14)
    for m, c in enumerate(prob.coupled):
        tv = np.zeros(c.K, bool)
        tv[c.cols] = True
        step = V[m] - 0.5 * gV[m]
        clipped += int(np.sum(step[tv] < 0))
        np.testing.assert_allclose(o.V[m], np.where(tv[:, None], np.maximum(0.0, step), V[m]),
                                   rtol=1e-12, atol=1e-14)
    assert clipped > 0


def test_nonneg_equals_plain_where_no_projection_binds():
    """Non-negative parameters and values far above every prediction: each error is
    positive, every step keeps the parameters non-negative, and the projected epochs
    (sequential and minibatch) are the plain ones bit for bit."""
    prob, (G, U, V) = random_problem((6, 5, 4), (2, 3, 2), nnz=40, n_coupled=1, seed=15,
                                     coupled_nnz=20)
    rng = np.random.default_rng(3)
    prob.train_val[:] = 30.0 + rng.random(prob.train_val.shape[0])
    prob.coupled[0].vals[:] = 30.0 + rng.random(prob.coupled[0].vals.shape[0])
    params = (np.abs(G), U, V)
    hp = dict(lr0=0.002, mu=0.1, lambda_reg=0.2, lambda_m=1.5, core_scale=2.0, batch=16)
    order = np.random.default_rng(4).permutation(60)
    for epoch in ("epoch_sequential", "epoch_minibatch"):
        a = make(prob, params, **hp)
        b = make(prob, params, nonneg=1, **hp)
        for t in range(3):
            getattr(a, epoch)(t, order)
            getattr(b, epoch)(t, order)
        for x, y in zip([a.G] + a.U + a.V, [b.G] + b.U + b.V):
            assert np.array_equal(x, y)
        assert all(np.all(x >= 0) for x in [a.G] + a.U + a.V)


def test_nonneg_minibatch_of_one_is_sequential():
    prob, params = random_problem((6, 5, 4), (2, 3, 2), nnz=40, n_coupled=1, seed=16,
                                  coupled_nnz=20)
    order = np.random.default_rng(0).permutation(60)
    hp = dict(lr0=0.1, mu=0.1, lambda_reg=0.2, lambda_m=1.5, nonneg=1)
    a = make(prob, params, **hp)
    b = make(prob, params, batch=1, **hp)
    for t in range(2):
        a.epoch_sequential(t, order)
        b.epoch_minibatch(t, order)
    for x, y in zip([a.G] + a.U + a.V, [b.G] + b.U + b.V):
        np.testing.assert_allclose(x, y, rtol=1e-13, atol=1e-14)
    assert all(np.all(x >= 0) for x in [a.G] + a.U + a.V)
    # the projection binds on this example: the plain epochs leave negative parameters
    c = make(prob, params, **{k: v for k, v in hp.items() if k != "nonneg"})
    for t in range(2):
        c.epoch_sequential(t, order)
    assert np.any(c.G < 0) and np.any(c.V[0] < 0) and np.any(a.V[0] == 0)
