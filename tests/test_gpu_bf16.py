"""The HOGWILD epoch kernels against the oracle on problems that fit one tile (then an epoch
is one deterministic group step: every gradient at the start parameters, rows summed, the
core's mean step), and the BF16 tensor-core form against the FP32 form on a rating tensor.

Tolerances: the FP32 kernel within 1e-5 (plus FP32 storage rounding); the BF16 kernel
within 3e-2 relative on the step (its tensor-core operands a3, G, a1 o a2 and e a3 are
rounded to BF16: 8 significant bits, relative error 2^-9 per operand, a few operands per
product) and within 1% on the test RMSE per epoch."""
import numpy as np
import pytest

import oracle
from paper_1708_08640_gb300 import synth
from tests.gpu_common import assert_step_close, f32, fp32_params, make_pair, rel
from tests.oracle_cases import random_problem

pytestmark = pytest.mark.gpu


def one_tile_problem(J, seed=4, nnz=120, dims=(30, 20, 10)):
    # 120 entries: one tile of the FP32 kernel (128 entries, two lanes each) and of the
    # BF16 kernel (128 entries); 60 entries: one tile of 64 (four lanes each); 4-way
    # tensors: one lane per entry, tiles of up to 256
    N = len(dims)
    prob, params = random_problem(dims, (J,) * N, nnz=nnz, n_coupled=1, seed=seed,
                                  coupled_nnz=nnz // 3, K=9)
    prob.train_val = f32(prob.train_val + 2.0)
    for c in prob.coupled:
        c.vals = f32(c.vals)
    G, U, V = params
    G = G * np.sqrt(3.0 ** N / J ** N)
    return prob, fp32_params((G, U, V))


def run_one_tile(prob, params, precision, lr0=0.01, tile=128):
    from paper_1708_08640_gb300.model import S3CMTF
    hp = dict(lr0=lr0, mu=0.0, lambda_reg=0.1, lambda_m=2.0, core_scale=1.0)
    cpl = [(c.mode, c.K, c.rows, c.cols, c.vals) for c in prob.coupled]
    # one tile (128 entries: the FP32 kernel's largest, on two lanes) on one CTA (the BF16
    # form's tile then holds the same 128) and no staleness scaling: with one tile nothing
    # is stale, and the oracle's group step is the plain one
    gpu = S3CMTF(prob.dims, prob.J, prob.train_idx, prob.train_val, cpl, hog_staleness=-1.0,
                 hog_tile=tile, hog_ctas=1, **hp)
    gpu.set_params(*params)
    gpu.epoch("hogwild", precision)
    G, U, V = gpu.get_params()
    orc = oracle.Oracle(prob, **hp)
    orc.set_params(*params)
    n_union = prob.train_val.shape[0] + sum(c.rows.shape[0] for c in prob.coupled)
    orc.epoch_minibatch(0, np.arange(n_union), batch=n_union)
    return (G, U, V), orc


@pytest.mark.parametrize("J,tile,nnz,dims", [
    (5, 128, 120, (30, 20, 10)), (16, 128, 120, (30, 20, 10)), (10, 64, 60, (30, 20, 10)),
    (20, 128, 120, (30, 20, 10)), (32, 64, 60, (30, 20, 10)),
    (8, 256, 200, (12, 10, 8, 6)), (7, 256, 256, (12, 10, 8, 6))])
def test_fp32_hogwild_single_tile_is_group_step(cuda_lib, J, tile, nnz, dims):
    """1e-4 for the core: the HOGWILD kernel sums a tile's core gradients in plain FP32 (the
    minibatch kernels compensate theirs); 1e-5 for the rows.  3-way tiles of 128 entries
    run two lanes per entry, tiles of 64 four (ranks 5, 10, 16, 20 and 32: every 3-way
    instantiation the default launches use; rank 32 takes tiles of at most 64, its core
    fills most of shared memory); 4-way tiles (rank 8, and rank 7 padded to 8, a full tile
    of 256) one lane per entry."""
    prob, params = one_tile_problem(J, nnz=nnz, dims=dims)
    (G, U, V), orc = run_one_tile(prob, params, "fp32", tile=tile)
    G0, U0, V0 = params
    assert_step_close(G.cpu().double().numpy(), orc.G, G0, 1e-4, "G")
    for n in range(len(dims)):
        assert_step_close(U[n].cpu().double().numpy(), orc.U[n], U0[n], 1e-5, f"U{n}")
    assert_step_close(V[0].cpu().double().numpy(), orc.V[0], V0[0], 1e-5, "V")


@pytest.mark.parametrize("J", [16, 24, 10, 20])
def test_bf16_hogwild_single_tile_step(cuda_lib, J):
    """J = 16: rank 16 as is; J = 24: the layout's rank 32 with zero padding; J = 10 and 20:
    layouts of rank 10 and 20 (rows of 12 and 20 floats) extended to 16 and 32 inside the
    kernel."""
    prob, params = one_tile_problem(J)
    (G, U, V), orc = run_one_tile(prob, params, "bf16")
    G0, U0, V0 = params
    errs = {}
    for name, got, ref, old in ([("G", G, orc.G, G0)]
                                + [(f"U{n}", U[n], orc.U[n], U0[n]) for n in range(3)]
                                + [("V", V[0], orc.V[0], V0[0])]):
        d_got = got.cpu().double().numpy() - old
        d_ref = ref - old
        errs[name] = rel(d_got, d_ref)
    print("BF16 step relative error per parameter block:", errs)
    assert max(errs.values()) < 3e-2, errs


@pytest.mark.parametrize("J", [16, 32])
def test_bf16_rmse_tracks_fp32_on_rating_tensor(cuda_lib, rating_tensor, J):
    """cfg2 data at J = 16 and 32 (the cfg1 rating tensor): the BF16 form's test RMSE per
    epoch within 1% of the FP32 form's (both HOGWILD, same data, start and order)."""
    from paper_1708_08640_gb300.model import S3CMTF
    q = synth.with_rank(rating_tensor, (J, J, J))
    init = synth.init_params(q, 1)
    order = synth.union_order(q, 2)
    curves = {}
    for prec in ("fp32", "bf16"):
        m = S3CMTF.from_problem(q, order=order)
        m.set_params(*init)
        m.set_test(q.test_idx, q.test_val)
        out = []
        for t in range(3):
            try:
                m.epoch("hogwild", prec)
            except Exception as exc:
                raise AssertionError(f"{prec} epoch {t}: {exc}") from exc
            out.append(m.rmse())
        curves[prec] = out
        m.close()
    print(curves)
    for x, y in zip(curves["fp32"], curves["bf16"]):
        assert abs(y - x) / x <= 0.01
