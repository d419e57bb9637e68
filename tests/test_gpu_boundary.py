"""The C-ABI boundary against the FP64 oracle where the earlier parity tests do not reach:
the gradient with caller weights (s3_gradient's w), the gradient pass split into many
chunks (small ragged chunks, and the full-size cfg1 pass of 14 chunks checked on sampled
rows), and out-of-range indices in the caller's device memory, which the forward kernel
must catch (S3_ERR_INDEX, no parameter read with them, the context still usable).

Tolerance: 1e-5 relative, norm-wise and element-wise with a floor of 1e-6 of the largest
reference value (FP32 arithmetic, compensated FP32 sums, as in the other parity tests)."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
from paper_1708_08640_gb300 import synth
from tests.gpu_common import assert_close_blocks, f32, fp32_params, fp32_problem, make_pair, rel

pytestmark = pytest.mark.gpu


def as_np(t):
    return t.detach().cpu().double().numpy()


@pytest.mark.parametrize("name", ["cfg0", "cfg3_tiny"])
def test_weighted_gradient_matches_oracle(cuda_lib, name):
    """s3_gradient with per-entry weights w (train-entry order) in place of -e."""
    p = synth.make_problem(name)
    gpu, orc, q, _ = make_pair(p)
    w = f32(np.random.default_rng(3).normal(size=q.nnz))
    dG, dU, dV = gpu.gradient(w=torch.tensor(w, dtype=torch.float32, device="cuda"))
    gG, gU, gV = orc.full_gradient(w=w)
    assert_close_blocks(as_np(dG), gG, 1e-5, 1e-6, "dG")
    for n in range(p.N):
        assert_close_blocks(as_np(dU[n]), gU[n], 1e-5, 1e-6, f"dU{n}")
    for m in range(len(p.coupled)):
        assert_close_blocks(as_np(dV[m]), gV[m], 1e-5, 1e-6, f"dV{m}")
    # w = -e (the errors at the current parameters, from the oracle) gives the loss gradient
    e = q.train_val - orc.predict(q.train_idx.astype(np.int32))
    dG2, dU2, _ = gpu.gradient(w=torch.tensor(f32(-e), dtype=torch.float32, device="cuda"))
    gG0, gU0, _ = orc.full_gradient()
    assert_close_blocks(as_np(dG2), gG0, 1e-5, 1e-6, "dG(w=-e)")
    for n in range(p.N):
        assert_close_blocks(as_np(dU2[n]), gU0[n], 1e-5, 1e-6, f"dU{n}(w=-e)")
    gpu.close()


@pytest.mark.parametrize("name,chunk", [("cfg1_tiny", 10007), ("cfg3_tiny", 4099), ("cfg0", 1000)])
def test_gradient_over_many_chunks_matches_oracle(cuda_lib, name, chunk):
    """The gradient pass in chunks of `chunk` items (ragged last chunk): the compensated
    sums carried from chunk to chunk give the oracle's gradient."""
    p = synth.make_problem(name)
    gpu, orc, q, _ = make_pair(p, grad_chunk=chunk)
    n_chunks = -(-p.n_union // chunk)
    assert n_chunks >= 8
    dG, dU, dV = gpu.gradient()
    gG, gU, gV = orc.full_gradient()
    assert_close_blocks(as_np(dG), gG, 1e-5, 1e-6, "dG")
    for n in range(p.N):
        assert_close_blocks(as_np(dU[n]), gU[n], 1e-5, 1e-6, f"dU{n}")
    for m in range(len(p.coupled)):
        assert_close_blocks(as_np(dV[m]), gV[m], 1e-5, 1e-6, f"dV{m}")
    # the same gradient as one chunk, up to FP32 summation order
    one, _, _, _ = make_pair(p)
    dG1, dU1, _ = one.gradient()
    assert rel(as_np(dG), as_np(dG1)) <= 1e-5
    gpu.close()
    one.close()


def _rows_subproblem(q, mode_rows, cpl_rows, cpl_cols):
    """The tensor entries that touch the sampled rows (mode -> rows) and the coupled
    entries that touch the sampled rows of U^(c) or of V (numpy selection; the oracle's
    gradient of those rows over this subset equals its gradient over the whole data: a
    row's data terms come from the entries that touch it, and its regulariser sums to
    lambda_reg times the row)."""
    import copy
    keep = np.zeros(q.nnz, dtype=bool)
    for n, rows in mode_rows.items():
        keep |= np.isin(q.train_idx[n], rows)
    s = copy.copy(q)
    s.train_idx = q.train_idx[:, keep]
    s.train_val = q.train_val[keep]
    s.coupled = []
    for m, c in enumerate(q.coupled):
        k = np.isin(c.rows, cpl_rows.get(m, [])) | np.isin(c.cols, cpl_cols.get(m, []))
        s.coupled.append(synth.Coupled(c.mode, c.K, c.rows[k], c.cols[k], c.vals[k]))
    return s


def test_full_size_gradient_on_sampled_rows(cuda_lib, rating_tensor):
    """cfg1 at full size (9M train entries, 5M coupled entries, J = 10): the pass runs in 4
    chunks of 2^22 items (the default), as in the bench.  Sampled rows of every factor (rows
    of modest count, and the hottest row of modes 2 and 3) against the oracle's gradient of
    the same rows, computed from the entries that touch them."""
    p = rating_tensor
    q = fp32_problem(p)
    params = fp32_params(synth.init_params(p, 1))
    from paper_1708_08640_gb300.model import S3CMTF
    gpu = S3CMTF.from_problem(q, order=synth.union_order(p, 2))
    gpu.set_params(*params)
    assert -(-p.n_union // (1 << 22)) == 4
    dG, dU, dV = gpu.gradient()
    rng = np.random.default_rng(11)
    mode_rows = {}
    for n, k in [(0, 12), (1, 8), (2, 2)]:
        cnt = np.bincount(q.train_idx[n], minlength=p.dims[n])
        cand = np.nonzero((cnt > 0) & (cnt <= np.median(cnt[cnt > 0])))[0]
        rows = list(rng.choice(cand, size=k, replace=False))
        if n > 0:
            rows.append(int(np.argmax(cnt)))         # the hottest row of the mode
        mode_rows[n] = np.array(sorted(set(rows)))
    c = q.coupled[0]
    vcnt = np.bincount(c.cols, minlength=c.K)
    vrows = rng.choice(np.nonzero((vcnt > 0) & (vcnt < 500))[0], size=6, replace=False)
    sub = _rows_subproblem(q, mode_rows, {0: mode_rows[0]}, {0: vrows})
    orc = oracle.Oracle(sub, **{k: v for k, v in p.hparams.items()
                               if k in ("lr0", "mu", "lambda_reg", "lambda_m")})
    orc.set_params(*params)
    _, gU, gV = orc.full_gradient()
    for n, rows in mode_rows.items():
        got = as_np(dU[n])[rows]
        ref = gU[n][rows]
        for r, a, b in zip(rows, got, ref):
            assert rel(a, b) <= 1e-5, (n, r, rel(a, b))
    got = as_np(dV[0])[vrows]
    for r, a, b in zip(vrows, got, gV[0][vrows]):
        assert rel(a, b) <= 1e-5, ("V", r, rel(a, b))
    gpu.close()


def test_out_of_range_device_indices_are_caught(cuda_lib):
    """Device-resident coordinates outside [0, I_n) (too large, negative) given to
    s3_predict and to the device-pointer s3_rmse: the kernel reads no row for them and the
    call returns S3_ERR_INDEX; the context stays usable and valid calls still agree with the
    oracle."""
    from paper_1708_08640_gb300 import _lib as L
    p = synth.make_problem("cfg0")
    gpu, orc, q, _ = make_pair(p)
    lib = gpu.lib
    dev = torch.device("cuda")
    rng = np.random.default_rng(4)
    n = 777
    idx = np.stack([rng.integers(0, d, n) for d in p.dims]).astype(np.int32)
    for mode, badv in [(0, p.dims[0]), (2, -1), (1, 2 ** 31 - 1)]:
        bad = idx.copy()
        bad[mode, 500] = badv
        idx_d = [torch.tensor(bad[k], device=dev) for k in range(3)]
        out = torch.zeros(n, dtype=torch.float32, device=dev)
        st = lib.s3_predict(gpu.ctx, L.ptr_array([a.data_ptr() for a in idx_d]), n, out.data_ptr())
        assert st == L.S3_ERR_INDEX, st
        assert b"outside" in lib.s3_last_error(gpu.ctx)
        o = as_np(out)
        assert np.isnan(o[500]) and np.isfinite(np.delete(o, 500)).all()
        val_d = torch.zeros(n, dtype=torch.float32, device=dev)
        t = L.s3_coo_tensor(3, gpu._dims_arr, n, L.ptr_array([a.data_ptr() for a in idx_d]),
                            val_d.data_ptr())
        r = C.c_double(-1.0)
        st = lib.s3_rmse(gpu.ctx, C.byref(t), 1, C.byref(r))
        assert st == L.S3_ERR_INDEX and r.value == -1.0
    # the context is still usable
    got = gpu.predict(idx).cpu().double().numpy()
    assert_close_blocks(got, orc.predict(idx), 1e-5, 1e-6, "predict after the rejections")
    assert rel(gpu.loss()[0], orc.loss()[0]) <= 1e-5
    gpu.close()
