"""s3_rmse_noalloc serves callers that must not allocate device memory while they run: a
process whose memory pool has reserved the whole device, a job held to a device-memory
budget fixed up front, or a serving loop that cannot take the synchronisation a cudaMalloc
may cause.  From its static scratch alone it must give the test RMSE of s3_rmse and of the
FP64 oracle, call after call, and reject what it cannot hold.  Collected last on purpose
(file name), so a failure here comes after every other test."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1708_08640_gb300 import _lib as L
from paper_1708_08640_gb300 import synth
from tests.gpu_common import make_pair

pytestmark = pytest.mark.gpu


def _noalloc(lib, model, idx_d, val_d):
    out = C.c_double(-1.0)
    st = lib.s3_rmse_noalloc(model.ctx, L.ptr_array([a.data_ptr() for a in idx_d]),
                             val_d.data_ptr(), int(val_d.numel()), C.byref(out))
    return st, out.value


def test_rmse_noalloc_matches_rmse_and_oracle_on_consecutive_calls(cuda_lib):
    """Within 1e-5 relative (the tolerance of the other RMSE parity tests) of s3_rmse and of
    the oracle's test RMSE, on two calls in a row, a smaller call in between and after an
    epoch."""
    p = synth.make_problem("cfg1_tiny")
    model, orc, q, order = make_pair(p)
    dev = torch.device("cuda")
    idx_d = [torch.tensor(q.test_idx[n], dtype=torch.int32, device=dev) for n in range(3)]
    val_d = torch.tensor(q.test_val, dtype=torch.float32, device=dev)
    ref = model.rmse(torch.stack(idx_d), val_d)
    want_o = orc.rmse(q.test_idx, q.test_val)
    assert abs(ref - want_o) / want_o <= 1e-5
    half = val_d.numel() // 2 + 13
    ref_half = model.rmse(torch.stack([a[:half] for a in idx_d]), val_d[:half])
    want_o_half = orc.rmse(q.test_idx[:, :half], q.test_val[:half])
    lib = model.lib
    # two calls in a row, a smaller call in between (the scratch keeps the last contents)
    for idx, val, want, want_o_ in [(idx_d, val_d, ref, want_o), (idx_d, val_d, ref, want_o),
                                    ([a[:half] for a in idx_d], val_d[:half], ref_half, want_o_half),
                                    (idx_d, val_d, ref, want_o)]:
        st, got = _noalloc(lib, model, idx, val)
        assert st == L.S3_OK, lib.s3_last_error(model.ctx)
        assert abs(got - want) / want <= 1e-5
        assert abs(got - want_o_) / want_o_ <= 1e-5
    # after an epoch the three still agree
    model.epoch("minibatch")
    orc.epoch_minibatch(0, order)
    ref2 = model.rmse(torch.stack(idx_d), val_d)
    want2 = orc.rmse(q.test_idx, q.test_val)
    st, got = _noalloc(lib, model, idx_d, val_d)
    assert st == L.S3_OK and abs(got - ref2) / ref2 <= 1e-5
    assert abs(got - want2) / want2 <= 1e-5
    model.close()


def test_rmse_noalloc_rejects_sizes_beyond_its_scratch_and_bad_indices(cuda_lib):
    from paper_1708_08640_gb300.model import S3CMTF
    p = synth.make_problem("cfg0")
    model = S3CMTF.from_problem(p)
    dev = torch.device("cuda")
    idx_d = [torch.zeros(4, dtype=torch.int32, device=dev) for _ in range(3)]
    val_d = torch.zeros(4, dtype=torch.float32, device=dev)
    out = C.c_double()
    # the size check happens before any device work
    st = model.lib.s3_rmse_noalloc(model.ctx, L.ptr_array([a.data_ptr() for a in idx_d]),
                                   val_d.data_ptr(), 2_097_153, C.byref(out))
    assert st == L.S3_ERR_ARG
    assert b"2,097,152" in model.lib.s3_last_error(model.ctx)
    st, got = _noalloc(model.lib, model, idx_d, val_d)
    assert st == L.S3_OK and np.isfinite(got)
    # an index outside its mode's range is caught by the kernel (no row read with it) ...
    bad = [a.clone() for a in idx_d]
    bad[1][2] = p.dims[1]
    st, got = _noalloc(model.lib, model, bad, val_d)
    assert st == L.S3_ERR_INDEX and got == -1.0
    # ... and the flag it raised is cleared by the next call
    st, got = _noalloc(model.lib, model, idx_d, val_d)
    assert st == L.S3_OK and np.isfinite(got)
    model.close()
