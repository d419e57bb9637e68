"""s3_rmse_noalloc serves callers that cannot allocate device memory (code inside a CUDA graph
capture, under a fixed memory budget, or beside an allocator that owns the whole device).
It must give the test RMSE of s3_rmse, call after call, from its static scratch alone.
Collected last on purpose (file name), so a failure here comes after every other test."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1708_08640_gb300 import _lib as L
from paper_1708_08640_gb300 import synth

pytestmark = pytest.mark.gpu


def _noalloc(lib, model, idx_d, val_d):
    out = C.c_double()
    st = lib.s3_rmse_noalloc(model.ctx, L.ptr_array([a.data_ptr() for a in idx_d]),
                             val_d.data_ptr(), int(val_d.numel()), C.byref(out))
    return st, out.value


def test_rmse_noalloc_matches_rmse_on_consecutive_calls(cuda_lib):
    from paper_1708_08640_gb300.model import S3CMTF
    p = synth.make_problem("cfg1_tiny")
    model = S3CMTF.from_problem(p, order=synth.union_order(p, 2))
    model.set_params(*synth.init_params(p, 1))
    dev = torch.device("cuda")
    idx_d = [torch.tensor(p.test_idx[n], dtype=torch.int32, device=dev) for n in range(3)]
    val_d = torch.tensor(p.test_val, dtype=torch.float32, device=dev)
    ref = model.rmse(torch.stack(idx_d), val_d)
    half = val_d.numel() // 2 + 13
    ref_half = model.rmse(torch.stack([a[:half] for a in idx_d]), val_d[:half])
    lib = model.lib
    # two calls in a row, a smaller call in between (the scratch keeps the last contents)
    for idx, val, want in [(idx_d, val_d, ref), (idx_d, val_d, ref),
                           ([a[:half] for a in idx_d], val_d[:half], ref_half),
                           (idx_d, val_d, ref)]:
        st, got = _noalloc(lib, model, idx, val)
        assert st == L.S3_OK, lib.s3_last_error(model.ctx)
        assert abs(got - want) / want <= 1e-5
    # after an epoch the two still agree
    model.epoch("minibatch")
    ref2 = model.rmse(torch.stack(idx_d), val_d)
    st, got = _noalloc(lib, model, idx_d, val_d)
    assert st == L.S3_OK and abs(got - ref2) / ref2 <= 1e-5
    model.close()


def test_rmse_noalloc_rejects_sizes_beyond_its_scratch(cuda_lib):
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
    model.close()
