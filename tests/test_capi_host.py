"""The C-ABI library: it loads, exports every function include/s3cmtf.h declares, and
rejects invalid input on the host with the documented status (no compute calls)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1708_08640_gb300 import _lib as L
from tests.conftest import ROOT, gpu_available


def header_functions():
    text = open(os.path.join(ROOT, "include", "s3cmtf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(s3_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    return L.load(build_if_missing=True)


def test_exports_every_declared_function(lib):
    names = header_functions()
    assert len(names) >= 15
    assert sorted(L.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n


def _init(lib, idx, val, dims, J, coupled=(), order=None, hp=None):
    N = len(dims)
    idx = [np.ascontiguousarray(i, dtype=np.int32) for i in idx]
    val = np.ascontiguousarray(val, dtype=np.float32)
    dims_a = (C.c_int64 * N)(*dims)
    t = L.s3_coo_tensor(N, dims_a, int(val.shape[0]), L.ptr_array([a.ctypes.data for a in idx]),
                        val.ctypes.data)
    ys = (L.s3_coo_matrix * max(1, len(coupled)))()
    keep = []
    for m, (mode, rows, K, r, c) in enumerate(coupled):
        r = np.ascontiguousarray(r, dtype=np.int32)
        c = np.ascontiguousarray(c, dtype=np.int32)
        keep += [r, c]
        ys[m] = L.s3_coo_matrix(mode, rows, K, r.shape[0], r.ctypes.data, c.ctypes.data, None)
    h = hp or L.s3_hparams(0.01, 0.1, 0.01, 1.0, 64, 1.0, 0, 0, 0.0, 0)
    Ja = (C.c_int * N)(*J)
    ordr = None if order is None else np.ascontiguousarray(order, dtype=np.int64)
    ctx = C.c_void_p()
    st = lib.s3_init(C.byref(ctx), C.byref(t), ys if coupled else None, len(coupled), Ja,
                     C.byref(h), 0, None if ordr is None else ordr.ctypes.data, 0, None)
    msg = lib.s3_last_error(ctx).decode() if ctx else ""
    if ctx:
        lib.s3_destroy(ctx)
    return st, msg


def _valid():
    rng = np.random.default_rng(0)
    idx = [rng.integers(0, 5, 20), rng.integers(0, 4, 20), rng.integers(0, 3, 20)]
    return idx, rng.normal(size=20)


def test_rejects_bad_order_of_tensor(lib):
    idx, val = _valid()
    st, _ = _init(lib, idx[:2], val, (5, 4), (2, 2))
    assert st == L.S3_ERR_ARG


def test_rejects_bad_rank(lib):
    idx, val = _valid()
    assert _init(lib, idx, val, (5, 4, 3), (2, 0, 2))[0] == L.S3_ERR_ARG
    assert _init(lib, idx, val, (5, 4, 3), (2, 33, 2))[0] == L.S3_ERR_ARG
    assert _init(lib, idx + [np.zeros(20)], val, (5, 4, 3, 1), (9, 2, 2, 1))[0] == L.S3_ERR_ARG


def test_rejects_index_out_of_range(lib):
    idx, val = _valid()
    idx[1] = idx[1].copy()
    idx[1][7] = 4
    st, msg = _init(lib, idx, val, (5, 4, 3), (2, 2, 2))
    assert st == L.S3_ERR_INDEX and "mode 1" in msg
    idx, val = _valid()
    idx[0] = idx[0].copy()
    idx[0][0] = -1
    assert _init(lib, idx, val, (5, 4, 3), (2, 2, 2))[0] == L.S3_ERR_INDEX


def test_rejects_non_finite_values(lib):
    idx, val = _valid()
    val[3] = np.nan
    assert _init(lib, idx, val, (5, 4, 3), (2, 2, 2))[0] == L.S3_ERR_ARG


def test_rejects_bad_coupled(lib):
    idx, val = _valid()
    r = np.array([0, 1, 2])
    c = np.array([0, 1, 1])
    assert _init(lib, idx, val, (5, 4, 3), (2, 2, 2), coupled=[(0, 4, 3, r, c)])[0] == L.S3_ERR_ARG
    assert _init(lib, idx, val, (5, 4, 3), (2, 2, 2), coupled=[(3, 5, 3, r, c)])[0] == L.S3_ERR_ARG
    c2 = np.array([0, 1, 3])
    assert _init(lib, idx, val, (5, 4, 3), (2, 2, 2), coupled=[(0, 5, 3, r, c2)])[0] == L.S3_ERR_INDEX


def test_rejects_order_that_is_not_a_permutation(lib):
    idx, val = _valid()
    order = np.arange(20)
    order[5] = 4
    assert _init(lib, idx, val, (5, 4, 3), (2, 2, 2), order=order)[0] == L.S3_ERR_INDEX


def test_rejects_bad_hparams(lib):
    idx, val = _valid()
    h = L.s3_hparams(-1.0, 0.1, 0.01, 1.0, 64, 1.0, 0, 0, 0.0, 0)
    assert _init(lib, idx, val, (5, 4, 3), (2, 2, 2), hp=h)[0] == L.S3_ERR_ARG
    h = L.s3_hparams(0.01, 0.1, 0.01, 1.0, 0, 1.0, 0, 0, 0.0, 0)
    assert _init(lib, idx, val, (5, 4, 3), (2, 2, 2), hp=h)[0] == L.S3_ERR_ARG
    # the non-negative form is a flag: 0 or 1
    h = L.s3_hparams(0.01, 0.1, 0.01, 1.0, 64, 1.0, 0, 0, 0.0, 0, 0, 0, 2)
    st, msg = _init(lib, idx, val, (5, 4, 3), (2, 2, 2), hp=h)
    assert st == L.S3_ERR_ARG and "hyper-parameters" in msg


@pytest.mark.skipif(gpu_available(), reason="checks the no-device path")
def test_valid_input_without_device_reports_cuda_error(lib):
    idx, val = _valid()
    st, msg = _init(lib, idx, val, (5, 4, 3), (2, 2, 2))
    assert st == L.S3_ERR_CUDA and "no CUDA device" in msg


def test_null_context_calls(lib):
    assert lib.s3_epoch(None, 0, 0) == L.S3_ERR_STATE
    assert lib.s3_loss(None, None, None) == L.S3_ERR_STATE
    assert lib.s3_set_epoch(None, 1) == L.S3_ERR_STATE
    assert lib.s3_last_error(None) == b"NULL context"
    lib.s3_destroy(None)
