"""FP64 CPU oracle for S3CMTF -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It shares no code with the CUDA path (``paper_1708_08640_gb300``) and
imports nothing from it; the product path never reaches it.

The arithmetic lives in ``s3cmtf_oracle.c`` (plain double-precision loops written from the
paper's Eq. (3), Eq. (4), Eq. (7), Eq. (8), Algorithms 1-3 and the test RMSE of Section 4.1).
This module only compiles it with gcc and marshals numpy arrays through ctypes.

Any object with the attributes ``dims, J, train_idx, train_val`` and ``coupled`` (a list of
objects with ``mode, K, rows, cols, vals``) describes a problem.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "s3cmtf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the oracle (gcc -O2, plain C11).  Returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (force or not os.path.exists(_LIB_PATH)
            or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Data(C.Structure):
    _fields_ = [
        ("N", C.c_int), ("I", C.POINTER(C.c_int64)), ("J", C.POINTER(C.c_int)),
        ("nnz", C.c_int64), ("idx", C.POINTER(C.c_int32)), ("x", C.POINTER(C.c_double)),
        ("M", C.c_int), ("cmode", C.POINTER(C.c_int)), ("K", C.POINTER(C.c_int64)),
        ("ynnz", C.POINTER(C.c_int64)), ("yr", C.POINTER(C.POINTER(C.c_int32))),
        ("yc", C.POINTER(C.POINTER(C.c_int32))), ("y", C.POINTER(C.POINTER(C.c_double))),
        ("cnt_total", C.POINTER(C.POINTER(C.c_int64))), ("nnz_total", C.c_int64),
    ]


class _Params(C.Structure):
    _fields_ = [("G", C.POINTER(C.c_double)), ("U", C.POINTER(C.POINTER(C.c_double))),
                ("V", C.POINTER(C.POINTER(C.c_double)))]


class _HParams(C.Structure):
    _fields_ = [("lr0", C.c_double), ("mu", C.c_double), ("lambda_reg", C.c_double),
                ("lambda_m", C.c_double), ("core_scale", C.c_double), ("batch", C.c_int64),
                ("row_mean", C.c_int), ("cp", C.c_int), ("nonneg", C.c_int)]


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P, D, H = C.POINTER(_Params), C.POINTER(_Data), C.POINTER(_HParams)
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int32)
            lp = C.POINTER(C.c_int64)
            lib.s3o_predict.argtypes = [D, P, ip, C.c_int64, dp]
            lib.s3o_partials.argtypes = [D, P, ip, dp]
            lib.s3o_predict_coupled.argtypes = [D, P, C.c_int, ip, ip, C.c_int64, dp]
            lib.s3o_loss.argtypes = [D, P, H, dp]
            lib.s3o_loss_rowform.argtypes = [D, P, H]
            lib.s3o_loss_rowform.restype = C.c_double
            lib.s3o_rmse.argtypes = [D, P, ip, dp, C.c_int64]
            lib.s3o_rmse.restype = C.c_double
            lib.s3o_entry_gradient.argtypes = [D, P, H, C.c_int64, dp, dp]
            lib.s3o_entry_gradient.restype = C.c_double
            lib.s3o_entry_gradient_opt.argtypes = [D, P, H, C.c_int64, dp, dp]
            lib.s3o_entry_gradient_opt.restype = C.c_double
            lib.s3o_full_gradient.argtypes = [D, P, H, dp, C.POINTER(dp), C.POINTER(dp)]
            lib.s3o_full_gradient_w.argtypes = [D, P, H, dp, dp, C.POINTER(dp), C.POINTER(dp)]
            lib.s3o_learning_rate.argtypes = [H, C.c_int64]
            lib.s3o_learning_rate.restype = C.c_double
            lib.s3o_epoch_sequential.argtypes = [D, P, H, C.c_int64, lp, C.c_int64]
            lib.s3o_epoch_sequential.restype = C.c_int
            lib.s3o_epoch_minibatch.argtypes = [D, P, H, C.c_int64, lp, C.c_int64]
            lib.s3o_epoch_minibatch.restype = C.c_int
            lib.s3o_finalize_qr.argtypes = [D, P, C.POINTER(dp)]
            lib.s3o_finalize_qr.restype = C.c_int
            _lib = lib
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _ptr_array(arrs, ct):
    arr = (C.POINTER(ct) * max(1, len(arrs)))()
    for k, a in enumerate(arrs):
        arr[k] = _ptr(a, ct)
    return arr


class Oracle:
    """FP64 model state plus the problem it is fitted to."""

    def __init__(self, prob, hparams=None, counts=None, nnz_total=0, **hp_overrides):
        """counts, nnz_total: when prob is a part of a larger problem, that problem's row
        counts (one int64 array per factor: U^(1..N), then V_m) and |Omega|, which the
        regularisation terms use; None / 0 = prob's own."""
        self.lib = _lib_handle()
        self.dims = tuple(int(d) for d in prob.dims)
        self.J = tuple(int(j) for j in prob.J)
        self.N = len(self.dims)
        self._keep = []
        keep = self._keep.append
        self._I = np.ascontiguousarray(self.dims, dtype=np.int64); keep(self._I)
        self._Jc = np.ascontiguousarray(self.J, dtype=np.int32); keep(self._Jc)
        self._idx = np.ascontiguousarray(prob.train_idx, dtype=np.int32); keep(self._idx)
        self._x = np.ascontiguousarray(prob.train_val, dtype=np.float64); keep(self._x)
        cps = list(prob.coupled)
        self.M = len(cps)
        self.coupled = cps
        self._cmode = np.ascontiguousarray([c.mode for c in cps] or [0], dtype=np.int32)
        self._K = np.ascontiguousarray([c.K for c in cps] or [0], dtype=np.int64)
        self._ynnz = np.ascontiguousarray([c.rows.shape[0] for c in cps] or [0], dtype=np.int64)
        self._yr = [np.ascontiguousarray(c.rows, dtype=np.int32) for c in cps]
        self._yc = [np.ascontiguousarray(c.cols, dtype=np.int32) for c in cps]
        self._y = [np.ascontiguousarray(c.vals, dtype=np.float64) for c in cps]
        for a in (self._cmode, self._K, self._ynnz, *self._yr, *self._yc, *self._y):
            keep(a)
        self.data = _Data(
            self.N, _ptr(self._I, C.c_int64), _ptr(self._Jc, C.c_int),
            int(self._x.shape[0]), _ptr(self._idx, C.c_int32), _ptr(self._x, C.c_double),
            self.M, _ptr(self._cmode, C.c_int), _ptr(self._K, C.c_int64),
            _ptr(self._ynnz, C.c_int64), _ptr_array(self._yr, C.c_int32),
            _ptr_array(self._yc, C.c_int32), _ptr_array(self._y, C.c_double),
            None, int(nnz_total))
        if counts is not None:
            self._cnt = [np.ascontiguousarray(c, dtype=np.int64) for c in counts]
            assert len(self._cnt) == self.N + self.M
            self._cnt_ptrs = _ptr_array(self._cnt, C.c_int64)
            self.data.cnt_total = self._cnt_ptrs
        hp = dict(getattr(prob, "hparams", {}) or {})
        hp.update(hparams or {})
        hp.update(hp_overrides)
        self.hp = dict(lr0=hp.get("lr0", 0.01), mu=hp.get("mu", 0.1),
                       lambda_reg=hp.get("lambda_reg", 0.01),
                       lambda_m=hp.get("lambda_m", 1.0), core_scale=hp.get("core_scale", 1.0),
                       batch=int(hp.get("batch", 1)), row_mean=int(hp.get("row_mean", 0)),
                       cp=int(hp.get("cp", 0)), nonneg=int(hp.get("nonneg", 0)))
        self.G = np.zeros(self.J)
        self.U = [np.zeros((d, j)) for d, j in zip(self.dims, self.J)]
        self.V = [np.zeros((c.K, self.J[c.mode])) for c in cps]
        self._bind_params()

    # -- state
    def _bind_params(self):
        self.params_c = _Params(_ptr(self.G, C.c_double), _ptr_array(self.U, C.c_double),
                                _ptr_array(self.V, C.c_double))

    def set_params(self, G, U, V):
        self.G = np.array(G, dtype=np.float64, order="C", copy=True).reshape(self.J)
        self.U = [np.array(u, dtype=np.float64, order="C", copy=True) for u in U]
        self.V = [np.array(v, dtype=np.float64, order="C", copy=True) for v in V]
        for n, u in enumerate(self.U):
            assert u.shape == (self.dims[n], self.J[n])
        for m, v in enumerate(self.V):
            assert v.shape == (self.coupled[m].K, self.J[self.coupled[m].mode])
        self._bind_params()

    def get_params(self):
        return self.G.copy(), [u.copy() for u in self.U], [v.copy() for v in self.V]

    def _h(self, **over):
        h = dict(self.hp)
        h.update(over)
        return _HParams(h["lr0"], h["mu"], h["lambda_reg"], h["lambda_m"], h["core_scale"],
                        int(h["batch"]), int(h["row_mean"]), int(h["cp"]), int(h["nonneg"]))

    # -- O1
    def predict(self, idx):
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        n = idx.shape[1]
        out = np.empty(n)
        self.lib.s3o_predict(C.byref(self.data), C.byref(self.params_c), _ptr(idx, C.c_int32),
                             n, _ptr(out, C.c_double))
        return out

    def partials(self, alpha):
        alpha = np.ascontiguousarray(alpha, dtype=np.int32)
        out = np.empty(sum(self.J))
        self.lib.s3o_partials(C.byref(self.data), C.byref(self.params_c),
                              _ptr(alpha, C.c_int32), _ptr(out, C.c_double))
        res, o = [], 0
        for j in self.J:
            res.append(out[o:o + j].copy())
            o += j
        return res

    def predict_coupled(self, m, rows, cols):
        r = np.ascontiguousarray(rows, dtype=np.int32)
        c = np.ascontiguousarray(cols, dtype=np.int32)
        out = np.empty(r.shape[0])
        self.lib.s3o_predict_coupled(C.byref(self.data), C.byref(self.params_c), m,
                                     _ptr(r, C.c_int32), _ptr(c, C.c_int32), r.shape[0],
                                     _ptr(out, C.c_double))
        return out

    # -- O2 / O7
    def loss(self, **over):
        """(f, sum of squared tensor errors, [sum of squared errors per coupled matrix])"""
        out = np.zeros(2 + max(1, self.M))
        h = self._h(**over)
        self.lib.s3o_loss(C.byref(self.data), C.byref(self.params_c), C.byref(h),
                          _ptr(out, C.c_double))
        return float(out[0]), float(out[1]), [float(v) for v in out[2:2 + self.M]]

    def loss_rowform(self, **over):
        h = self._h(**over)
        return float(self.lib.s3o_loss_rowform(C.byref(self.data), C.byref(self.params_c),
                                               C.byref(h)))

    def rmse(self, idx, val):
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float64)
        return float(self.lib.s3o_rmse(C.byref(self.data), C.byref(self.params_c),
                                       _ptr(idx, C.c_int32), _ptr(val, C.c_double),
                                       val.shape[0]))

    # -- O3 / O6
    def _entry_grad(self, fn, e, **over):
        gu = np.empty(sum(self.J))
        gG = np.empty(int(np.prod(self.J)))
        h = self._h(**over)
        err = fn(C.byref(self.data), C.byref(self.params_c), C.byref(h), int(e),
                 _ptr(gu, C.c_double), _ptr(gG, C.c_double))
        res, o = [], 0
        for j in self.J:
            res.append(gu[o:o + j].copy())
            o += j
        return float(err), res, gG.reshape(self.J)

    def entry_gradient(self, e, **over):
        return self._entry_grad(self.lib.s3o_entry_gradient, e, **over)

    def entry_gradient_opt(self, e, **over):
        return self._entry_grad(self.lib.s3o_entry_gradient_opt, e, **over)

    def full_gradient(self, w=None, **over):
        """Eq. (8) summed over every entry.  w: None, or one weight per train entry that
        takes the place of -(x - x~) in the entry's data terms."""
        gG = np.empty(self.J)
        gU = [np.empty((d, j)) for d, j in zip(self.dims, self.J)]
        gV = [np.empty((c.K, self.J[c.mode])) for c in self.coupled]
        h = self._h(**over)
        if w is None:
            self.lib.s3o_full_gradient(C.byref(self.data), C.byref(self.params_c), C.byref(h),
                                       _ptr(gG, C.c_double), _ptr_array(gU, C.c_double),
                                       _ptr_array(gV, C.c_double))
        else:
            w = np.ascontiguousarray(w, dtype=np.float64)
            if w.shape != (self._x.shape[0],):
                raise ValueError("w needs one weight per train entry")
            self.lib.s3o_full_gradient_w(C.byref(self.data), C.byref(self.params_c), C.byref(h),
                                         _ptr(w, C.c_double), _ptr(gG, C.c_double),
                                         _ptr_array(gU, C.c_double), _ptr_array(gV, C.c_double))
        return gG, gU, gV

    # -- O4 / O5
    def learning_rate(self, t, **over):
        h = self._h(**over)
        return float(self.lib.s3o_learning_rate(C.byref(h), int(t)))

    def epoch_sequential(self, t, order, **over):
        order = np.ascontiguousarray(order, dtype=np.int64)
        h = self._h(**over)
        rc = self.lib.s3o_epoch_sequential(C.byref(self.data), C.byref(self.params_c),
                                           C.byref(h), int(t), _ptr(order, C.c_int64),
                                           order.shape[0])
        if rc != 0:
            raise ValueError("order holds an item outside the union of entries")

    def epoch_minibatch(self, t, order, **over):
        order = np.ascontiguousarray(order, dtype=np.int64)
        h = self._h(**over)
        rc = self.lib.s3o_epoch_minibatch(C.byref(self.data), C.byref(self.params_c),
                                          C.byref(h), int(t), _ptr(order, C.c_int64),
                                          order.shape[0])
        if rc != 0:
            raise ValueError("order holds an item outside the union of entries")

    def finalize_qr(self):
        """Algorithm 1's final step: U^(n) <- Q^(n), G <- G x_n R^(n), V_m <- V_m R^(c)^T
        (thin QR with diag(R) > 0).  Returns the R^(n); raises if a factor is rank deficient."""
        Rs = [np.zeros((j, j)) for j in self.J]
        rc = self.lib.s3o_finalize_qr(C.byref(self.data), C.byref(self.params_c),
                                      _ptr_array(Rs, C.c_double))
        if rc != 0:
            raise ValueError("a factor matrix does not have full column rank")
        return Rs
