"""Python face of the S3CMTF GB300 path: one object per fitted problem.

All arithmetic runs in the CUDA library behind ``include/s3cmtf.h``; this class only
marshals arguments.  PyTorch provides the device buffers and the stream the library
enqueues its work on.
"""
from __future__ import annotations

import ctypes as C

import os

import numpy as np
import torch

from . import _lib as L

_MODES = {"minibatch": L.S3_MINIBATCH, "hogwild": L.S3_HOGWILD}
_PREC = {"fp32": L.S3_FP32, "bf16": L.S3_BF16}
_ROW = {"sum": L.S3_ROW_SUM, "mean": L.S3_ROW_MEAN}


def _host(a, dtype):
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


def _dev(t, dtype, device):
    if isinstance(t, torch.Tensor):
        return t.to(device=device, dtype=dtype).contiguous()
    return torch.as_tensor(np.ascontiguousarray(t), dtype=dtype, device=device)


class S3CMTF:
    """Sparse coupled Tucker factorisation state on one GPU.

    dims        (I_1..I_N)
    J           (J_1..J_N) core dimensionalities
    train_idx   int [N, nnz] tensor coordinates (0-based); train_val [nnz]
    coupled     sequence of (mode, K, rows, cols, vals_or_None) coupled matrices
    order       optional int64 visiting order of the union of items (see s3_init)
    """

    def __init__(self, dims, J, train_idx, train_val, coupled=(), *, lr0=0.01, mu=0.1,
                 lambda_reg=0.01, lambda_m=1.0, batch=4096, core_scale=1.0, row_rule="sum",
                 hog_tile=0, hog_staleness=0.0, hog_ctas=0, mb_ctas=0, cp=0, nonneg=0,
                 grad_chunk=0, hog_core_sync=0, wait_limit_us=0, device_bytes_cap=0, seed=0,
                 order=None,
                 device=None,
                 stream=None):
        self.lib = L.load()
        self.lr0, self.mu = float(lr0), float(mu)
        self._has_test = False
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.type != "cuda":
            raise ValueError("S3CMTF runs on a CUDA device")
        self.dims = tuple(int(d) for d in dims)
        self.N = len(self.dims)
        self.J = tuple(int(j) for j in J)
        self.coupled = [(int(c[0]), int(c[1])) for c in coupled]
        self.M = len(self.coupled)
        idx = _host(train_idx, np.int32)
        val = _host(train_val, np.float32)
        self.nnz = int(val.shape[0])
        self._dims_arr = (C.c_int64 * self.N)(*self.dims)
        self._idx_rows = [np.ascontiguousarray(idx[n]) for n in range(self.N)]
        idx_ptrs = L.ptr_array([a.ctypes.data for a in self._idx_rows])
        train = L.s3_coo_tensor(self.N, self._dims_arr, int(val.shape[0]), idx_ptrs,
                                val.ctypes.data)
        ys = (L.s3_coo_matrix * max(1, self.M))()
        keep = []
        for m, c in enumerate(coupled):
            mode, K, r, cc, v = c
            r = _host(r, np.int32)
            cc = _host(cc, np.int32)
            v = None if v is None else _host(v, np.float32)
            keep += [r, cc, v]
            ys[m] = L.s3_coo_matrix(int(mode), self.dims[int(mode)], int(K), int(r.shape[0]),
                                    r.ctypes.data, cc.ctypes.data,
                                    None if v is None else v.ctypes.data)
        hp = L.s3_hparams(lr0, mu, lambda_reg, lambda_m, int(batch), core_scale,
                          _ROW[row_rule] if isinstance(row_rule, str) else int(row_rule),
                          int(hog_tile), float(hog_staleness), int(hog_ctas), int(mb_ctas),
                          int(cp), int(nonneg), int(grad_chunk), int(hog_core_sync),
                          int(wait_limit_us), int(device_bytes_cap))
        Jarr = (C.c_int * self.N)(*self.J)
        order_arr = None if order is None else _host(order, np.int64)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            ctx = C.c_void_p()
            st = self.lib.s3_init(C.byref(ctx), C.byref(train), ys if self.M else None, self.M,
                                  Jarr, C.byref(hp), int(seed),
                                  None if order_arr is None else order_arr.ctypes.data, 0,
                                  C.c_void_p(self.stream.cuda_stream))
        self.ctx = ctx
        if st != L.S3_OK:
            msg = self.lib.s3_last_error(ctx) if ctx else b""
            self.close()
            raise L.S3Error(st, (msg or b"").decode(errors="replace"))
        del keep

    @classmethod
    def from_problem(cls, prob, **kw):
        hp = dict(prob.hparams)
        hp.update(kw)
        cpl = [(c.mode, c.K, c.rows, c.cols, c.vals) for c in prob.coupled]
        return cls(prob.dims, prob.J, prob.train_idx, prob.train_val, cpl, **hp)

    # ------------------------------------------------------------------ lifecycle
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.s3_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        return L.check(self.lib, self.ctx, st)

    # torch tensors handed to the library were produced on torch's current stream, and the
    # ones it fills are consumed there: order the two streams around every such call
    def _enter(self):
        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            self.stream.wait_stream(cur)

    def _leave(self, *tensors):
        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            cur.wait_stream(self.stream)
            for t in tensors:
                t.record_stream(self.stream)

    # ------------------------------------------------------------------ calls
    def epoch(self, mode="minibatch", precision="fp32"):
        self._check(self.lib.s3_epoch(self.ctx, _MODES[mode], _PREC[precision]))

    def fit(self, epochs, mode="hogwild", precision="fp32", log=None):
        """Runs `epochs` epochs and returns one record per epoch: its number t (from 0, the
        context's counter), the learning rate eta_t = lr0 / (1 + mu t) it used (Section 3.4),
        the loss f of Eq. (7) and the RMSE over the training entries after it, the test RMSE
        (None without a test set), the epoch's device time in ms (CUDA events on the
        context's stream; the loss and RMSE reads are outside it) and the nnz-updates/s that
        time gives (tensor plus coupled entries).  With `log` (a path, opened for appending,
        or a writable text file) every record is also written as one JSON line when its
        epoch ends."""
        import json
        out = []
        fh = open(log, "a") if isinstance(log, (str, os.PathLike)) else log
        try:
            n_items = self.info()["n_union"]
            for _ in range(int(epochs)):
                t = self.epoch_count
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(self.stream)
                self.epoch(mode, precision)
                e1.record(self.stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                f, train_rmse = self.loss()
                rec = {"epoch": t, "eta": self.lr0 / (1.0 + self.mu * t), "mode": mode,
                       "precision": precision, "loss": f, "train_rmse": train_rmse,
                       "test_rmse": self.rmse() if self._has_test else None,
                       "epoch_ms": ms, "nnz_updates_per_s": n_items / (ms / 1000.0)}
                out.append(rec)
                if fh is not None:
                    fh.write(json.dumps(rec) + "\n")
                    fh.flush()
        finally:
            if fh is not None and fh is not log:
                fh.close()
        return out

    def loss(self):
        f, r = C.c_double(), C.c_double()
        self._check(self.lib.s3_loss(self.ctx, C.byref(f), C.byref(r)))
        return f.value, r.value

    def set_test(self, idx, val):
        idx = _host(idx, np.int32)
        val = _host(val, np.float32)
        rows = [np.ascontiguousarray(idx[n]) for n in range(self.N)]
        t = L.s3_coo_tensor(self.N, self._dims_arr, int(val.shape[0]),
                            L.ptr_array([a.ctypes.data for a in rows]), val.ctypes.data)
        self._check(self.lib.s3_set_test(self.ctx, C.byref(t), 0))
        self._has_test = True

    def rmse(self, idx=None, val=None):
        out = C.c_double()
        if idx is None:
            self._check(self.lib.s3_rmse(self.ctx, None, 0, C.byref(out)))
            return out.value
        if isinstance(idx, torch.Tensor) and idx.is_cuda:
            idx_d = [_dev(idx[n], torch.int32, self.device) for n in range(self.N)]
            val_d = _dev(val, torch.float32, self.device)
            t = L.s3_coo_tensor(self.N, self._dims_arr, int(val_d.numel()),
                                L.ptr_array([a.data_ptr() for a in idx_d]), val_d.data_ptr())
            self._enter()
            self._check(self.lib.s3_rmse(self.ctx, C.byref(t), 1, C.byref(out)))
            return out.value
        idx = _host(idx, np.int32)
        val = _host(val, np.float32)
        rows = [np.ascontiguousarray(idx[n]) for n in range(self.N)]
        t = L.s3_coo_tensor(self.N, self._dims_arr, int(val.shape[0]),
                            L.ptr_array([a.ctypes.data for a in rows]), val.ctypes.data)
        self._check(self.lib.s3_rmse(self.ctx, C.byref(t), 0, C.byref(out)))
        return out.value

    def predict(self, idx):
        idx_d = [_dev(np.asarray(idx[n]) if not isinstance(idx, torch.Tensor) else idx[n],
                      torch.int32, self.device) for n in range(self.N)]
        n = int(idx_d[0].numel())
        out = torch.empty(n, dtype=torch.float32, device=self.device)
        self._enter()
        self._check(self.lib.s3_predict(self.ctx, L.ptr_array([a.data_ptr() for a in idx_d]), n,
                                        out.data_ptr()))
        self._leave(out, *idx_d)
        return out

    def _param_buffers(self):
        G = torch.empty(self.J, dtype=torch.float32, device=self.device)
        U = [torch.empty((d, j), dtype=torch.float32, device=self.device)
             for d, j in zip(self.dims, self.J)]
        V = [torch.empty((K, self.J[mode]), dtype=torch.float32, device=self.device)
             for mode, K in self.coupled]
        return G, U, V

    def gradient(self, w=None):
        """The full gradient (s3_gradient).  w: None for the gradient of f, or per-entry
        weights [nnz] (train-entry order) that take the place of -e in the data terms."""
        dG, dU, dV = self._param_buffers()
        wd = None
        if w is not None:
            wd = _dev(w, torch.float32, self.device).reshape(-1)
            if wd.numel() != self.nnz:
                raise ValueError(f"w has {wd.numel()} entries, the model {self.nnz}")
        self._enter()
        self._check(self.lib.s3_gradient(self.ctx, None if wd is None else wd.data_ptr(),
                                         dG.data_ptr(),
                                         L.ptr_array([u.data_ptr() for u in dU]),
                                         L.ptr_array([v.data_ptr() for v in dV])))
        self._leave(dG, *dU, *dV, *([] if wd is None else [wd]))
        return dG, dU, dV

    def set_counts(self, counts, nnz_total):
        """The whole problem's row counts (one int64 array per factor: U^(1..N), then V_m)
        and |Omega|, for a model that holds one part of it (s3_set_counts)."""
        arrs = [np.ascontiguousarray(np.asarray(c), dtype=np.int64) for c in counts]
        self._check(self.lib.s3_set_counts(self.ctx, L.ptr_array([a.ctypes.data for a in arrs]),
                                           int(nnz_total)))

    def apply_gradient(self, dG, dU, dV):
        """One minibatch-rule step whose group is the whole epoch, from the whole problem's
        gradient (device tensors of the parameter shapes; s3_apply_gradient)."""
        dG = _dev(dG, torch.float32, self.device).contiguous()
        dU = [_dev(u, torch.float32, self.device).contiguous() for u in dU]
        dV = [_dev(v, torch.float32, self.device).contiguous() for v in dV]
        self._enter()
        self._check(self.lib.s3_apply_gradient(self.ctx, dG.data_ptr(),
                                               L.ptr_array([u.data_ptr() for u in dU]),
                                               L.ptr_array([v.data_ptr() for v in dV])))

    def get_params(self):
        G, U, V = self._param_buffers()
        self._enter()
        self._check(self.lib.s3_get_params(self.ctx, G.data_ptr(),
                                           L.ptr_array([u.data_ptr() for u in U]),
                                           L.ptr_array([v.data_ptr() for v in V])))
        self._leave(G, *U, *V)
        return G, U, V

    def set_params(self, G, U, V):
        Gd = _dev(G, torch.float32, self.device).reshape(self.J)
        Ud = [_dev(u, torch.float32, self.device) for u in U]
        Vd = [_dev(v, torch.float32, self.device) for v in V]
        for n, u in enumerate(Ud):
            if tuple(u.shape) != (self.dims[n], self.J[n]):
                raise ValueError(f"U[{n}] has shape {tuple(u.shape)}")
        for m, v in enumerate(Vd):
            mode, K = self.coupled[m]
            if tuple(v.shape) != (K, self.J[mode]):
                raise ValueError(f"V[{m}] has shape {tuple(v.shape)}")
        self._enter()
        self._check(self.lib.s3_set_params(self.ctx, Gd.data_ptr(),
                                           L.ptr_array([u.data_ptr() for u in Ud]),
                                           L.ptr_array([v.data_ptr() for v in Vd])))
        # keep the sources alive until the stream has copied them
        self.stream.synchronize()

    @property
    def epoch_count(self):
        t = C.c_int64()
        self._check(self.lib.s3_get_epoch(self.ctx, C.byref(t)))
        return t.value

    @epoch_count.setter
    def epoch_count(self, t):
        self._check(self.lib.s3_set_epoch(self.ctx, int(t)))

    def info(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(self.lib.s3_info(self.ctx, C.byref(a), C.byref(b), C.byref(c)))
        return dict(n_union=a.value, n_batches=b.value, n_tiles=c.value)

    def finalize_qr(self):
        """Algorithm 1's final step: orthonormal factors, the core and coupled factors
        transformed so that every prediction stays the same."""
        self._enter()
        self._check(self.lib.s3_finalize_qr(self.ctx))
        self._leave()

    def hog_config(self, precision="fp32"):
        """The HOGWILD launch of a precision form: CTAs, entries per tile, dynamic shared
        memory per CTA, CTAs per SM (ctas x tile = entries in flight)."""
        v = [C.c_int64() for _ in range(4)]
        self._check(self.lib.s3_hog_config(self.ctx, _PREC[precision], *[C.byref(x) for x in v]))
        return dict(ctas=v[0].value, tile=v[1].value, smem_bytes=v[2].value,
                    ctas_per_sm=v[3].value)

    def update_values(self, x_val, y_vals=None):
        """x_val / y_vals: host float32 arrays (pinned torch tensors or numpy), in the order
        given at construction.  The copies are enqueued on the stream."""
        def hptr(a):
            if isinstance(a, torch.Tensor):
                assert a.dtype == torch.float32 and not a.is_cuda and a.is_contiguous()
                return a.data_ptr()
            assert a.dtype == np.float32 and a.flags.c_contiguous
            return a.ctypes.data
        ys = L.ptr_array([hptr(y) if y is not None else None for y in (y_vals or [])])
        self._check(self.lib.s3_update_values(self.ctx, hptr(x_val), ys if y_vals else None))
        if isinstance(x_val, np.ndarray):
            # pageable numpy memory: the copy must finish before the caller may reuse it
            self.stream.synchronize()
