#!/usr/bin/env python3
"""Epoch throughput of the S3CMTF GB300 path (SGD nnz-updates/s) on synthetic data shaped
like the paper's rating-tensor workloads.

One step = one SGD epoch over every observed item (train tensor entries and coupled-matrix
entries) followed by the test-RMSE pass; value = items updated per second over the K timed
steps (CUDA events on the library's stream, barrier + synchronize on both sides, max over
ranks).  The gradient pass (differentiation form) and the deterministic minibatch epoch are
timed in the same run and reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload cfg1] [--mode hogwild|minibatch]

N > 1 runs N independent replicas (one per rank, one problem each; weak scaling) -- the
method has no data-path exchange to distribute.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1708_08640_gb300 import synth  # noqa: E402

METRIC = "SGD nnz-updates/s at matched test RMSE, BF16 vs FP32 form; gradient-pass GB/s"
UNIT = "nnz-updates/s"
_FP32_PEAK = {}


def fp32_peak():
    """The FP32 CUDA-core roof of this GPU, measured once per run by the library's FFMA and
    packed FFMA2 microbenchmark (s3_measure_fp32_peak): the larger rate, TFLOP/s, and where
    it comes from."""
    if not _FP32_PEAK:
        import ctypes as C

        from paper_1708_08640_gb300 import _lib as L
        lib = L.load()
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        st = lib.s3_measure_fp32_peak(C.byref(a), C.byref(b), C.byref(c))
        if st != 0:
            raise RuntimeError(f"s3_measure_fp32_peak failed: {st}")
        _FP32_PEAK.update(peak=max(a.value, b.value),
                          source=f"measured: FFMA {a.value:.1f}, FFMA2 {b.value:.1f} TFLOP/s "
                                 f"(s3_measure_fp32_peak, all SMs, best of 3; nominal SM clock "
                                 f"{c.value:.0f} MHz)")
    return _FP32_PEAK["peak"], _FP32_PEAK["source"]
# the sources of the FP32 HOGWILD kernel: a committed DRAM-traffic figure counts only while
# their hash is the one it was captured on
_CS = "paper_1708_08640_gb300/csrc/"
_BASE = [_CS + "common.cuh", _CS + "kernels.h", _CS + "tensor_fp32.cuh"]
# the source files each profiled kernel is compiled from (its own file and every header)
KERNEL_SOURCES = {
    "k_tensor_hog": [_CS + "k_tensor_hog2.cu", _CS + "tensor_hog.cuh", _CS + "hog_common.cuh"] + _BASE,
    "k_tensor_hog_bf16": [_CS + "k_tensor_bf16.cu", _CS + "tc.cuh", _CS + "hog_common.cuh"] + _BASE,
    "k_mb_epoch": [_CS + "k_minibatch.cu"] + _BASE,
    "k_cp_hog": [_CS + "k_cp.cu", _CS + "hog_common.cuh"] + _BASE,
    "k_tensor_contrib": [_CS + "k_tensor.cu", _CS + "tensor_hog.cuh", _CS + "hog_common.cuh"] + _BASE,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="cfg1")
    ap.add_argument("--mode", choices=["hogwild", "minibatch", "gradient", "scalability"],
                    default="hogwild",
                    help="the step: a HOGWILD or minibatch epoch (nnz-updates/s), or one full "
                         "gradient pass, the differentiation form (GB/s; e.g. --workload cfg3); "
                         "scalability: the Section 4.3 sweeps of HOGWILD epoch time over |Omega| "
                         "and over I")
    ap.add_argument("--precision", choices=["fp32", "bf16"], default="fp32",
                    help="the step's precision form (bf16: HOGWILD mode, 3-way tensors)")
    ap.add_argument("--cpu-sample", type=int, default=600_000,
                    help="items of the visiting order the CPU oracle baseline processes "
                         "(0: no CPU baseline, e.g. under a profiler)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the gradient-pass and minibatch side measurements")
    ap.add_argument("--rank", type=int, default=0,
                    help="run the workload at rank J in every mode instead of its own "
                         "(rating workloads, e.g. --workload cfg1_small --rank 32)")
    ap.add_argument("--forms", action="store_true",
                    help="also run both precision forms of the HOGWILD epoch on the step's data "
                         "at its own rank (--steps epochs each) and report the comparison "
                         "(with --no-extras: the BF16 vs FP32 comparison of a large workload "
                         "from one generation of its data)")
    ap.add_argument("--variant", choices=["plain", "cp", "nonneg"], default="plain",
                    help="the step's method: plain S3CMTF-TUCKER, S3CMTF-CP (hyper-diagonal "
                         "core) or the non-negative form (projected SGD)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers
def max_over_ranks(x, world, device="cuda"):
    """The largest of every rank's x (the job's time is its slowest rank's); x itself when
    the job has one rank.  The process group is NCCL on the GPU box (device "cuda") and can
    be gloo on the CPU (device "cpu")."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, steps, world, seconds):
    """Whole-job throughput of a weakly scaled run: every rank processes units_per_rank per
    step; the job takes the slowest rank's time."""
    return world * units_per_rank * steps / seconds


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def source_sha(kernel="k_tensor_hog"):
    """A digest of the sources `kernel` is compiled from: a committed DRAM figure is used only
    while it matches."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:12]


def committed_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was taken on
    the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    if kernel not in KERNEL_SOURCES:
        return None
    sha = source_sha(kernel)
    for line in open(path):
        f = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if f.get("kernel") == kernel and f.get("workload") == workload and f.get("sha") == sha:
            return float(f["bytes_per_launch"])
    return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def cpu_baseline(p, sample, order):
    """The FP64 oracle (as it stands: one thread, plain loops) on a bounded prefix of the
    visiting order: sequential SGD (Algorithm 1, P = 1)."""
    import oracle
    o = oracle.Oracle(p, **{k: v for k, v in p.hparams.items()
                           if k in ("lr0", "mu", "lambda_reg", "lambda_m", "batch", "core_scale")})
    o.set_params(*synth.init_params(p, 1))
    sub = order[:sample]
    t0 = time.perf_counter()
    o.epoch_sequential(0, sub)
    dt = time.perf_counter() - t0
    return {"value": sample / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {sample} items of the {p.name} visiting order, one sequential "
                      f"SGD pass (Algorithm 1, P=1), FP64, {dt:.1f} s"}


def _part_gradient(args):
    """One worker of the multi-core CPU baseline: the FP64 oracle's gradient of one mode-1
    part of a problem, with the whole problem's counts (the partition's rule)."""
    import oracle
    from paper_1708_08640_gb300 import partition
    q, world, rank, hp, params = args
    part, _ = partition.mode1_part(q, world, rank)
    counts, nnz_total = partition.whole_counts(q)
    o = oracle.Oracle(part, counts=counts, nnz_total=nnz_total, **hp)
    o.set_params(*params)
    return o.full_gradient()


def cpu_baseline_multicore(p, sample, reps=2):
    """The FP64 oracle on every host core: the minibatch rule with one batch per pass over a
    bounded sample (the first `sample` tensor entries and a proportional share of each
    coupled matrix), each core computing the gradient of one mode-1 part with the oracle as
    it stands, the parts summed in a fixed order and one step taken (the multi-GPU
    partition's rule, on CPU processes).  Items per second of the pass."""
    import multiprocessing as mp

    from paper_1708_08640_gb300 import partition
    cores = max(1, os.cpu_count() or 1)
    frac = sample / max(p.nnz, 1)
    q = sub_problem(p, min(sample, p.nnz), max(1, int(round(frac * (p.coupled[0].nnz if p.coupled else 0)))))
    hp = {k: v for k, v in p.hparams.items() if k in ("lr0", "mu", "lambda_reg", "lambda_m", "core_scale")}
    params = synth.init_params(q, 1)
    items = q.nnz + sum(c.nnz for c in q.coupled)
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_part_gradient, [(q, cores, r, hp, params) for r in range(cores)])   # warm-up
        best = None
        for _ in range(reps):
            t0 = time.perf_counter()
            parts = pool.map(_part_gradient, [(q, cores, r, hp, params) for r in range(cores)])
            gG = sum(g[0] for g in parts)                       # parts added in rank order
            G, U, V = params
            eta = hp["lr0"]
            G1 = G - eta * hp["core_scale"] * gG / q.nnz
            U1 = [u - eta * sum(g[1][n] for g in parts) for n, u in enumerate(U)]
            V1 = [v - eta * sum(g[2][m] for g in parts) for m, v in enumerate(V)]
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
    del G1, U1, V1
    return {"value": items / best, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"the first {q.nnz} tensor entries and {q.n_union - q.nnz} coupled entries of "
                      f"{p.name}: one minibatch-rule pass with a single batch (the mode-1 partition "
                      f"over {cores} processes, FP64 oracle gradients summed in a fixed order, "
                      f"one step), best of {reps}, {best:.1f} s"}


def workload_desc(p, mode, precision="fp32"):
    return {"workload": f"{p.name}: {p.recipe}; J={p.J}; {precision.upper()} form, {mode}",
            "dims": list(p.dims), "J": list(p.J), "train_nnz": p.nnz,
            "coupled_nnz": [c.nnz for c in p.coupled], "test_nnz": int(p.test_val.shape[0]),
            "hparams": p.hparams, "mode": mode, "precision": precision,
            "l2": "inputs larger than L2 (COO and layout arrays >> 129 MB); no flush"}


def gradient_bytes(p):
    """Algorithmic bytes of one full-gradient pass: the COO of every tensor and coupled
    entry, every touched factor row read once, every gradient written once."""
    J = p.J
    coo = p.nnz * (4 * p.N + 4) + sum(c.nnz * 12 for c in p.coupled)
    rows = sum(int(np.unique(p.train_idx[n]).shape[0]) * J[n] for n in range(p.N))
    rows += sum(int(np.unique(c.cols).shape[0]) * J[c.mode] for c in p.coupled)
    grad_out = int(np.prod(J)) + sum(d * j for d, j in zip(p.dims, J)) + sum(
        c.K * J[c.mode] for c in p.coupled)
    return coo + 4 * rows + 4 * grad_out


def flops_per_entry(p):
    J = p.J
    return 6.0 * float(np.prod(J)) if p.N == 3 else 6.0 * float(np.prod(J)) + 4.0 * float(np.prod(J[:3]))


def sub_problem(p, n_tensor, n_coupled):
    """The first n entries of the tensor and of each coupled matrix (a bounded sample)."""
    import copy
    q = copy.copy(p)
    q.train_idx = p.train_idx[:, :n_tensor]
    q.train_val = p.train_val[:n_tensor]
    q.coupled = [synth.Coupled(c.mode, c.K, c.rows[:n_coupled], c.cols[:n_coupled],
                               c.vals[:n_coupled]) for c in p.coupled]
    return q


# ----------------------------------------------------------------------------- reference arm
def run_reference_gradient(args):
    """The oracle's full gradient (FP64, one thread) on a bounded sample of the workload."""
    import oracle
    p = synth.make_problem(args.workload)
    S = max(1000, min(args.cpu_sample // 20, p.nnz))
    q = sub_problem(p, S, max(1, S // 2))
    o = oracle.Oracle(q, **{k: v for k, v in q.hparams.items()
                           if k in ("lr0", "mu", "lambda_reg", "lambda_m", "batch", "core_scale")})
    o.set_params(*synth.init_params(q, 1))
    for _ in range(args.warmup):
        o.full_gradient()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        o.full_gradient()
        times.append(time.perf_counter() - t0)
    gb = gradient_bytes(q)
    value = gb / (sum(times) / len(times)) / 1e9
    sample = (f"the first {q.nnz} tensor entries and first {q.coupled[0].nnz if q.coupled else 0} "
              f"entries of each coupled matrix of {p.name}; one full gradient per step, FP64")
    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": dict(workload_desc(p, "gradient"), parallelism="oracle, 1 thread"),
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference(args, world, rank):
    if rank != 0:
        return
    if args.mode == "gradient":
        return run_reference_gradient(args)
    import oracle  # noqa: F401
    p = synth.make_problem(args.workload)
    order = synth.union_order(p, 2)
    o = oracle.Oracle(p, **{k: v for k, v in p.hparams.items()
                           if k in ("lr0", "mu", "lambda_reg", "lambda_m", "batch", "core_scale")})
    o.set_params(*synth.init_params(p, 1))
    S = max(1000, min(args.cpu_sample // 4, p.n_union))
    for w in range(args.warmup):
        o.epoch_sequential(0, order[(w * S) % p.n_union:][:S])
    times = []
    for k in range(args.steps):
        s0 = ((args.warmup + k) * S) % p.n_union
        t0 = time.perf_counter()
        o.epoch_sequential(0, order[s0:s0 + S])
        times.append(time.perf_counter() - t0)
    ms = 1000.0 * sum(times) / len(times)
    value = S / (ms / 1000.0)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": dict(workload_desc(p, "sequential", "fp64"),
                           step=f"{S} items of the visiting order per step"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{S} items per step, sequential Algorithm 1, FP64"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- forms
def precision_forms(p, order, stream, args, J=16, epochs=4, model=None):
    """The FP32 and BF16 forms of the HOGWILD epoch on the same data at rank J (the cfg2
    workloads, J = 16 and 32, and the cfg1 data at J = 10 and 20): epoch time, nnz-updates/s, test RMSE after every epoch (the
    "matched RMSE" check: the largest relative gap between the two forms' curves), and the
    tensor-pass kernel's roofline (FP32 FFMA roof for the FP32 form, BF16 tensor roof for
    the BF16 form).  Epochs are timed one by one with CUDA events; the RMSE reads between
    them are outside the timed regions.  With `model` (a context of p at rank J, with its
    test set) both forms run on it, each from the same start (parameters and epoch counter
    reset): one copy of the layout on the device instead of two, for workloads whose layout
    fills much of HBM."""
    import ctypes as C

    import torch

    from paper_1708_08640_gb300 import _lib as L
    from paper_1708_08640_gb300.model import S3CMTF
    q = synth.with_rank(p, (J, J, J))
    init = synth.init_params(q, 1)
    peaks, src = measured_peaks()
    out = {}
    flops_entry = 6.0 * J ** 3
    for prec in ("fp32", "bf16"):
        if model is not None:
            m = model
            m.epoch_count = 0
        else:
            m = S3CMTF.from_problem(q, order=order, stream=stream)
            m.set_test(q.test_idx, q.test_val)
        m.set_params(*init)
        curve = []
        m.epoch("hogwild", prec)          # warm-up epoch (its RMSE is the curve's first point)
        curve.append(m.rmse())
        L.check(m.lib, m.ctx, m.lib.s3_profile(m.ctx, 1))
        total = 0.0
        for _ in range(epochs):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            m.epoch("hogwild", prec)
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
            curve.append(m.rmse())
        ms = total / epochs
        kms, kn, ke = C.c_double(), C.c_int64(), C.c_int64()
        L.check(m.lib, m.ctx, m.lib.s3_profile_read(m.ctx, L.S3_K_TENSOR_HOG, C.byref(kms),
                                                      C.byref(kn), C.byref(ke)))
        L.check(m.lib, m.ctx, m.lib.s3_profile(m.ctx, 0))
        achieved = flops_entry * ke.value / (kms.value / 1000.0) / 1e12
        if prec == "fp32":
            fpk, fsrc = fp32_peak()
            roof = {"bound": "alu", "peak": fpk, "peak_source": fsrc}
        else:
            roof = {"bound": "tensor", "peak": peaks["bf16_tflops_sustained"],
                    "peak_source": f"{src} bf16_tflops_sustained"}
        roof.update({"achieved": achieved, "unit": "TFLOP/s", "frac": achieved / roof["peak"],
                     "kernel_ms_per_epoch": kms.value / epochs, "flops_per_entry": flops_entry})
        out[prec] = {"ms_per_epoch": ms, "nnz_updates_per_s": q.n_union / (ms / 1000.0),
                     "test_rmse": curve, "epochs": 1 + epochs, "roofline": roof,
                     "launch": m.hog_config(prec)}
        if model is None:
            m.close()
    # each form's test RMSE per epoch against the FP64 oracle's Algorithm 1 curve on the same
    # data, rank, start and order, where one is stored (tests/golden, written by the oracle)
    ref = stored_curve(q, "sequential")
    if ref is not None:
        k = min(len(ref["test_rmse"]), 1 + epochs)
        r = np.array(ref["test_rmse"][:k])
        out["vs_oracle_algorithm1"] = {
            prec: ((np.array(out[prec]["test_rmse"][:k]) - r) / r).tolist() for prec in ("fp32", "bf16")}
        out["vs_oracle_algorithm1"]["source"] = ref["file"]
    out["bf16_speedup"] = out["fp32"]["ms_per_epoch"] / out["bf16"]["ms_per_epoch"]
    out["rmse_max_rel_gap"] = max(abs(b - a) / a for a, b in
                                  zip(out["fp32"]["test_rmse"], out["bf16"]["test_rmse"]))
    # time to target: epochs (at the measured time per epoch) until a form's test RMSE is
    # within 0.1% of the FP32 form's final RMSE
    target = out["fp32"]["test_rmse"][-1] * 1.001
    for prec in ("fp32", "bf16"):
        hit = next((i + 1 for i, r in enumerate(out[prec]["test_rmse"]) if r <= target), None)
        out[prec]["time_to_target_ms"] = None if hit is None else hit * out[prec]["ms_per_epoch"]
    out["target_rmse"] = target
    return out


def stored_curve(q, mode):
    """The oracle's stored test-RMSE curve (tests/golden) of problem q in this mode, if one
    was written for q's data (same fingerprint) and ranks; else None."""
    import glob
    import hashlib
    h = hashlib.sha256()
    for a in (q.train_idx, q.train_val, q.test_idx, q.test_val):
        h.update(np.ascontiguousarray(a).tobytes())
    for c in q.coupled:
        for a in (c.rows, c.cols, c.vals):
            h.update(np.ascontiguousarray(a).tobytes())
    fp = h.hexdigest()[:16]
    for path in sorted(glob.glob(os.path.join(ROOT, "tests", "golden", f"curve_*_{mode}.json"))):
        rec = json.load(open(path))
        rank = rec.get("rank", [10] * q.N)
        if rec["fingerprint"] == fp and list(rank) == list(q.J) and not rec["hparams"].get("nonneg"):
            rec["file"] = os.path.relpath(path, ROOT)
            return rec
    return None


def gradient_pass(p, stream, steps=3):
    """One full-gradient pass (the differentiation form) of problem p: time per pass (CUDA
    events), algorithmic GB/s, and the tensor-entry kernel's FFMA roofline."""
    import ctypes as C

    import torch

    from paper_1708_08640_gb300 import _lib as L
    from paper_1708_08640_gb300.model import S3CMTF
    m = S3CMTF.from_problem(p, order=synth.union_order(p, 2), stream=stream)
    m.set_params(*synth.init_params(p, 1))
    m.gradient()
    L.check(m.lib, m.ctx, m.lib.s3_profile(m.ctx, 1))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        m.gradient()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    kms, kn, ke = C.c_double(), C.c_int64(), C.c_int64()
    L.check(m.lib, m.ctx, m.lib.s3_profile_read(m.ctx, L.S3_K_TENSOR_GRAD, C.byref(kms), C.byref(kn),
                                                  C.byref(ke)))
    L.check(m.lib, m.ctx, m.lib.s3_profile(m.ctx, 0))
    m.close()
    gb = gradient_bytes(p)
    fpe = flops_per_entry(p)
    fpk, fsrc = fp32_peak()
    achieved = fpe * ke.value / (kms.value / 1000.0) / 1e12 if kms.value > 0 else None
    return {"workload": f"{p.name}: {p.recipe}; J={p.J}", "ms": ms, "bytes": gb,
            "GB/s": gb / (ms / 1000.0) / 1e9, "chunks": -(-p.n_union // (1 << 22)),
            "roofline": {"bound": "alu", "kernel": "k_tensor_contrib", "achieved": achieved,
                         "peak": fpk, "unit": "TFLOP/s", "frac": achieved / fpk if achieved else None,
                         "kernel_ms_per_pass": kms.value / steps, "flops_per_entry": fpe,
                         "share_of_pass": (kms.value / steps) / ms, "peak_source": fsrc}}


def cp_bytes(p):
    """Algorithmic DRAM bytes of one S3CMTF-CP HOGWILD epoch: COO (4N + 4 B) and slot
    positions (4N B) per tensor entry, COO and positions (20 B) per coupled entry, and each
    touched row read and written once."""
    J = p.J[0]
    rows = sum(int(np.unique(p.train_idx[n]).shape[0]) for n in range(p.N))
    rows += sum(int(np.unique(c.cols).shape[0]) for c in p.coupled)
    ld = 4 * ((J + 3) // 4)
    return p.nnz * (8 * p.N + 4) + sum(c.nnz * 20 for c in p.coupled) + rows * ld * 4 * 2


def cp_params(p):
    """The seeded start of S3CMTF-CP: the usual factors and a hyper-diagonal N(0,1) core."""
    G, U, V = synth.init_params(p, 1)
    J = p.J[0]
    G = np.zeros(p.J)
    G[(np.arange(J),) * p.N] = np.random.default_rng(1).normal(size=J)
    return G, U, V


def cp_hogwild(p, order, stream, epochs=3):
    """S3CMTF-CP (hyper-diagonal core) on the same data: HOGWILD epoch time, test RMSE, and
    the roofline of its O(N J) per-entry kernel, which is bandwidth-shaped: algorithmic DRAM
    bytes = COO (4N + 4 B) and slot positions (4N B) per tensor entry, COO and positions
    (20 B) per coupled entry, and each touched row read and written once."""
    import ctypes as C

    import torch

    from paper_1708_08640_gb300 import _lib as L
    from paper_1708_08640_gb300.model import S3CMTF
    m = S3CMTF.from_problem(p, order=order, stream=stream, cp=1)
    m.set_params(*cp_params(p))
    m.set_test(p.test_idx, p.test_val)
    m.epoch("hogwild")
    L.check(m.lib, m.ctx, m.lib.s3_profile(m.ctx, 1))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(epochs):
        m.epoch("hogwild")
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / epochs
    kms, kn, ke = C.c_double(), C.c_int64(), C.c_int64()
    L.check(m.lib, m.ctx, m.lib.s3_profile_read(m.ctx, L.S3_K_TENSOR_HOG, C.byref(kms),
                                                  C.byref(kn), C.byref(ke)))
    L.check(m.lib, m.ctx, m.lib.s3_profile(m.ctx, 0))
    nbytes = cp_bytes(p)
    peaks, src = measured_peaks()
    k_ms = kms.value / epochs
    achieved = nbytes / (k_ms / 1000.0) / 1e9
    out = {"ms_per_epoch": ms, "nnz_updates_per_s": p.n_union / (ms / 1000.0),
           "test_rmse_after": m.rmse(), "epochs": 1 + epochs, "launch": m.hog_config("fp32"),
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                        "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                        "bytes_per_epoch": nbytes, "kernel_ms_per_epoch": k_ms,
                        "peak_source": f"{src} hbm_gbs"}}
    m.close()
    return out


def nonneg_hogwild(p, order, stream, epochs=4):
    """The non-negative form (projected SGD, Section 5) on the same data and start: FP32
    HOGWILD epoch time (each row and core atomic add followed by its projection), test RMSE
    per epoch, and the smallest parameter value afterwards (0 or more)."""
    import torch

    from paper_1708_08640_gb300.model import S3CMTF
    m = S3CMTF.from_problem(p, order=order, stream=stream, nonneg=1)
    m.set_params(*synth.init_params(p, 1))
    m.set_test(p.test_idx, p.test_val)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms, rmse = [], []
    for _ in range(epochs):
        torch.cuda.synchronize()
        e0.record(stream)
        m.epoch("hogwild")
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        rmse.append(m.rmse())
    G, U, V = m.get_params()
    low = min(float(x.min()) for x in [G, *U, *V])
    m.close()
    t = float(np.median(ms))
    return {"ms_per_epoch": t, "nnz_updates_per_s": p.n_union / (t / 1000.0),
            "test_rmse": rmse, "epochs": epochs, "min_parameter": low,
            "timing": "median of the epochs, each bracketed by CUDA events"}


# ----------------------------------------------------------------------------- our arm
SCAL_NNZ = (100_000, 1_000_000, 10_000_000, 100_000_000)     # at I = 10^4
SCAL_I = (1_000, 10_000, 100_000, 1_000_000, 10_000_000, 100_000_000)   # at |Omega| = 10^6
# the reduced sweep the default run carries (a few seconds of input generation)
SCAL_NNZ_QUICK = (250_000, 1_000_000, 4_000_000, 16_000_000)
SCAL_I_QUICK = (1_000, 10_000, 100_000)


def scalability_sweep(nnz_list, i_list, steps=3, warmup=1, stream=None):
    """Section 4.3 (data scalability): HOGWILD epoch time of the FP32 form on the synthetic
    I x I x I tensors, over |Omega| at I = 10^4 and over I at |Omega| = 10^6 (coupled
    I x I matrix with |Omega|/10 entries, J = 10).  The paper's claim: time linear in
    |Omega|, independent of I.  Returns the per-point times, the least-squares line of time
    over items with its R^2, and the largest / smallest time across I."""
    import torch

    from paper_1708_08640_gb300.model import S3CMTF
    stream = stream or torch.cuda.Stream()

    def one(I, nnz):
        p = synth.make_problem(f"scal:{I}:{nnz}")
        m = S3CMTF.from_problem(p, order=synth.union_order(p, 2), stream=stream)
        for _ in range(max(1, warmup)):
            m.epoch("hogwild")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            m.epoch("hogwild")
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        m.close()
        return {"I": I, "nnz": nnz, "train_nnz": p.nnz, "items": p.n_union, "ms_per_epoch": ms,
                "nnz_updates_per_s": p.n_union / (ms / 1000.0)}

    by_nnz = [one(10_000, n) for n in nnz_list]
    by_i = [one(i, 1_000_000) for i in i_list]
    x = np.array([r["items"] for r in by_nnz], dtype=np.float64)
    y = np.array([r["ms_per_epoch"] for r in by_nnz])
    slope, icpt = np.polyfit(x, y, 1)
    r2 = 1.0 - np.sum((y - (slope * x + icpt)) ** 2) / np.sum((y - y.mean()) ** 2)
    ti = np.array([r["ms_per_epoch"] for r in by_i])
    return {"over_nnz_at_I_1e4": by_nnz, "over_I_at_nnz_1e6": by_i,
            "linear_fit_ms_per_item": float(slope), "linear_fit_intercept_ms": float(icpt),
            "linear_fit_r2": float(r2), "time_ratio_max_over_min_across_I": float(ti.max() / ti.min())}


def run_scalability(args):
    """The full Section 4.3 sweeps (|Omega| from 10^5 to 10^8, I from 10^3 to 10^8) as the
    bench line's step."""
    import torch
    torch.cuda.set_device(0)
    sc = scalability_sweep(SCAL_NNZ, SCAL_I, args.steps, args.warmup)
    top = sc["over_nnz_at_I_1e4"][-1]
    line = {"metric": METRIC, "value": top["nnz_updates_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": top["ms_per_epoch"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "Section 4.3 scalability: I x I x I uniform tensors, coupled "
                                   "I x I matrix with |Omega|/10 entries, J = 10, FP32 HOGWILD",
                       "parallelism": "replicas x1"},
            "scalability": sc}
    print(json.dumps(line), flush=True)


def run_gradient(args, world, rank, local):
    """The differentiation form: one full-gradient pass (loss gradient with respect to the
    core, every factor and every coupled factor) per step; value = algorithmic GB/s."""
    import ctypes as C

    import torch
    import torch.distributed as dist

    from paper_1708_08640_gb300 import _lib as L
    from paper_1708_08640_gb300.model import S3CMTF

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    p = synth.make_problem(args.workload, seed=rank)
    if args.rank:
        p = synth.with_rank(p, (args.rank,) * p.N)
    stream = torch.cuda.Stream()
    model = S3CMTF.from_problem(p, order=synth.union_order(p, 2), stream=stream)
    model.set_params(*synth.init_params(p, 1))
    lib, ctx = model.lib, model.ctx
    gb = gradient_bytes(p)
    for _ in range(args.warmup):
        model.gradient()
    L.check(lib, ctx, lib.s3_profile(ctx, 1))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0.record(stream)
    for _ in range(args.steps):
        model.gradient()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    ms_total = ev0.elapsed_time(ev1)
    ms_total = max_over_ranks(ms_total, world)
    ms_step = ms_total / args.steps
    value = job_rate(gb, args.steps, world, ms_total / 1000.0) / 1e9

    def read(fam):
        ms, n, e = C.c_double(), C.c_int64(), C.c_int64()
        L.check(lib, ctx, lib.s3_profile_read(ctx, fam, C.byref(ms), C.byref(n), C.byref(e)))
        return ms.value, n.value, e.value

    k_ms, k_n, k_entries = read(L.S3_K_TENSOR_GRAD)
    _, launches, _ = read(L.S3_K_ALL)
    L.check(lib, ctx, lib.s3_profile(ctx, 0))
    fpe = flops_per_entry(p)
    achieved = fpe * k_entries / (k_ms / 1000.0) / 1e12 if k_ms > 0 else None
    fpk, fsrc = fp32_peak()
    wl = args.workload + (f"@J{args.rank}" if args.rank else "")
    roofline = {"bound": "alu", "achieved": achieved, "peak": fpk, "unit": "TFLOP/s",
                "frac": (achieved / fpk) if achieved else None,
                "traffic": committed_traffic("k_tensor_contrib", wl),
                "kernel": "k_tensor_contrib", "launches": k_n,
                "kernel_ms_per_step": k_ms / args.steps, "flops_per_entry": fpe,
                "peak_source": fsrc,
                "share_of_step": (k_ms / args.steps) / ms_step}
    # end to end through the public API: fresh values from pinned host memory, the pass,
    # and the whole gradient back to pinned host memory
    xv = torch.tensor(p.train_val, dtype=torch.float32).pin_memory()
    yv = [torch.tensor(c.vals, dtype=torch.float32).pin_memory() for c in p.coupled]
    dG, dU, dV = model.gradient()
    hosts = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in [dG, *dU, *dV]]
    d2h = sum(h.numel() * 4 for h in hosts)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        model.update_values(xv, yv)
        outs = model.gradient()
        with torch.cuda.stream(stream):
            for h, d in zip(hosts, [outs[0], *outs[1], *outs[2]]):
                h.copy_(d, non_blocking=True)
        stream.synchronize()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world)
    e2e = {"value": job_rate(gb, args.steps, world, e2e_s) / 1e9, "unit": "GB/s",
           "h2d_bytes_per_step": 4 * p.n_union, "d2h_bytes_per_step": d2h,
           "copies": "every step: the tensor and coupled values (FP32) from pinned host memory "
                     "in, the whole gradient (core, every factor, every coupled factor) out; "
                     "the coordinates stay resident"}
    cpu = None
    if rank == 0 and world == 1 and args.cpu_sample > 0:
        import oracle
        S = max(1000, min(args.cpu_sample // 20, p.nnz))
        q = sub_problem(p, S, max(1, S // 2))
        o = oracle.Oracle(q, **{k: v for k, v in q.hparams.items()
                               if k in ("lr0", "mu", "lambda_reg", "lambda_m", "batch", "core_scale")})
        o.set_params(*synth.init_params(q, 1))
        t0 = time.perf_counter()
        o.full_gradient()
        dt = time.perf_counter() - t0
        cpu = {"value": gradient_bytes(q) / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"full gradient of the first {q.nnz} tensor entries and "
                         f"{q.coupled[0].nnz if q.coupled else 0} entries of each coupled "
                         f"matrix, FP64, {dt:.1f} s"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": dict(workload_desc(p, "gradient"), parallelism=f"replicas x{world}",
                               bytes_per_step=gb),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk}
        print(json.dumps(line), flush=True)
    model.close()
    if world > 1:
        dist.destroy_process_group()


def _sig(x, n=4):
    return None if x is None else float(f"{x:.{n}g}")


def summary_of(extras):
    """The side measurements' headline figures in a few hundred bytes (the full objects follow
    in the line): per rank the BF16/FP32 epoch times, the BF16 speedup, both forms' largest
    test-RMSE deviation from the oracle's Algorithm 1 curve (where one is stored) and the
    gap between the two forms; the gradient pass in GB/s; the other epoch forms."""
    out = {}
    for key in ("forms_j10", "forms_j16", "forms_j20", "forms_j32"):
        f = extras.get(key)
        if not f:
            continue
        row = {"fp32_ms": _sig(f["fp32"]["ms_per_epoch"]), "bf16_ms": _sig(f["bf16"]["ms_per_epoch"]),
               "bf16_speedup": _sig(f["bf16_speedup"], 3),
               "bf16_tensor_frac": _sig(f["bf16"]["roofline"]["frac"], 3),
               "fp32_ffma_frac": _sig(f["fp32"]["roofline"]["frac"], 3),
               "rmse_gap_bf16_vs_fp32": _sig(f["rmse_max_rel_gap"], 2)}
        v = f.get("vs_oracle_algorithm1")
        if v:
            row["max_dev_vs_alg1"] = {prec: _sig(max(abs(x) for x in v[prec]), 3) for prec in ("fp32", "bf16")}
        out[key.replace("forms_", "")] = row
    g = {}
    if "gradient_pass" in extras:
        g["cfg1"] = _sig(extras["gradient_pass"]["GB/s"])
    if "gradient_pass_cfg3" in extras:
        g["cfg3"] = _sig(extras["gradient_pass_cfg3"]["GB/s"])
    if g:
        out["gradient_pass_GBps"] = g
    if "minibatch_epoch" in extras:
        out["minibatch_ms"] = _sig(extras["minibatch_epoch"]["ms"])
    if "cp_hogwild" in extras:
        out["cp_ms"] = _sig(extras["cp_hogwild"]["ms_per_epoch"])
    if "nonneg_hogwild" in extras:
        out["nonneg_ms"] = _sig(extras["nonneg_hogwild"]["ms_per_epoch"])
    sc = extras.get("scalability")
    if sc:
        out["scalability"] = {"r2_over_nnz": _sig(sc["linear_fit_r2"], 6),
                              "time_ratio_across_I": _sig(sc["time_ratio_max_over_min_across_I"], 3)}
    return out


def run_ours(args, world, rank, local):
    import ctypes as C

    import torch
    import torch.distributed as dist

    from paper_1708_08640_gb300 import _lib as L
    from paper_1708_08640_gb300.model import S3CMTF

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    # each rank fits its own replica problem (weak scaling)
    t_gen = time.perf_counter()
    p = synth.make_problem(args.workload, seed=rank)
    if args.rank:
        p = synth.with_rank(p, (args.rank,) * p.N)
    order = synth.union_order(p, 2)
    t_gen = time.perf_counter() - t_gen
    stream = torch.cuda.Stream()
    variant = {"cp": dict(cp=1), "nonneg": dict(nonneg=1)}.get(args.variant, {})
    t_init = time.perf_counter()
    model = S3CMTF.from_problem(p, order=order, stream=stream, **variant)
    torch.cuda.synchronize()
    t_init = time.perf_counter() - t_init
    model.set_params(*(cp_params(p) if args.variant == "cp" else synth.init_params(p, 1)))
    model.set_test(p.test_idx, p.test_val)
    lib, ctx = model.lib, model.ctx

    def step():
        model.epoch(args.mode, args.precision)
        return model.rmse()

    rmse0 = model.rmse()
    hog_launch = model.hog_config(args.precision) if args.mode == "hogwild" else None
    for _ in range(args.warmup):
        step()
    # ---- timed region
    L.check(lib, ctx, lib.s3_profile(ctx, 1))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0.record(stream)
    rmses = [step() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    ms_total = ev0.elapsed_time(ev1)
    ms_total = max_over_ranks(ms_total, world)
    ms_step = ms_total / args.steps
    items = p.n_union
    value = job_rate(items, args.steps, world, ms_total / 1000.0)
    # the same epochs, counted by kind of update (they run in one kernel)
    split = {"tensor_updates_per_s": world * p.nnz * args.steps / (ms_total / 1000.0),
             "coupled_updates_per_s": world * (p.n_union - p.nnz) * args.steps / (ms_total / 1000.0)}

    def read(fam):
        ms, n, e = C.c_double(), C.c_int64(), C.c_int64()
        L.check(lib, ctx, lib.s3_profile_read(ctx, fam, C.byref(ms), C.byref(n), C.byref(e)))
        return ms.value, n.value, e.value

    fam = L.S3_K_TENSOR_HOG if args.mode == "hogwild" else L.S3_K_TENSOR_MB
    k_ms, k_n, k_entries = read(fam)
    _, launches, _ = read(L.S3_K_ALL)
    L.check(lib, ctx, lib.s3_profile(ctx, 0))
    J = p.J
    flops_per_entry = 6.0 * float(np.prod(J)) if p.N == 3 else (
        6.0 * float(np.prod(J)) + 4.0 * float(np.prod(J[:3])))
    achieved = flops_per_entry * k_entries / (k_ms / 1000.0) / 1e12 if k_ms > 0 else None
    kname = "k_tensor_hog" if args.mode == "hogwild" else "k_mb_epoch"
    if args.precision == "bf16":
        kname = "k_tensor_hog_bf16"
        peaks, src = measured_peaks()
        peak, bound, psrc = peaks["bf16_tflops_sustained"], "tensor", f"{src} bf16_tflops_sustained"
    else:
        peak, psrc = fp32_peak()
        bound = "alu"
    wl = args.workload + (f"@J{args.rank}" if args.rank else "")
    traffic = committed_traffic(kname, wl)
    roofline = {"bound": bound, "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None,
                "traffic": traffic, "kernel": kname, "launches": k_n,
                "kernel_ms_per_step": k_ms / args.steps,
                "flops_per_entry": flops_per_entry, "peak_source": psrc}
    if args.variant == "cp" and args.mode == "hogwild":
        # O(N J) work per entry: the bandwidth roof of its algorithmic bytes
        peaks, src = measured_peaks()
        nbytes = cp_bytes(p)
        gbs = nbytes * k_n / (k_ms / 1000.0) / 1e9 if k_ms > 0 else None
        roofline = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": gbs / peaks["hbm_gbs"] if gbs else None,
                    "traffic": committed_traffic("k_cp_hog", wl), "kernel": "k_cp_hog",
                    "launches": k_n, "kernel_ms_per_step": k_ms / args.steps,
                    "bytes_per_launch": nbytes, "peak_source": f"{src} hbm_gbs"}

    extras = {}
    if args.forms and p.N == 3 and len(set(p.J)) == 1:
        extras[f"forms_j{p.J[0]}"] = precision_forms(p, order, stream, args, J=p.J[0],
                                                     epochs=args.steps, model=model)
    if not args.no_extras:
        # gradient pass (differentiation form): bytes moved per pass / time
        model.gradient()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ng = 3
        for _ in range(ng):
            model.gradient()
        e1.record(stream)
        torch.cuda.synchronize()
        g_ms = e0.elapsed_time(e1) / ng
        coo = p.nnz * (4 * p.N + 4) + sum(c.nnz * 12 for c in p.coupled)
        rows = sum(int(np.unique(p.train_idx[n]).shape[0]) * J[n] for n in range(p.N))
        rows += sum(int(np.unique(c.cols).shape[0]) * J[c.mode] for c in p.coupled)
        grad_out = int(np.prod(J)) + sum(d * j for d, j in zip(p.dims, J)) + sum(
            c.K * J[c.mode] for c in p.coupled)
        gbytes = coo + 4 * rows + 4 * grad_out
        extras["gradient_pass"] = {"ms": g_ms, "GB/s": gbytes / (g_ms / 1000.0) / 1e9,
                                   "bytes": gbytes}
        if args.mode != "minibatch":
            m2 = S3CMTF.from_problem(p, order=order, stream=stream)
            m2.set_params(*synth.init_params(p, 1))
            m2.epoch("minibatch")
            torch.cuda.synchronize()
            e0.record(stream)
            m2.epoch("minibatch")
            e1.record(stream)
            torch.cuda.synchronize()
            mb_ms = e0.elapsed_time(e1)
            extras["minibatch_epoch"] = {"ms": mb_ms, "nnz_updates_per_s": items / (mb_ms / 1000.0),
                                         "batches": model.info()["n_batches"]}
            m2.close()
        extras["cp_hogwild"] = cp_hogwild(p, order, stream)
        extras["nonneg_hogwild"] = nonneg_hogwild(p, order, stream)
        extras["forms_j10"] = precision_forms(p, order, stream, args, J=10)
        extras["forms_j16"] = precision_forms(p, order, stream, args, J=16)
        extras["forms_j20"] = precision_forms(p, order, stream, args, J=20, epochs=3)
        extras["forms_j32"] = precision_forms(p, order, stream, args, J=32, epochs=2)
        # the differentiation form at config 3's size (4-way, 45M train entries, two coupled
        # matrices, J = 8): the gradient pass in GB/s, the metric's second half
        extras["gradient_pass_cfg3"] = gradient_pass(synth.make_problem("cfg3"), stream)
        # Section 4.3's scalability claim, reduced sweep: epoch time linear in |Omega|, flat in I
        extras["scalability"] = scalability_sweep(SCAL_NNZ_QUICK, SCAL_I_QUICK, 3, 1, stream)

    # ---- end to end through the public API with host buffers
    xv = torch.tensor(p.train_val, dtype=torch.float32).pin_memory()
    yv = [torch.tensor(c.vals, dtype=torch.float32).pin_memory() for c in p.coupled]
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        model.update_values(xv, yv)
        model.epoch(args.mode, args.precision)
        model.rmse()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world)
    h2d = 4 * items + 4
    e2e = {"value": job_rate(items, args.steps, world, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 12,
           "copies": "every step: the tensor and coupled values (FP32) from pinned host memory "
                     "(s3_update_values) and the learning rate in, the test RMSE (FP64) and "
                     "status out; the coordinates and the layout built from them stay resident "
                     "(they are fixed for a fit)"}

    cpu = None
    if rank == 0 and world == 1 and args.cpu_sample > 0:
        cpu = cpu_baseline(p, min(args.cpu_sample, p.n_union), order)
        # the oracle on every host core beside it (the minibatch rule, one batch, mode-1 parts)
        cpu["all_cores"] = cpu_baseline_multicore(p, min(4 * args.cpu_sample, p.nnz))
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "bf16" if args.precision == "bf16" else "f32", "data": "synthetic",
                "summary": summary_of(extras),
                "config": dict(workload_desc(p, args.mode, args.precision),
                               parallelism=f"replicas x{world}", variant=args.variant,
                               setup_s={"generate": round(t_gen, 2), "init": round(t_init, 2),
                                        "init_what": "s3_init: inputs validated, layouts built "
                                                     "on the host and uploaded"},
                               hogwild_launch=hog_launch),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk, "updates_by_kind": split,
                "test_rmse": {"before": rmse0, "per_step": rmses}, **extras}
        print(json.dumps(line), flush=True)
    model.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.mode == "gradient":
        run_gradient(args, world, rank, local)
    elif args.mode == "scalability":
        if rank == 0:
            run_scalability(args)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
