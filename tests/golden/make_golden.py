"""Writes the stored oracle curves used by the GPU curve tests.

Calls only ``oracle`` (FP64 CPU) and the seeded input generator.  For each workload it
records a fingerprint of the generated inputs (so a test can verify it regenerated the
same data) and the test RMSE after every epoch of
  - the sequential epoch of Algorithm 1 (P = 1), and
  - the deterministic minibatch epoch (batch 4096, row sum, core_scale 32),
starting from the seeded initial parameters and the seeded visiting order.  With
``--nonneg`` it writes the curves of the non-negative form (projected SGD, Section 5) to
curve_<workload>_<mode>_nonneg.json.  With ``--rank J`` the workload is fitted at ranks
(J, J, J) (the rating workloads at other ranks, with the core step scale of that rank) and
the file is curve_<workload>_j<J>_<mode>.json.  The file is rewritten after every epoch,
so a long run leaves the epochs it has finished.

usage: python tests/golden/make_golden.py cfg1_small [--epochs 10]
           [--modes sequential,minibatch] [--nonneg] [--rank J]
"""
import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1708_08640_gb300 import synth  # noqa: E402

HPARAMS = dict(lr0=0.001, mu=0.1, lambda_reg=0.1, lambda_m=10.0)
MB = dict(batch=4096, row_mean=0, core_scale=32.0)


def fingerprint(p):
    h = hashlib.sha256()
    for a in (p.train_idx, p.train_val, p.test_idx, p.test_val):
        h.update(np.ascontiguousarray(a).tobytes())
    for c in p.coupled:
        for a in (c.rows, c.cols, c.vals):
            h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()[:16]


def curve(p, mode, epochs, hparams, rec, path):
    o = oracle.Oracle(p, **hparams, **(MB if mode == "minibatch" else {}))
    o.set_params(*synth.init_params(p, 1))
    order = synth.union_order(p, 2)
    t0 = time.time()
    rec["test_rmse"] = []
    for t in range(epochs):
        (o.epoch_minibatch if mode == "minibatch" else o.epoch_sequential)(t, order)
        rec["test_rmse"].append(o.rmse(p.test_idx, p.test_val))
        rec["epochs"] = t + 1
        rec["seconds"] = round(time.time() - t0, 1)
        json.dump(rec, open(path, "w"), indent=1)
        print(mode, t, rec["test_rmse"][-1], rec["seconds"], flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload")
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--modes", default="sequential,minibatch")
    ap.add_argument("--nonneg", action="store_true")
    ap.add_argument("--rank", type=int, default=0)
    a = ap.parse_args()
    hparams = dict(HPARAMS, nonneg=1) if a.nonneg else dict(HPARAMS)
    p = synth.make_problem(a.workload)
    tag = a.workload
    if a.rank:
        p = synth.with_rank(p, (a.rank,) * p.N)
        tag = f"{a.workload}_j{a.rank}"
    for mode in a.modes.split(","):
        rec = dict(workload=a.workload, rank=list(p.J), mode=mode, recipe=p.recipe,
                   fingerprint=fingerprint(p), hparams=hparams,
                   minibatch=MB if mode == "minibatch" else None, init_seed=1, order_seed=2,
                   source="oracle/ (FP64 CPU), written by tests/golden/make_golden.py")
        path = os.path.join(HERE, f"curve_{tag}_{mode}{'_nonneg' if a.nonneg else ''}.json")
        curve(p, mode, a.epochs, hparams, rec, path)


if __name__ == "__main__":
    main()
