"""Writes the stored oracle curves used by the GPU curve tests.

Calls only ``oracle`` (FP64 CPU) and the seeded input generator.  For each workload it
records a fingerprint of the generated inputs (so a test can verify it regenerated the
same data) and the test RMSE after every epoch of
  - the sequential epoch of Algorithm 1 (P = 1), and
  - the deterministic minibatch epoch (batch 4096, row sum, core_scale 32),
starting from the seeded initial parameters and the seeded visiting order.  With the
fourth argument ``nonneg`` it writes the curves of the non-negative form (projected SGD,
Section 5) to curve_<workload>_<mode>_nonneg.json.

usage: python tests/golden/make_golden.py cfg1_small [epochs] [modes] [nonneg]
"""
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


def curve(p, mode, epochs, hparams):
    o = oracle.Oracle(p, **hparams, **(MB if mode == "minibatch" else {}))
    o.set_params(*synth.init_params(p, 1))
    order = synth.union_order(p, 2)
    out = []
    for t in range(epochs):
        (o.epoch_minibatch if mode == "minibatch" else o.epoch_sequential)(t, order)
        out.append(o.rmse(p.test_idx, p.test_val))
    return out


def main():
    name = sys.argv[1]
    epochs = int(sys.argv[2]) if len(sys.argv) > 2 else 10
    modes = sys.argv[3].split(",") if len(sys.argv) > 3 else ["sequential", "minibatch"]
    nonneg = len(sys.argv) > 4 and sys.argv[4] == "nonneg"
    hparams = dict(HPARAMS, nonneg=1) if nonneg else HPARAMS
    p = synth.make_problem(name)
    for mode in modes:
        t0 = time.time()
        rec = dict(workload=name, mode=mode, recipe=p.recipe, fingerprint=fingerprint(p),
                   hparams=hparams, minibatch=MB if mode == "minibatch" else None,
                   init_seed=1, order_seed=2, epochs=epochs,
                   source="oracle/ (FP64 CPU), written by tests/golden/make_golden.py")
        rec["test_rmse"] = curve(p, mode, epochs, hparams)
        rec["seconds"] = round(time.time() - t0, 1)
        path = os.path.join(HERE, f"curve_{name}_{mode}{'_nonneg' if nonneg else ''}.json")
        json.dump(rec, open(path, "w"), indent=1)
        print(mode, rec["test_rmse"], flush=True)


if __name__ == "__main__":
    main()
