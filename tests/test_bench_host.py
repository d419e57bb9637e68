"""Host logic of bench.py, without a GPU: the compact summary of the side measurements, the
DRAM-traffic records (used only while the kernel's sources are those they were taken on),
and the algorithmic bytes of the S3CMTF-CP epoch."""
import os

import numpy as np

import bench
from paper_1708_08640_gb300 import synth


def _forms(fp32_ms, bf16_ms, dev=None):
    f = {"fp32": {"ms_per_epoch": fp32_ms, "roofline": {"frac": 0.2}},
         "bf16": {"ms_per_epoch": bf16_ms, "roofline": {"frac": 0.02}},
         "bf16_speedup": fp32_ms / bf16_ms, "rmse_max_rel_gap": 1e-4}
    if dev is not None:
        f["vs_oracle_algorithm1"] = {"fp32": dev, "bf16": [-x for x in dev], "source": "x"}
    return f


def test_summary_carries_the_headline_figures():
    extras = {"forms_j16": _forms(11.7, 7.3, [0.002, -0.0049, 0.001]),
              "forms_j20": _forms(21.4, 9.9),
              "gradient_pass": {"GB/s": 60.2}, "gradient_pass_cfg3": {"GB/s": 30.2},
              "minibatch_epoch": {"ms": 41.1}, "cp_hogwild": {"ms_per_epoch": 3.0},
              "nonneg_hogwild": {"ms_per_epoch": 5.3},
              "scalability": {"linear_fit_r2": 0.9999986, "time_ratio_max_over_min_across_I": 1.03}}
    s = bench.summary_of(extras)
    assert s["j16"]["bf16_speedup"] == 1.6
    assert s["j16"]["max_dev_vs_alg1"] == {"fp32": 0.0049, "bf16": 0.0049}
    assert "max_dev_vs_alg1" not in s["j20"]          # no stored oracle curve at that rank
    assert s["gradient_pass_GBps"] == {"cfg1": 60.2, "cfg3": 30.2}
    assert s["minibatch_ms"] == 41.1 and s["cp_ms"] == 3.0 and s["nonneg_ms"] == 5.3
    assert s["scalability"]["r2_over_nnz"] == 0.999999
    assert bench.summary_of({}) == {}


def test_traffic_record_is_used_only_on_the_sources_it_was_taken_on(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    csrc = tmp_path / "paper_1708_08640_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES["k_tensor_hog"]:
        (tmp_path / f).write_text("source of " + os.path.basename(f))
    (tmp_path / "profiles").mkdir()
    sha = bench.source_sha("k_tensor_hog")
    (tmp_path / "profiles" / "traffic.txt").write_text(
        f"kernel=k_tensor_hog workload=cfg1 sha={sha} bytes_per_launch=750985216 source=x (note)\n")
    assert bench.committed_traffic("k_tensor_hog", "cfg1") == 750985216.0
    assert bench.committed_traffic("k_tensor_hog", "cfg1@J16") is None    # another workload
    assert bench.committed_traffic("k_unknown", "cfg1") is None
    (tmp_path / bench.KERNEL_SOURCES["k_tensor_hog"][0]).write_text("changed")
    assert bench.committed_traffic("k_tensor_hog", "cfg1") is None        # sources changed


def test_committed_traffic_records_parse():
    """Every line of profiles/traffic.txt names a known kernel, a summary that exists and a
    positive byte count."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for line in open(os.path.join(root, "profiles", "traffic.txt")):
        f = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        assert f["kernel"] in bench.KERNEL_SOURCES
        assert float(f["bytes_per_launch"]) > 0
        assert os.path.exists(os.path.join(root, f["source"]))


def test_cp_bytes_counts_coo_positions_and_touched_rows():
    p = synth.make_problem("cfg0")
    rows = sum(int(np.unique(p.train_idx[n]).shape[0]) for n in range(p.N))
    rows += sum(int(np.unique(c.cols).shape[0]) for c in p.coupled)
    ld = 4 * ((p.J[0] + 3) // 4)
    expect = p.nnz * (8 * p.N + 4) + sum(c.nnz * 20 for c in p.coupled) + rows * ld * 8
    assert bench.cp_bytes(p) == expect
