"""The per-epoch log of S3CMTF.fit: one JSON line per epoch with its number, learning rate,
loss of Eq. (7), train and test RMSE, device time and nnz-updates/s.  On the deterministic
minibatch epoch the logged loss, train RMSE and test RMSE are the FP64 oracle's after the
same epochs (1e-4 relative, the bound of the multi-epoch minibatch parity tests), and the
learning rate is the oracle's eta_t of Section 3.4."""
import json

import numpy as np
import pytest

from paper_1708_08640_gb300 import synth
from tests.gpu_common import make_pair

pytestmark = pytest.mark.gpu


def test_fit_logs_every_epoch_and_matches_the_oracle(cuda_lib, tmp_path):
    p = synth.make_problem("cfg0")
    gpu, orc, q, order = make_pair(p, batch=256)
    gpu.set_test(q.test_idx, q.test_val)
    log = tmp_path / "fit.jsonl"
    recs = gpu.fit(3, mode="minibatch", log=str(log))
    lines = [json.loads(x) for x in log.read_text().splitlines()]
    assert lines == recs
    assert [r["epoch"] for r in recs] == [0, 1, 2]
    n_train = q.train_val.shape[0]
    for t, r in enumerate(recs):
        orc.epoch_minibatch(t, order)
        assert r["eta"] == pytest.approx(orc.learning_rate(t), rel=1e-12)
        f, sse, _ = orc.loss()
        assert abs(r["loss"] - f) / f <= 1e-4, (t, r["loss"], f)
        assert abs(r["train_rmse"] - np.sqrt(sse / n_train)) / np.sqrt(sse / n_train) <= 1e-4
        ref = orc.rmse(q.test_idx, q.test_val)
        assert abs(r["test_rmse"] - ref) / ref <= 1e-4
        assert r["epoch_ms"] > 0 and r["nnz_updates_per_s"] > 0
        assert r["mode"] == "minibatch" and r["precision"] == "fp32"
    # appending: a second call continues the epoch count in the same file
    more = gpu.fit(1, mode="hogwild", log=str(log))
    assert more[0]["epoch"] == 3
    assert len(log.read_text().splitlines()) == 4
    gpu.close()
