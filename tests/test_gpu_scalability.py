"""Section 4.3's data-scalability claim on the GPU, at reduced sizes: the HOGWILD epoch
time grows linearly with the number of observed entries (I = 10^4, |Omega| from 2.5*10^5 to
1.6*10^7: least-squares R^2 >= 0.99), and does not grow with the dimensionality I while
the factor matrices stay in L2 (I = 10^3, 10^4, 10^5 at |Omega| = 10^6: largest over
smallest epoch time <= 1.5).  The same sweep, as bench.scalability_sweep, is reported by
the default bench run."""
import pytest

pytestmark = pytest.mark.gpu


def test_epoch_time_linear_in_entries_and_flat_in_dimensionality(cuda_lib):
    import bench
    sc = bench.scalability_sweep(bench.SCAL_NNZ_QUICK, bench.SCAL_I_QUICK, steps=3, warmup=1)
    times = [(r["items"], round(r["ms_per_epoch"], 3)) for r in sc["over_nnz_at_I_1e4"]]
    print("over |Omega|:", times, "R^2", sc["linear_fit_r2"])
    print("over I:", [(r["I"], round(r["ms_per_epoch"], 3)) for r in sc["over_I_at_nnz_1e6"]])
    assert sc["linear_fit_r2"] >= 0.99, sc
    assert sc["linear_fit_ms_per_item"] > 0
    assert sc["time_ratio_max_over_min_across_I"] <= 1.5, sc
