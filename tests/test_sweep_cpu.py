"""Host-side pieces of the ablation sweep: the paper's quantile scores and the report tables."""
import numpy as np

from paper_2208_09985_gb300 import sweep


def test_worst_quantile_counts_from_the_worst_pair():
    # for 1000 pairs the 0.01 quantile is the 10th worst score and the 0.5 quantile the 500th worst
    v = np.random.default_rng(1).permutation(1000)
    assert sweep.worst_quantile(v, 0.01) == 990
    assert sweep.worst_quantile(v, 0.5) == 500
    assert sweep.worst_quantile(v, 0.001) == 999
    assert sweep.worst_quantile([3.0], 0.001) == 3.0
    assert np.isnan(sweep.worst_quantile([], 0.5))


def test_summary_reports_quantiles_and_same_kernel_sene():
    q = {str(x): {"windowed": 12, "exact": 10, "excess": 2} for x in sweep.QUANTILES}
    base = {"rate": 0.1, "W": 64, "O": 33, "k": 64, "mean_edits": 10.0, "free_end_mean": 9.5,
            "mean_excess_over_free_end": 0.5, "pairs_at_optimum": 0.97, "mean_rows_per_window": 7.7,
            "quantiles": q, "dent": 1, "et": 1, "method_table_bytes_per_window": 100.0,
            "smem_bytes_per_pair": 64.0, "kernel": "band"}
    rows = [dict(base, sene=1, form="plain", alignments_per_s=4e6), dict(base, sene=1, form="learned", alignments_per_s=4.2e6),
            dict(base, sene=1, form="full", alignments_per_s=3e6), dict(base, sene=0, form="plain", alignments_per_s=1e6),
            dict(base, sene=0, form="learned", alignments_per_s=1.1e6)]
    text = sweep.summary(rows)
    assert "12 / 10 / 2" in text
    assert "| 0.10 | 64 | 33 | 3.000M | 1.000M | 3.00 |" in text
