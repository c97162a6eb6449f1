"""Host-side helpers of bench.py and of the scan autotuner (no GPU)."""
import numpy as np
import pytest

import bench
import graphgen as gg
from paper_1702_04645_gb300 import tune


def test_nmi_matches_library_and_its_special_cases():
    sk = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(4)
    for _ in range(6):
        a = rng.integers(0, 9, 700)
        b = np.where(rng.random(700) < 0.6, a, rng.integers(0, 5, 700))
        assert abs(bench.nmi(a, b) - sk.normalized_mutual_info_score(a, b)) < 1e-12
    a = rng.integers(0, 6, 300)
    assert bench.nmi(a, 100 - 3 * a) == pytest.approx(1.0)  # names do not matter
    assert bench.nmi(np.zeros(50), np.zeros(50)) == 1.0       # one community each


def test_rates_and_rank_max_without_a_process_group():
    assert bench.whole_job_rate(1000.0, 4, 500.0) == pytest.approx(8000.0)
    assert bench.max_over_ranks(3.5) == 3.5
    # algorithmic bytes of one scan: 8 per entry, 32 per node
    assert bench.scan_bytes(1048576, 31401261) == 284764520


def test_scan_tuning_shape_key():
    g = gg.random_small(200, 0.05, 3)
    k1 = tune.shape_key(g.row_ptr)
    k2 = tune.shape_key(g.row_ptr.copy())
    assert k1 == k2 and k1[0] == g.n and k1[1] == g.nnz and sum(k1[2]) == g.n
    h = gg.random_small(200, 0.2, 3)
    assert tune.shape_key(h.row_ptr) != k1
