"""Host-side helpers of the shrinking study (no GPU)."""
import math

import numpy as np

from paper_2603_23891_gb300 import shrink_study


def test_kpc_summary_bins_and_counts():
    k = np.array([0.0, 0.005, 0.01, 0.049, 0.05, 0.3, 1.0, 4.99, 5.0, 70.0], np.float64)
    s = shrink_study.kpc_summary(k)
    assert s["pairs"] == 10
    assert sum(s["counts"]) == 10
    # [0,.01) [.01,.05) [.05,.1) [.1,.2) [.2,.5) [.5,1) [1,2) [2,5) [5,inf)
    assert s["counts"] == [2, 2, 1, 0, 1, 0, 1, 1, 2]
    assert s["below_0.01"] == 2 and s["below_0.05"] == 4
    assert s["edges"][-1] == "inf" and len(s["edges"]) == len(s["counts"]) + 1


def test_merge_summaries_adds():
    a = shrink_study.kpc_summary(np.array([0.0, 1.0]))
    b = shrink_study.kpc_summary(np.array([0.02, 0.03, 7.0]))
    m = shrink_study.merge_summaries(shrink_study.merge_summaries(None, a), b)
    assert m["pairs"] == 5 and m["below_0.05"] == 3 and m["below_0.01"] == 1
    assert sum(m["counts"]) == 5
    assert shrink_study.LAMBDAS[0] == 0.02 and shrink_study.LAMBDAS[-1] == 0.43
    assert math.isinf(shrink_study.KPC_EDGES[-1])
