"""Host logic of the benchmark (no GPU): the algorithmic bytes of one trial
that the roofline divides by, and the committed-traffic lookup."""
import numpy as np
import scipy.sparse as sp

import bench


def test_trial_bytes_hand_count():
    # n = 3 variables, m = 2 rows (one equality, one inequality); Q has one
    # zero diagonal entry, which the solver stores explicitly.
    Q = sp.csr_matrix(np.array([[1.0, 2.0, 0.0], [2.0, 0.0, 0.0], [0.0, 0.0, 3.0]]))
    A = sp.csr_matrix(np.array([[1.0, 1.0, 0.0], [0.0, 1.0, 1.0]]))
    inst = dict(Q=Q, A=A, l_c=np.array([1.0, 0.0]), u_c=np.array([1.0, 2.0]))
    for v in (4, 8):
        nnz_h = 4 + 1  # Q's 4 stored entries plus the explicit zero diagonal of row 1
        mats = (v + 4) * (nnz_h + 2 * 4) + 4 * (2 * 3 + 2 + 2)
        want = mats + 14 * v * 3 + 20 * v * 1 + 12 * v * 1
        assert bench.trial_bytes(inst, v) == want


def test_trial_bytes_large_workload_matches_stated_figure():
    """The 1M-variable workload: 210 MB per trial in FP32, 358 MB in FP64 (the
    figures the roofline quotes), from the sizes alone."""
    n, m = 1_000_000, 500_000
    nnz_q, nnz_a = 4_999_994, 4_000_000  # band (3 per row) + random pairs; 8 per row of A

    class Fake:
        def __init__(self, shape, nnz, diag_zero=0):
            self.shape, self.nnz, self._dz = shape, nnz, diag_zero

        def diagonal(self):
            d = np.ones(self.shape[0])
            d[:self._dz] = 0.0
            return d

    inst = dict(Q=Fake((n, n), nnz_q), A=Fake((m, n), nnz_a), l_c=np.zeros(m), u_c=np.ones(m))
    assert abs(bench.trial_bytes(inst, 4) / 1e6 - 210.0) < 0.1
    assert abs(bench.trial_bytes(inst, 8) / 1e6 - 358.0) < 0.1


def test_captured_traffic_scales_per_launch():
    """Traffic per launch = the capture's DRAM bytes per trial x trials per
    launch, only while the kernel sources hash to the captured ones."""
    import json
    import os
    assert bench.captured_traffic(7, 10.0) is None  # no capture for that precision
    path = os.path.join(bench.ROOT, "profiles", "traffic_trials_fp32.json")
    per_trial = json.load(open(path))["dram_bytes_per_trial"]
    t = bench.captured_traffic(32, 2.0)
    assert t is None or t == 2.0 * per_trial
