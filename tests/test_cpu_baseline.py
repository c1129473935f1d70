"""The multicore CPU baseline (the paper's Section 5 scheme) runs and converges.

It is benchmark infrastructure, not an oracle: only convergence and the count of
projections are checked (its threads race by design)."""
import numpy as np

from oracle import cpu_baseline
from paper_1401_4780_gb300 import synth


def test_multicore_scheme_converges_and_counts():
    s = synth.make_system(1 << 14, 1 << 12, 16, 8, row_norms="unit", value_dtype="f32")
    x = np.zeros(s.n, dtype=np.float32)
    total = 0
    for _ in range(40):
        done, secs, threads = cpu_baseline.run(s.m, s.row_ptr, s.col, s.val_store, s.b, x,
                                               threads=4, scans=1, seed=3)
        assert secs > 0.0 and threads == 4
        total += done
    assert total == 40 * s.m
    assert np.linalg.norm(x - s.x_true) <= 1e-5 * np.linalg.norm(s.x_true)


def test_single_thread_is_one_shuffled_scan_per_call():
    s = synth.make_system(500, 100, 6, 2, row_norms="lognormal", value_dtype="f32")
    x = np.zeros(s.n, dtype=np.float32)
    done, _, _ = cpu_baseline.run(s.m, s.row_ptr, s.col, s.val_store, s.b, x, threads=1,
                                  scans=3)
    assert done == 3 * s.m
    r0 = np.linalg.norm(s.b)
    A = np.zeros((s.m, s.n))
    for i in range(s.m):
        A[i, s.col[s.row_ptr[i]:s.row_ptr[i + 1]]] = s.val64[s.row_ptr[i]:s.row_ptr[i + 1]]
    assert np.linalg.norm(A @ x - s.b) < 0.5 * r0
