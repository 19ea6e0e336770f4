"""Host logic of the learned schedule's labels (no GPU needed)."""
import numpy as np

from paper_1605_00930_gb300 import learned


def test_sweep_label_prefers_fewer_sweeps_within_margin():
    opts = (0, 1, 2, 4, 8)
    # rows: options; columns: blocks
    cyc = np.array([
        [100.0, 100.0, 100.0, 100.0],
        [96.0, 90.0, 99.0, 101.0],    # block 1: 10 % better with 1 sweep
        [95.0, 80.0, 60.0, 102.0],    # block 1: 2 is >5 % better than 1; block 2: 2 is 40 % better than 0
        [94.0, 79.0, 58.0, 103.0],    # within 5 % of the current best: ignored
        [10.0, 79.5, 57.0, 104.0],    # block 0: 8 sweeps by far the best
    ])
    np.testing.assert_array_equal(learned.sweep_label(cyc, opts, 0.05), [8, 2, 2, 0])


def test_sweep_label_zero_margin_is_argmin_with_ties_to_fewer():
    opts = (0, 1, 2)
    cyc = np.array([[5.0, 3.0, 2.0], [4.0, 3.0, 1.0], [4.0, 1.0, 1.0]])
    np.testing.assert_array_equal(learned.sweep_label(cyc, opts, 0.0), [1, 2, 1])
