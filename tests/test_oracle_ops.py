"""Pins of the reconstruction-based operators' plain definitions (oracle/ops.py)."""
import numpy as np
import pytest

from oracle import ops
from paper_1605_00930_gb300 import synth


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_regional_maxima_two_definitions_agree(conn, dtype):
    rng = np.random.default_rng([90, conn, np.dtype(dtype).itemsize])
    for trial in range(120):
        H, W = int(rng.integers(1, 12)), int(rng.integers(1, 12))
        f = rng.integers(0, 6 if trial % 2 else 300, size=(H, W)).astype(dtype)   # plateaus and ties
        np.testing.assert_array_equal(ops.regional_maxima(f, conn), ops.regional_maxima_flood(f, conn))


def test_hmaxima_and_dome_properties():
    f = synth.blob_field_u8(120, 170, 12, synth.rng_for(91))
    for conn in (4, 8):
        for h in (0, 1, 15, 60, 255):
            hm = ops.hmaxima(f, h, conn)
            dome = ops.hdome(f, h, conn)
            assert np.all(hm <= f) and np.all(hm.astype(int) >= f.astype(int) - h)   # f - h <= HMAX <= f
            np.testing.assert_array_equal(dome.astype(int), f.astype(int) - hm.astype(int))
            assert dome.max() <= h
        np.testing.assert_array_equal(ops.hmaxima(f, 0, conn), f)   # h = 0 changes nothing


def test_hand_case():
    """Two peaks on a plateau: the h-maxima transform clips the lower one to its saddle."""
    f = np.array([[1, 1, 1, 1, 1, 1, 1],
                  [1, 5, 1, 1, 1, 9, 1],
                  [1, 1, 1, 1, 1, 1, 1]], np.uint8)
    hm = ops.hmaxima(f, 3, 8)
    exp = np.array([[1, 1, 1, 1, 1, 1, 1],
                    [1, 2, 1, 1, 1, 6, 1],
                    [1, 1, 1, 1, 1, 1, 1]], np.uint8)
    np.testing.assert_array_equal(hm, exp)
    rm = np.zeros_like(f)
    rm[1, 1] = rm[1, 5] = 1
    np.testing.assert_array_equal(ops.regional_maxima(f, 8), rm)
