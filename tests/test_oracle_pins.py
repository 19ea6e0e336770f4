"""Pins for the CPU oracle (Vincent's hybrid, Sec. 3.1 Algorithm 7) and the
brute force (Sec. 2.1.2 Algorithm 1), against things other than themselves:
hand-worked cases, exhaustive random comparison between the two independent
algorithms, invariants of reconstruction, duality, threshold decomposition and
the binary special cases that reduce to library routines (connected-component
labelling, binary hole filling)."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import bruteforce
from paper_1605_00930_gb300 import synth
from tests._golden import load_hand_cases

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

STRUCT = {4: ndimage.generate_binary_structure(2, 1), 8: np.ones((3, 3), dtype=bool)}


def _random_case(rng, H, W, dtype, op, vmax=None):
    top = synth.maxval(dtype)
    vmax = top if vmax is None else vmax
    mask = rng.integers(0, vmax + 1, size=(H, W)).astype(dtype)
    kind = rng.integers(0, 3)
    if op == "dilate":
        if kind == 0:
            marker = (mask.astype(np.int64) * (rng.random((H, W)) < 0.15)).astype(dtype)
        elif kind == 1:
            marker = np.maximum(mask.astype(np.int64) - rng.integers(0, vmax // 2 + 2), 0).astype(dtype)
        else:
            marker = (mask.astype(np.int64) * rng.random((H, W))).astype(dtype)
    else:
        if kind == 0:
            marker = synth.fillholes_marker(mask)
        elif kind == 1:
            marker = np.minimum(mask.astype(np.int64) + rng.integers(0, vmax // 2 + 2), top).astype(dtype)
        else:
            lift = (rng.random((H, W)) * (top - mask.astype(np.int64))).astype(np.int64)
            marker = (mask.astype(np.int64) + lift).astype(dtype)
    return marker, mask


# ---- hand-worked cases ----------------------------------------------------------

@pytest.mark.parametrize("case", load_hand_cases(), ids=lambda c: c["name"])
def test_hand_cases(oracle_lib, case):
    for conn in case["conn"]:
        got = oracle_lib.reconstruct(case["marker"], case["mask"], conn, case["op"])
        np.testing.assert_array_equal(got, case["expected"], err_msg=f"oracle conn={conn}")
        bf = bruteforce.reconstruct(case["marker"], case["mask"], conn, case["op"])
        np.testing.assert_array_equal(bf, case["expected"], err_msg=f"bruteforce conn={conn}")


# ---- the two independent algorithms agree on tiny inputs -------------------------

@pytest.mark.parametrize("op", ["dilate", "erode"])
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("conn", [4, 8])
def test_oracle_matches_bruteforce_random(oracle_lib, op, dtype, conn):
    rng = np.random.default_rng([7, conn, int(np.dtype(dtype).itemsize), op == "erode"])
    for it in range(400):
        H, W = int(rng.integers(1, 13)), int(rng.integers(1, 13))
        vmax = [3, 15, None][it % 3]
        marker, mask = _random_case(rng, H, W, dtype, op, vmax)
        got = oracle_lib.reconstruct(marker, mask, conn, op)
        exp = bruteforce.reconstruct(marker, mask, conn, op)
        np.testing.assert_array_equal(got, exp, err_msg=f"H={H} W={W} it={it}")


@pytest.mark.parametrize("shape", [(1, 1), (1, 17), (17, 1), (2, 2), (1, 2), (2, 1), (3, 40)])
@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_oracle_edge_shapes(oracle_lib, shape, op):
    rng = np.random.default_rng(11)
    for conn in (4, 8):
        for _ in range(20):
            marker, mask = _random_case(rng, *shape, np.uint8, op, 9)
            np.testing.assert_array_equal(oracle_lib.reconstruct(marker, mask, conn, op),
                                          bruteforce.reconstruct(marker, mask, conn, op))


def test_fillholes_thin_images_are_identity(oracle_lib):
    # With H = 1 or W = 1 every pixel lies on the border, so fill-holes returns I.
    rng = np.random.default_rng(3)
    for shape in [(1, 9), (9, 1), (1, 1)]:
        mask = rng.integers(0, 256, size=shape).astype(np.uint8)
        for conn in (4, 8):
            np.testing.assert_array_equal(
                oracle_lib.reconstruct(synth.fillholes_marker(mask), mask, conn, "erode"), mask)


# ---- invariants ---------------------------------------------------------------------

def _one_step(J, I, conn, op):
    ext = bruteforce._neigh_extreme(J.astype(np.int64), conn, op)
    return np.minimum(ext, I) if op == "dilate" else np.maximum(ext, I)


@pytest.mark.parametrize("op", ["dilate", "erode"])
@pytest.mark.parametrize("conn", [4, 8])
def test_invariants(oracle_lib, op, conn):
    rng = np.random.default_rng([23, conn, op == "erode"])
    for it in range(40):
        H, W = int(rng.integers(1, 40)), int(rng.integers(1, 40))
        marker, mask = _random_case(rng, H, W, np.uint8, op, [7, 60, 255][it % 3])
        R = oracle_lib.reconstruct(marker, mask, conn, op)
        m64, I64, R64 = (a.astype(np.int64) for a in (marker, mask, R))
        if op == "dilate":
            assert (m64 <= R64).all() and (R64 <= I64).all()
        else:
            assert (m64 >= R64).all() and (R64 >= I64).all()
        # stability: R is a fixed point of the elementary step
        np.testing.assert_array_equal(_one_step(R, I64, conn, op), R64)
        # idempotence
        np.testing.assert_array_equal(oracle_lib.reconstruct(R, mask, conn, op), R)
        # R(I, I) = I
        np.testing.assert_array_equal(oracle_lib.reconstruct(mask.copy(), mask, conn, op), mask)


@pytest.mark.parametrize("conn", [4, 8])
def test_zero_marker_and_monotonicity(oracle_lib, conn):
    rng = np.random.default_rng([29, conn])
    for _ in range(30):
        H, W = int(rng.integers(2, 30)), int(rng.integers(2, 30))
        mask = rng.integers(0, 20, size=(H, W)).astype(np.uint8)
        zero = np.zeros_like(mask)
        np.testing.assert_array_equal(oracle_lib.reconstruct(zero, mask, conn, "dilate"), zero)
        J1 = (mask * (rng.random((H, W)) < 0.1)).astype(np.uint8)
        J2 = np.maximum(J1, (mask * (rng.random((H, W)) < 0.1)).astype(np.uint8))
        R1 = oracle_lib.reconstruct(J1, mask, conn, "dilate")
        R2 = oracle_lib.reconstruct(J2, mask, conn, "dilate")
        assert (R1 <= R2).all()  # monotone in the marker
        bigger = np.minimum(mask.astype(np.int64) + rng.integers(0, 5, (H, W)), 255).astype(np.uint8)
        R3 = oracle_lib.reconstruct(J1, bigger, conn, "dilate")
        assert (R1 <= R3).all()  # monotone in the mask


def test_hdome_bound(oracle_lib):
    case = synth.tissue_case(192, 160, nblobs=12)
    for conn in (4, 8):
        R = oracle_lib.reconstruct(case.marker, case.mask, conn, "dilate").astype(np.int64)
        d = case.mask.astype(np.int64) - R
        assert d.min() >= 0 and d.max() <= 30


# ---- duality ----------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("conn", [4, 8])
def test_duality(oracle_lib, dtype, conn):
    rng = np.random.default_rng([31, conn])
    top = synth.maxval(dtype)
    C = lambda a: (top - a.astype(np.int64)).astype(dtype)
    for it in range(40):
        H, W = int(rng.integers(1, 30)), int(rng.integers(1, 30))
        marker, mask = _random_case(rng, H, W, dtype, "erode", [5, 100, None][it % 3])
        ero = oracle_lib.reconstruct(marker, mask, conn, "erode")
        dil = oracle_lib.reconstruct(C(marker), C(mask), conn, "dilate")
        np.testing.assert_array_equal(ero, C(dil))


# ---- binary special cases = library routines -------------------------------------------

def _binary_recon(seed_bin, mask_bin, conn):
    lab, _ = ndimage.label(mask_bin, structure=STRUCT[conn])
    keep = np.unique(lab[seed_bin & mask_bin])
    keep = keep[keep > 0]
    return np.isin(lab, keep) & mask_bin


@pytest.mark.parametrize("conn", [4, 8])
def test_binary_is_connected_component_selection(oracle_lib, conn):
    rng = np.random.default_rng([37, conn])
    for _ in range(30):
        H, W = int(rng.integers(1, 70)), int(rng.integers(1, 70))
        I = (rng.random((H, W)) < rng.uniform(0.3, 0.75)).astype(np.uint8)
        J = (I & (rng.random((H, W)) < 0.03)).astype(np.uint8)
        R = oracle_lib.reconstruct(J, I, conn, "dilate")
        np.testing.assert_array_equal(R.astype(bool), _binary_recon(J.astype(bool), I.astype(bool), conn))


@pytest.mark.parametrize("conn", [4, 8])
def test_binary_fill_holes_matches_scipy(oracle_lib, conn):
    rng = np.random.default_rng([41, conn])
    for _ in range(30):
        H, W = int(rng.integers(1, 60)), int(rng.integers(1, 60))
        I = (rng.random((H, W)) < rng.uniform(0.4, 0.8)).astype(np.uint8)
        R = oracle_lib.reconstruct(synth.fillholes_marker(I), I, conn, "erode")
        exp = ndimage.binary_fill_holes(I.astype(bool), structure=STRUCT[conn])
        np.testing.assert_array_equal(R.astype(bool), exp)


@pytest.mark.parametrize("conn", [4, 8])
def test_threshold_decomposition(oracle_lib, conn):
    """R(p) >= t  <=>  p lies in the binary reconstruction of {I >= t} from {J >= t}."""
    cases = [synth.tissue_case(96, 130, conn=conn, nblobs=6),
             synth.noise_blur_case(64, 77)]
    cases[1].conn = conn
    for c in cases:
        R = oracle_lib.reconstruct(c.marker, c.mask, conn, "dilate")
        levels = np.unique(np.concatenate([c.mask.ravel(), c.marker.ravel()]))
        for t in levels[levels > 0]:
            exp = _binary_recon(c.marker >= t, c.mask >= t, conn)
            np.testing.assert_array_equal(R >= t, exp, err_msg=f"t={t}")


# ---- argument checking and precondition --------------------------------------------

def test_precondition_detection(oracle_lib):
    mask = np.full((4, 5), 10, np.uint8)
    marker = np.zeros_like(mask)
    assert oracle_lib.precondition_ok(marker, mask, "dilate")
    marker[2, 3] = 11
    assert not oracle_lib.precondition_ok(marker, mask, "dilate")
    assert oracle_lib.precondition_ok(np.full_like(mask, 10), mask, "erode")
    low = np.full_like(mask, 10)
    low[0, 0] = 9
    assert not oracle_lib.precondition_ok(low, mask, "erode")


def test_oracle_rejects_bad_arguments(oracle_lib):
    a = np.zeros((3, 3), np.uint8)
    with pytest.raises(ValueError):
        oracle_lib.reconstruct(a, a, 6, "dilate")
    with pytest.raises(ValueError):
        oracle_lib.reconstruct(a, np.zeros((3, 3), np.uint16), 8, "dilate")
    with pytest.raises(ValueError):
        bruteforce.reconstruct(a, a, 6, "dilate")
