"""Pins of the oracle's marker-controlled watershed (flooding of (level, label) pairs):

  * the levels are unique: they equal brute-force Jacobi relaxation of the same rule and
    the reconstruction by erosion of the marker levels under the gradient (marker =
    gradient at the markers, maximum elsewhere) — an independent, pinned routine;
  * labels (order-dependent where several markers reach a pixel at its level): markers
    keep theirs, every label is delivered by a neighbour at the pixel's level, no
    neighbour offers a smaller pair; one marker labels everything; a ridge between two
    markers splits the labels; no marker reaches nothing.
"""
import numpy as np
import pytest

import oracle
from paper_1605_00930_gb300 import synth
from tests._wshed_checks import check_labels

NB = {4: [(-1, 0), (0, -1), (0, 1), (1, 0)],
      8: [(-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 1), (1, -1), (1, 0), (1, 1)]}


def brute(markers, grad, conn):
    H, W = grad.shape
    INF = 1 << 40
    lev = np.where(markers > 0, grad.astype(np.int64), INF)
    lab = np.where(markers > 0, markers.astype(np.int64), INF)
    while True:
        nl, nb = lev.copy(), lab.copy()
        for y in range(H):
            for x in range(W):
                if markers[y, x]:
                    continue
                for dy, dx in NB[conn]:
                    yy, xx = y + dy, x + dx
                    if 0 <= yy < H and 0 <= xx < W and lev[yy, xx] < INF:
                        cl, cb = max(lev[yy, xx], int(grad[y, x])), lab[yy, xx]
                        if (cl, cb) < (nl[y, x], nb[y, x]):
                            nl[y, x], nb[y, x] = cl, cb
        if np.array_equal(nl, lev) and np.array_equal(nb, lab):
            break
        lev, lab = nl, nb
    return np.where(lab == INF, 0, lab).astype(np.uint32), np.where(lev == INF, -1, lev).astype(np.int32)


@pytest.mark.parametrize("conn", [4, 8])
def test_brute_force(conn):
    rng = np.random.default_rng([100, conn])
    for trial in range(80):
        H, W = int(rng.integers(1, 10)), int(rng.integers(1, 10))
        grad = rng.integers(0, 5 if trial % 2 else 255, size=(H, W)).astype(np.uint8)
        markers = np.zeros((H, W), np.uint32)
        for _ in range(int(rng.integers(0, 4))):
            markers[rng.integers(0, H), rng.integers(0, W)] = rng.integers(1, 9)
        lab, lev = oracle.watershed(markers, grad, conn)
        _, blev = brute(markers, grad, conn)
        np.testing.assert_array_equal(lev, blev)
        check_labels(markers, grad, lab, lev, conn)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("conn", [4, 8])
def test_levels_are_reconstruction_by_erosion(dtype, conn):
    f = synth.blob_field_u8(90, 130, 10, synth.rng_for(101))
    grad = synth.to_u16(f) if dtype == np.uint16 else f
    rng = np.random.default_rng(102)
    markers = np.zeros(grad.shape, np.uint32)
    ys, xs = rng.integers(0, 90, 12), rng.integers(0, 130, 12)
    markers[ys, xs] = np.arange(1, 13)
    lab, lev = oracle.watershed(markers, grad, conn)
    top = np.iinfo(dtype).max
    J0 = np.where(markers > 0, grad, top).astype(dtype)
    rec = oracle.reconstruct(J0, grad, conn, "erode")
    np.testing.assert_array_equal(lev, rec.astype(np.int32))
    assert set(np.unique(lab)) <= set(range(1, 13))
    check_labels(markers, grad, lab, lev, conn)


def test_hand_cases():
    grad = np.array([[0, 0, 9, 1, 1],
                     [0, 0, 9, 1, 1],
                     [0, 0, 9, 1, 1]], np.uint8)
    markers = np.zeros_like(grad, dtype=np.uint32)
    markers[1, 0] = 7
    markers[1, 4] = 3
    lab, lev = oracle.watershed(markers, grad, 4)
    np.testing.assert_array_equal(lab[:, :2], [[7, 7]] * 3)      # each basin keeps its marker's label
    np.testing.assert_array_equal(lab[:, 3:], [[3, 3]] * 3)
    np.testing.assert_array_equal(lev, [[0, 0, 9, 1, 1]] * 3)
    one = np.zeros_like(markers)
    one[0, 0] = 5
    lab, _ = oracle.watershed(one, grad, 8)
    assert np.all(lab == 5)
    lab, lev = oracle.watershed(np.zeros_like(markers), grad, 8)
    assert np.all(lab == 0) and np.all(lev == -1)
