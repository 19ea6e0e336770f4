"""Pins for the SKIZ oracle (oracle/skiz_oracle.c): the geodesic influence zones of labelled
markers inside a binary domain, and the skeleton where two or more labels are nearest.

What fixes the result without the oracle: (1) brute force — each label's own geodesic
distance map by Bellman-Ford relaxation in numpy, then the minimum and the labels that reach
it; (2) a library routine — with no obstacles the geodesic distance is the chessboard (conn 8)
or city-block (conn 4) distance, scipy's chamfer transform; (3) connected components — with a
single label the reached pixels are the domain components that hold a marker; (4) hand-worked
cases on lines and around a wall."""
import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle

BIG = np.int64(1) << 40


def _shifts(conn):
    if conn == 4:
        return [(-1, 0), (1, 0), (0, -1), (0, 1)]
    return [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dy, dx) != (0, 0)]


def _relax(seeds, domain, conn):
    """Geodesic distance from the pixels `seeds` inside `domain` by relaxation to a fixed point:
    d(p) = min(d(p), d(q) + 1) over neighbours q, restricted to domain pixels."""
    H, W = domain.shape
    d = np.where(seeds, 0, BIG).astype(np.int64)
    while True:
        pad = np.pad(d, 1, constant_values=BIG)
        best = d.copy()
        for dy, dx in _shifts(conn):
            best = np.minimum(best, pad[1 + dy:1 + dy + H, 1 + dx:1 + dx + W] + 1)
        best = np.where(domain, best, BIG)
        best = np.where(seeds, 0, best)
        if np.array_equal(best, d):
            return d
        d = best


def brute(markers, mask, conn):
    domain = (mask != 0) | (markers != 0)
    labels = sorted(set(np.unique(markers).tolist()) - {0})
    H, W = markers.shape
    if not labels:
        z = np.zeros((H, W), np.uint32)
        return {"dist": np.full((H, W), -1, np.int32), "lmin": z, "lmax": z.copy(), "zone": z.copy()}
    per = np.stack([_relax(markers == l, domain, conn) for l in labels])
    dmin = per.min(axis=0)
    reached = dmin < BIG
    lab = np.array(labels, np.int64)[:, None, None]
    at = per == dmin[None]
    lmin = np.where(at, lab, BIG).min(axis=0)
    lmax = np.where(at, lab, -1).max(axis=0)
    out = {"dist": np.where(reached, dmin, -1).astype(np.int32),
           "lmin": np.where(reached, lmin, 0).astype(np.uint32),
           "lmax": np.where(reached, lmax, 0).astype(np.uint32)}
    out["zone"] = np.where(reached & (out["lmin"] == out["lmax"]), out["lmin"], 0).astype(np.uint32)
    return out


def _case(rng, H, W, nlab, nmark, pfore):
    mask = (rng.random((H, W)) < pfore).astype(np.uint8)
    markers = np.zeros((H, W), np.uint32)
    ys, xs = rng.integers(0, H, nmark), rng.integers(0, W, nmark)
    markers[ys, xs] = rng.integers(1, nlab + 1, nmark)
    return markers, mask


@pytest.mark.parametrize("conn", [4, 8])
def test_bruteforce_random(conn):
    rng = np.random.default_rng(160500930)
    for i in range(400):
        H, W = int(rng.integers(1, 13)), int(rng.integers(1, 13))
        markers, mask = _case(rng, H, W, int(rng.integers(1, 5)), int(rng.integers(0, 6)),
                              float(rng.choice([0.5, 0.7, 0.9, 1.0])))
        got, exp = oracle.skiz(markers, mask, conn), brute(markers, mask, conn)
        for k in ("dist", "lmin", "lmax", "zone"):
            np.testing.assert_array_equal(got[k], exp[k], err_msg=f"case {i} field {k}")


@pytest.mark.parametrize("conn,metric", [(8, "chessboard"), (4, "taxicab")])
def test_free_space_distance_is_scipy_chamfer(conn, metric):
    rng = np.random.default_rng(7)
    markers = np.zeros((97, 131), np.uint32)
    markers[rng.integers(0, 97, 25), rng.integers(0, 131, 25)] = rng.integers(1, 9, 25)
    got = oracle.skiz(markers, np.ones_like(markers, np.uint8), conn)
    np.testing.assert_array_equal(got["dist"], ndi.distance_transform_cdt(markers == 0, metric=metric))


@pytest.mark.parametrize("conn", [4, 8])
def test_single_label_reaches_marked_components(conn):
    rng = np.random.default_rng(11)
    mask = (rng.random((120, 90)) < 0.55).astype(np.uint8)
    markers = np.zeros(mask.shape, np.uint32)
    markers[rng.integers(0, 120, 6), rng.integers(0, 90, 6)] = 3
    domain = (mask != 0) | (markers != 0)
    comp, _ = ndi.label(domain, structure=np.ones((3, 3)) if conn == 8 else None)
    marked = np.unique(comp[markers != 0])
    reached = np.isin(comp, marked) & domain
    got = oracle.skiz(markers, mask, conn)
    np.testing.assert_array_equal(got["dist"] >= 0, reached)
    np.testing.assert_array_equal(got["zone"], np.where(reached, 3, 0))


def test_hand_line():
    # 1 x 5 line, labels 1 and 2 at the ends: the middle pixel is equidistant (skeleton)
    markers = np.array([[1, 0, 0, 0, 2]], np.uint32)
    got = oracle.skiz(markers, np.ones_like(markers, np.uint8), 4)
    assert got["dist"].tolist() == [[0, 1, 2, 1, 0]]
    assert got["zone"].tolist() == [[1, 1, 0, 2, 2]]
    assert got["lmin"].tolist() == [[1, 1, 1, 2, 2]] and got["lmax"].tolist() == [[1, 1, 2, 2, 2]]
    # even length: no pixel is equidistant
    markers = np.array([[1, 0, 0, 0, 0, 2]], np.uint32)
    got = oracle.skiz(markers, np.ones_like(markers, np.uint8), 8)
    assert got["zone"].tolist() == [[1, 1, 1, 2, 2, 2]]


def test_hand_wall_geodesic():
    # a wall (mask 0) with a gap at the bottom: the geodesic path from label 1 goes around it
    #   row 0:  1 . X . .
    #   row 1:  . . X . .
    #   row 2:  . . . . 2
    mask = np.ones((3, 5), np.uint8)
    mask[0:2, 2] = 0
    markers = np.zeros((3, 5), np.uint32)
    markers[0, 0], markers[2, 4] = 1, 2
    got = oracle.skiz(markers, mask, 4)
    assert got["dist"].tolist() == [[0, 1, -1, 3, 2], [1, 2, -1, 2, 1], [2, 3, 2, 1, 0]]
    assert got["zone"].tolist() == [[1, 1, 0, 2, 2], [1, 1, 0, 2, 2], [1, 0, 2, 2, 2]]
    # (2, 1): 3 steps from either marker -> skeleton
    assert got["lmin"][2, 1] == 1 and got["lmax"][2, 1] == 2


def test_markers_are_domain_and_labels_checked():
    mask = np.zeros((1, 3), np.uint8)
    markers = np.array([[5, 0, 0]], np.uint32)
    got = oracle.skiz(markers, mask, 8)
    assert got["dist"].tolist() == [[0, -1, -1]] and got["zone"].tolist() == [[5, 0, 0]]
    with pytest.raises(ValueError):
        oracle.skiz(np.array([[65535]], np.uint32), np.ones((1, 1), np.uint8), 8)
