"""Pins of the CPU oracle's distance transform (Sec. 3.2, Algorithm 8: Voronoi sites
propagated as a wavefront), against what the mathematics fixes without it:

  * the exact Euclidean transform (brute force on tiny masks, scipy on larger ones) is a
    lower bound everywhere, and equality holds with one or two background sites (each
    site's discrete Voronoi cell is connected and contains the site);
  * background pixels are their own sites (distance 0); every site is a background pixel
    and the stored squared distance is the distance to it;
  * the result is a fixed point of the propagation step: no neighbour offers a strictly
    closer site;
  * degenerate masks: all background, no background.
"""
import numpy as np
import pytest

import oracle

NB = {4: [(-1, 0), (0, -1), (0, 1), (1, 0)],
      8: [(-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 1), (1, -1), (1, 0), (1, 1)]}


def exact_d2(fg):
    """Brute force: squared distance from every pixel to the nearest background pixel."""
    ys, xs = np.nonzero(fg == 0)
    H, W = fg.shape
    if len(ys) == 0:
        return np.full((H, W), -1, np.int64)
    yy, xx = np.mgrid[0:H, 0:W]
    d = (yy[..., None] - ys) ** 2 + (xx[..., None] - xs) ** 2
    return d.min(axis=-1).astype(np.int64)


def check_valid(fg, site, d2, conn):
    H, W = fg.shape
    bg = fg == 0
    assert np.all(site[bg] == np.flatnonzero(bg)) and np.all(d2[bg] == 0)
    has = site >= 0
    if bg.any():
        assert has.all()
        sy, sx = site // W, site % W
        assert np.all(fg[sy, sx] == 0)
        yy, xx = np.mgrid[0:H, 0:W]
        np.testing.assert_array_equal(d2, (yy - sy) ** 2 + (xx - sx) ** 2)
        # fixed point: no neighbour's site is strictly closer
        for dy, dx in NB[conn]:
            ny, nx = yy + dy, xx + dx
            ok = (ny >= 0) & (ny < H) & (nx >= 0) & (nx < W)
            s2 = site[np.clip(ny, 0, H - 1), np.clip(nx, 0, W - 1)]
            cand = (yy - s2 // W) ** 2 + (xx - s2 % W) ** 2
            assert not np.any(ok & (cand < d2))
    else:
        assert np.all(site == -1) and np.all(d2 == -1)


@pytest.mark.parametrize("conn", [4, 8])
def test_single_and_two_sites_are_exact(conn):
    rng = np.random.default_rng([70, conn])
    for trial in range(60):
        H, W = int(rng.integers(1, 23)), int(rng.integers(1, 23))
        fg = np.ones((H, W), np.uint8)
        k = 1 if trial % 2 == 0 else 2
        for _ in range(k):
            fg[rng.integers(0, H), rng.integers(0, W)] = 0
        site, d2 = oracle.edt(fg, conn)
        check_valid(fg, site, d2, conn)
        np.testing.assert_array_equal(d2, exact_d2(fg))


@pytest.mark.parametrize("conn", [4, 8])
def test_random_masks_bounded_below_by_exact(conn):
    rng = np.random.default_rng([71, conn])
    for trial in range(200):
        H, W = int(rng.integers(1, 14)), int(rng.integers(1, 14))
        fg = (rng.random((H, W)) < rng.uniform(0.2, 0.95)).astype(np.uint8)
        site, d2 = oracle.edt(fg, conn)
        check_valid(fg, site, d2, conn)
        ex = exact_d2(fg)
        assert np.all(d2 >= ex)


def test_blob_mask_against_scipy():
    ndimage = pytest.importorskip("scipy.ndimage")
    from paper_1605_00930_gb300 import synth
    f = synth.blob_field_u8(180, 230, 25, synth.rng_for(72))
    fg = (f > 60).astype(np.uint8)
    for conn in (4, 8):
        site, d2 = oracle.edt(fg, conn)
        check_valid(fg, site, d2, conn)
        ex = np.rint(ndimage.distance_transform_edt(fg) ** 2).astype(np.int64)
        assert np.all(d2 >= ex)
        # the propagation misses the exact site only rarely, and then by little
        assert np.mean(d2 == ex) > 0.99
        assert np.max(np.sqrt(d2) - np.sqrt(ex)) < 1.5


def test_degenerate_masks():
    for shape in [(1, 1), (1, 17), (9, 1), (5, 6)]:
        for conn in (4, 8):
            site, d2 = oracle.edt(np.zeros(shape, np.uint8), conn)
            assert np.all(d2 == 0) and np.all(site == np.arange(np.prod(shape)).reshape(shape))
            site, d2 = oracle.edt(np.ones(shape, np.uint8), conn)
            assert np.all(site == -1) and np.all(d2 == -1)


def test_mistakes_are_caught():
    """A transposed site decoding or a dropped neighbour would break the single-site pin."""
    fg = np.ones((6, 11), np.uint8)
    fg[1, 8] = 0
    site, d2 = oracle.edt(fg, 8)
    yy, xx = np.mgrid[0:6, 0:11]
    np.testing.assert_array_equal(d2, (yy - 1) ** 2 + (xx - 8) ** 2)
    assert not np.array_equal(d2, (yy - 8 % 6) ** 2 + (xx - 1) ** 2)
