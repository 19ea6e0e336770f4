"""Shared checks of a distance-transform result (sites and squared distances)."""
import numpy as np

NB = {4: [(-1, 0), (0, -1), (0, 1), (1, 0)],
      8: [(-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 1), (1, -1), (1, 0), (1, 1)]}


def exact_d2(fg):
    """Brute force: squared distance from every pixel to the nearest background pixel
    (-1 everywhere when there is no background)."""
    ys, xs = np.nonzero(fg == 0)
    H, W = fg.shape
    if len(ys) == 0:
        return np.full((H, W), -1, np.int64)
    yy, xx = np.mgrid[0:H, 0:W]
    best = np.full((H, W), np.iinfo(np.int64).max, np.int64)
    for k in range(0, len(ys), 256):   # chunks keep the memory small
        d = (yy[..., None] - ys[k:k + 256]) ** 2 + (xx[..., None] - xs[k:k + 256]) ** 2
        best = np.minimum(best, d.min(axis=-1))
    return best


def check_valid(fg, sy, sx, d2, conn):
    """sy, sx: site coordinates (-1 = none); d2: squared distances (-1 = none).
    Background pixels are their own sites, every site is a background pixel, d2 is the
    distance to the site, and no neighbour offers a strictly closer site."""
    H, W = fg.shape
    bg = fg == 0
    yy, xx = np.mgrid[0:H, 0:W]
    assert np.all(sy[bg] == yy[bg]) and np.all(sx[bg] == xx[bg]) and np.all(d2[bg] == 0)
    if not bg.any():
        assert np.all(sy == -1) and np.all(sx == -1) and np.all(d2 == -1)
        return
    assert np.all(sy >= 0) and np.all(sx >= 0)
    assert np.all(fg[sy, sx] == 0)
    np.testing.assert_array_equal(d2, (yy - sy) ** 2 + (xx - sx) ** 2)
    for dy, dx in NB[conn]:
        ny, nx = yy + dy, xx + dx
        ok = (ny >= 0) & (ny < H) & (nx >= 0) & (nx < W)
        cy = sy[np.clip(ny, 0, H - 1), np.clip(nx, 0, W - 1)]
        cx = sx[np.clip(ny, 0, H - 1), np.clip(nx, 0, W - 1)]
        cand = (yy - cy) ** 2 + (xx - cx) ** 2
        assert not np.any(ok & (cand < d2)), "a neighbour offers a strictly closer site"
