"""Shared checks of a watershed-by-flooding result (labels and levels)."""
import numpy as np

import oracle

NB = {4: [(-1, 0), (0, -1), (0, 1), (1, 0)],
      8: [(-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 1), (1, -1), (1, 0), (1, 1)]}


def check_labels(markers, grad, label, level, conn, max_labels_checked=64):
    """Markers keep their label and the gradient as level; no neighbour offers a smaller
    (level, label) pair (the local fixed point); and every pixel's label belongs to
    markers that reach it at exactly its level (the minimax level from that label's
    markers alone, a reconstruction by erosion, equals the pixel's level)."""
    H, W = grad.shape
    g = grad.astype(np.int64)
    mk = markers > 0
    np.testing.assert_array_equal(label[mk], markers[mk])
    np.testing.assert_array_equal(level[mk], g[mk])
    if not mk.any():
        assert np.all(label == 0) and np.all(level == -1)
        return
    lab, lev = label.astype(np.int64), level.astype(np.int64)
    assert np.all(lab > 0) and np.all(lev >= 0)
    yy, xx = np.mgrid[0:H, 0:W]
    for dy, dx in NB[conn]:
        ny, nx = np.clip(yy + dy, 0, H - 1), np.clip(xx + dx, 0, W - 1)
        ok = (yy + dy >= 0) & (yy + dy < H) & (xx + dx >= 0) & (xx + dx < W)
        cl = np.maximum(lev[ny, nx], g)
        cb = lab[ny, nx]
        better = ok & ~mk & ((cl < lev) | ((cl == lev) & (cb < lab)))
        assert not better.any(), "a neighbour offers a smaller (level, label) pair"
    top = np.iinfo(grad.dtype).max
    for L in np.unique(lab)[:max_labels_checked]:
        J0 = np.where(markers == L, grad, top).astype(grad.dtype)
        levL = oracle.reconstruct(J0, grad, conn, "erode").astype(np.int64)
        sel = lab == L
        np.testing.assert_array_equal(levL[sel], lev[sel], err_msg=f"label {L} does not reach its pixels there")
