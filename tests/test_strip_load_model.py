"""Host model of the strip load of the register and cooperative solvers (RegTile::load_fused in
csrc/iwpp_regtile.cuh): every strip row is read as aligned two-pixel words, for odd widths
shifted by one on rows that start on an odd element and recombined across lanes, with the
pixels a lane cannot get from its neighbours taken from the halo-column lanes. The model
replays the warp's address arithmetic on the CPU for every width 2..140 and a few large
ones, every tile position and several heights, and checks that each load stays inside the
image, is aligned to its two-pixel size, and that every pixel inside the image ends up in
the right half of the right lane."""
import numpy as np
import pytest

TH, TW = 16, 64


def strip_values(H, W, y0, x0):
    """(rows TH + 2: halo above, strip, halo below) x (32 lanes) x 2 pixel indices, -1 for
    pixels the model does not define (outside the image); asserts bounds and alignment."""
    N = H * W
    odd = W & 1
    lanes = np.arange(32)
    gx = x0 + 2 * lanes
    xe0 = np.minimum(gx, W - 3) if odd else np.minimum(gx, W - 2)
    xe1 = np.minimum(gx, W - 1) - 1
    out = np.full((TH + 2, 32, 2), -1, np.int64)
    for hl in range(TH + 2):
        y = y0 + hl - 1
        yc = min(max(y, 0), H - 1)
        p = bool(odd and (yc & 1))
        ea = yc * W + (xe1 if p else xe0)
        assert np.all(ea >= 0) and np.all(ea + 1 < N), "pair outside the image"
        assert np.all(ea % 2 == 0), "pair not aligned"
        lo, hi = ea, ea + 1                      # element indices of the loaded pair
        sv = yc * W + min(x0 + 63, W - 1)        # the halo lane's extra pixel of this row
        assert 0 <= sv < N
        if p:
            v_lo = hi
            v_hi = np.append(lo[1:], sv)         # next lane's first pixel; lane 31: the halo lane's
        else:
            v_lo, v_hi = lo.copy(), hi.copy()
            if odd:
                v_lo = np.where(gx == W - 1, sv, v_lo)
        if 0 <= y < H:
            out[hl, :, 0] = np.where(gx < W, v_lo, -1)
            out[hl, :, 1] = np.where(gx + 1 < W, v_hi, -1)
    return out


def expected(H, W, y0, x0):
    lanes = np.arange(32)
    out = np.full((TH + 2, 32, 2), -1, np.int64)
    for hl in range(TH + 2):
        y = y0 + hl - 1
        if 0 <= y < H:
            for k in (0, 1):
                x = x0 + 2 * lanes + k
                out[hl, :, k] = np.where(x < W, y * W + x, -1)
    return out


WIDTHS = list(range(2, 141)) + [255, 257, 1023, 4097]


@pytest.mark.parametrize("W", WIDTHS)
def test_strip_load_addresses_and_pixels(W):
    for H in (1, 2, 3, 17, 64, 65, 130):
        for x0 in range(0, W, 64):
            for y0 in range(0, H, 16):
                got = strip_values(H, W, y0, x0)
                np.testing.assert_array_equal(got, expected(H, W, y0, x0), err_msg=f"H {H} W {W} y0 {y0} x0 {x0}")
