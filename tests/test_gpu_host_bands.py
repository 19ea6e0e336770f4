"""Reconstruction of images in host memory, band by band (iwpp_reconstruct_host): every
band height gives the oracle's result bit for bit, including band heights of one row,
ragged last bands, a maze whose propagation crosses band borders back and forth, u16,
fill-holes, and a precondition violation reported from a band."""
import numpy as np
import pytest
import torch

from paper_1605_00930_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def iw():
    from paper_1605_00930_gb300 import iwpp
    return iwpp


def run_host(iw, marker, mask, conn, op, band_rows, expect=0):
    m = torch.from_numpy(np.ascontiguousarray(marker).copy()).pin_memory()
    I = torch.from_numpy(np.ascontiguousarray(mask)).pin_memory()
    R = iw.HostReconstructor(marker.shape[0], marker.shape[1], m.dtype, band_rows)
    rc = R(m, I, conn, op)
    torch.cuda.synchronize()
    assert rc == expect, iw.STATUS.get(rc)
    return m.numpy(), R.band_visits


@pytest.mark.parametrize("band_rows", [1, 7, 64, 100, 5000])
def test_tissue_bands(iw, oracle_lib, band_rows):
    c = synth.tissue_case(517, 701, nblobs=40)
    for conn in (4, 8):
        got, visits = run_host(iw, c.marker, c.mask, conn, "dilate", band_rows)
        np.testing.assert_array_equal(got, oracle_lib.reconstruct(c.marker, c.mask, conn, "dilate"))
        assert visits >= -(-517 // band_rows)   # every band at least once


@pytest.mark.parametrize("band_rows", [3, 50])
def test_u16_fill_holes_and_seeds(iw, oracle_lib, band_rows):
    field = synth.blob_field_u8(300, 451, 20, synth.rng_for(93))
    mask16 = synth.to_u16(field)
    mk = synth.fillholes_marker(mask16)
    got, _ = run_host(iw, mk, mask16, 8, "erode", band_rows)
    np.testing.assert_array_equal(got, oracle_lib.reconstruct(mk, mask16, 8, "erode"))
    s = synth.sparse_seed_case(1024, 1536, nblobs=60, nseeds=8)
    got, _ = run_host(iw, s.marker, s.mask, 8, "dilate", band_rows * 7)
    np.testing.assert_array_equal(got, oracle_lib.reconstruct(s.marker, s.mask, 8, "dilate"))


def test_maze_crosses_band_borders(iw, oracle_lib):
    """Horizontal walls every 10 rows with one gap, alternating left and right: the only
    path from the seed at the bottom climbs through every band border, so bands are
    revisited as the propagation moves back up."""
    H, W = 200, 120
    mask = np.full((H, W), 200, np.uint8)
    for k, y in enumerate(range(9, H - 1, 10)):
        mask[y, :] = 0
        if k % 2:
            mask[y, :3] = 150
        else:
            mask[y, -3:] = 150
    marker = np.zeros_like(mask)
    marker[H - 1, W // 2] = 200
    exp = oracle_lib.reconstruct(marker, mask, 4, "dilate")
    assert exp[0, 0] == 150
    for band_rows in (4, 15, 33):
        got, visits = run_host(iw, marker, mask, 4, "dilate", band_rows)
        np.testing.assert_array_equal(got, exp)
        assert visits > -(-H // band_rows)


def test_serpentine_crosses_borders_both_ways(iw, oracle_lib):
    """Vertical walls every 8 columns with one gap, alternating bottom and top: the only path
    from the seed runs down one corridor and up the next, crossing every band border in both
    directions once per corridor. Bands of 16, 48 and 100 rows are reconstructed with 1, 3
    and 6 rows of each neighbour (the overlap) and must still give the oracle's result."""
    H, W = 230, 97
    mask = np.full((H, W), 180, np.uint8)
    for k, x in enumerate(range(7, W - 1, 8)):
        mask[:, x] = 0
        if k % 2:
            mask[:2, x] = 120
        else:
            mask[-2:, x] = 120
    marker = np.zeros_like(mask)
    marker[0, 0] = 180
    exp = oracle_lib.reconstruct(marker, mask, 8, "dilate")
    assert exp[H // 2, W - 1] == 120   # the last corridor is reached
    for band_rows in (16, 48, 100):
        got, visits = run_host(iw, marker, mask, 8, "dilate", band_rows)
        np.testing.assert_array_equal(got, exp)
        assert visits > -(-H // band_rows)


def test_random_ragged(iw, oracle_lib):
    rng = np.random.default_rng(1605)
    for H, W, b in [(1, 1, 1), (1, 700, 3), (700, 1, 9), (65, 130, 16), (129, 65, 64), (257, 513, 31)]:
        for op in ("dilate", "erode"):
            mask = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
            if op == "dilate":
                marker = (mask.astype(np.int64) * (rng.random((H, W)) < 0.05)).astype(np.uint8)
            else:
                marker = synth.fillholes_marker(mask)
            got, _ = run_host(iw, marker, mask, 8, op, b)
            np.testing.assert_array_equal(got, oracle_lib.reconstruct(marker, mask, 8, op))


def test_precondition_reported(iw):
    mask = np.full((70, 90), 10, np.uint8)
    marker = np.zeros_like(mask)
    marker[63, 44] = 11
    run_host(iw, marker, mask, 8, "dilate", 16, expect=2)
