"""GPU parity of the SKIZ (iwpp_skiz) against the oracle: distances, label pairs and zones
are unique, so every field is compared element by element (bit-exact)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1605_00930_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def iw():
    from paper_1605_00930_gb300 import iwpp
    return iwpp


def run(iw, markers, mask, conn):
    zone, dist, lpair = iw.skiz(torch.from_numpy(markers.astype(np.int32)).cuda(), torch.from_numpy(mask).cuda(),
                                conn, with_details=True)
    torch.cuda.synchronize()
    return zone.cpu().numpy().view(np.uint32), dist.cpu().numpy(), lpair.cpu().numpy().view(np.uint32)


def check(iw, markers, mask, conn):
    zone, dist, lpair = run(iw, markers, mask, conn)
    o = oracle.skiz(markers, mask, conn)
    np.testing.assert_array_equal(dist, o["dist"])
    np.testing.assert_array_equal(lpair, np.where(o["dist"] >= 0, (o["lmin"] << 16) | o["lmax"], 0))
    np.testing.assert_array_equal(zone, o["zone"])
    return o


@pytest.mark.parametrize("conn", [4, 8])
def test_random_small(iw, conn):
    rng = np.random.default_rng(1605)
    for i in range(12):
        H, W = int(rng.integers(1, 150)), int(rng.integers(1, 300))
        mask = (rng.random((H, W)) < rng.choice([0.45, 0.6, 0.8, 1.0])).astype(np.uint8)
        markers = np.zeros((H, W), np.uint32)
        nm = int(rng.integers(0, 12))
        markers[rng.integers(0, H, nm), rng.integers(0, W, nm)] = rng.integers(1, 6, nm)
        check(iw, markers, mask, conn)


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("shape", [(1000, 1300), (515, 2049)])
def test_porous_tissue(iw, conn, shape):
    markers, mask = synth.porous_skiz_case(*shape, nmarkers=300, nlabels=300, image_idx=shape[0] + conn)
    o = check(iw, markers, mask, conn)
    assert (o["dist"] > 40).any() and ((o["lmin"] != o["lmax"]) & (o["dist"] >= 0)).any()


def test_porous_4096(iw):
    markers, mask = synth.porous_skiz_case(4096, 4096, nmarkers=2000, nlabels=2000)
    check(iw, markers, mask, 8)


def test_free_space_ties(iw):
    # no obstacles, two labels on a checkerboard of seeds: many equidistant pixels
    markers = np.zeros((257, 333), np.uint32)
    markers[::37, ::41] = 1
    markers[18::37, 20::41] = 2
    for conn in (4, 8):
        check(iw, markers, np.ones_like(markers, np.uint8), conn)


def test_degenerate(iw):
    for H, W in [(1, 1), (1, 700), (700, 1), (17, 65)]:
        markers = np.zeros((H, W), np.uint32)
        mask = np.ones((H, W), np.uint8)
        check(iw, markers, mask, 8)                      # no markers: nothing reached
        markers.flat[0] = 3
        check(iw, markers, mask, 8)                      # one label
        markers.flat[-1] = 9
        check(iw, markers, np.zeros_like(mask), 4)       # markers only, empty domain
        check(iw, markers, mask, 4)


def test_bad_label_reported(iw):
    markers = np.zeros((40, 70), np.uint32)
    markers[3, 4] = 70000
    with pytest.raises(iw.IwppError):
        run(iw, markers, np.ones((40, 70), np.uint8), 8)
