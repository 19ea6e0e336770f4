"""GPU distance transform (Algorithm 8 on the tile engine) against what is unique:
the exact transform as a lower bound (equal with one or two background pixels), site
validity, distances, the propagation's fixed point; and against the oracle's accuracy on
tissue-like masks. Several fixed points are equally valid, so results are not compared
with the oracle bit by bit."""
import numpy as np
import pytest

import oracle
from paper_1605_00930_gb300 import synth
from tests._edt_checks import check_valid, exact_d2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def iw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_00930_gb300 import build
    build.build()
    from paper_1605_00930_gb300 import iwpp
    iwpp.lib()
    return iwpp


def gpu_edt(iw, fg, conn):
    H, W = fg.shape
    m = torch.from_numpy(np.ascontiguousarray(fg.astype(np.uint8))).cuda()
    site = torch.empty((H, W), dtype=torch.int32, device="cuda")
    d2 = torch.empty((H, W), dtype=torch.int32, device="cuda")
    T = iw.DistanceTransform(H, W)
    assert T(m, site, d2, conn) == 0
    assert T.status() == 0
    s = site.cpu().numpy().view(np.uint32).astype(np.int64)
    d = d2.cpu().numpy().view(np.uint32).astype(np.int64)
    none = s == 0xFFFFFFFF
    sy = np.where(none, -1, s >> 16)
    sx = np.where(none, -1, s & 0xFFFF)
    d = np.where(d == 0xFFFFFFFF, -1, d)
    return sy, sx, d


SHAPES = [(1, 1), (1, 90), (70, 1), (16, 64), (17, 65), (33, 130), (100, 257)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("conn", [4, 8])
def test_random_masks(iw, shape, conn):
    rng = np.random.default_rng([80, shape[0], shape[1], conn])
    for density in (0.3, 0.8, 0.97):
        fg = (rng.random(shape) < density).astype(np.uint8)
        sy, sx, d2 = gpu_edt(iw, fg, conn)
        check_valid(fg, sy, sx, d2, conn)
        ex = exact_d2(fg)
        assert np.all(d2 >= ex)


@pytest.mark.parametrize("conn", [4, 8])
def test_one_and_two_sites_exact(iw, conn):
    rng = np.random.default_rng([81, conn])
    for trial in range(12):
        H, W = int(rng.integers(20, 150)), int(rng.integers(20, 300))
        fg = np.ones((H, W), np.uint8)
        for _ in range(1 + trial % 2):
            fg[rng.integers(0, H), rng.integers(0, W)] = 0
        sy, sx, d2 = gpu_edt(iw, fg, conn)
        check_valid(fg, sy, sx, d2, conn)
        np.testing.assert_array_equal(d2, exact_d2(fg))


def test_degenerate(iw):
    for shape in [(1, 1), (5, 70), (40, 3)]:
        for conn in (4, 8):
            sy, sx, d2 = gpu_edt(iw, np.zeros(shape, np.uint8), conn)
            assert np.all(d2 == 0)
            sy, sx, d2 = gpu_edt(iw, np.ones(shape, np.uint8), conn)
            assert np.all(sy == -1) and np.all(d2 == -1)


@pytest.mark.parametrize("side", [600, 2048])
@pytest.mark.parametrize("conn", [4, 8])
def test_tissue_mask_accuracy(iw, side, conn):
    """Tissue-like mask: every property holds, and the propagation is as accurate as the
    oracle's (fraction of exact pixels, largest error)."""
    ndimage = pytest.importorskip("scipy.ndimage")
    f = synth.blob_field_u8(side, side + 37, max(4, side * side // 40000), synth.rng_for(82, side))
    fg = (f > 60).astype(np.uint8)
    sy, sx, d2 = gpu_edt(iw, fg, conn)
    check_valid(fg, sy, sx, d2, conn)
    ex = np.rint(ndimage.distance_transform_edt(fg) ** 2).astype(np.int64)
    assert np.all(d2 >= ex)
    _, od2 = oracle.edt(fg, conn)
    gpu_exact, ora_exact = np.mean(d2 == ex), np.mean(od2 == ex)
    assert gpu_exact > 0.99 and gpu_exact > ora_exact - 0.005
    assert np.max(np.sqrt(d2) - np.sqrt(ex)) < 1.5
