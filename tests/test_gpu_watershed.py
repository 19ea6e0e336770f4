"""GPU watershed by flooding against the oracle: levels bit-exact (they are unique);
labels checked for validity (markers keep theirs, no neighbour offers a smaller pair,
each label's markers reach its pixels at exactly their level)."""
import numpy as np
import pytest

import oracle
from paper_1605_00930_gb300 import synth
from tests._wshed_checks import check_labels

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


def run(iw, markers, grad, conn):
    lab, lev = iw.watershed(torch.from_numpy(markers.astype(np.int32)).cuda(), torch.from_numpy(grad).cuda(), conn,
                            with_levels=True)
    return lab.cpu().numpy().astype(np.uint32), lev.cpu().numpy()


@pytest.mark.parametrize("shape", [(1, 1), (1, 120), (90, 1), (16, 64), (37, 201), (300, 517)])
@pytest.mark.parametrize("is16", [False, True])
@pytest.mark.parametrize("conn", [4, 8])
def test_flooding(iw, shape, is16, conn):
    rng = np.random.default_rng([110, shape[0], shape[1], is16, conn])
    f = synth.blob_field_u8(*shape, max(1, shape[0] * shape[1] // 3000), rng)
    grad = synth.to_u16(f) if is16 else f
    for nm in (0, 1, 5, 40):
        markers = np.zeros(shape, np.uint32)
        if nm:
            ys, xs = rng.integers(0, shape[0], nm), rng.integers(0, shape[1], nm)
            markers[ys, xs] = rng.integers(1, 30, nm)
        lab, lev = run(iw, markers, grad, conn)
        _, olev = oracle.watershed(markers, grad, conn)
        np.testing.assert_array_equal(lev, olev)
        check_labels(markers, grad, lab, lev, conn)


def test_plateaus_and_ridges(iw):
    rng = np.random.default_rng(111)
    for trial in range(10):
        H, W = int(rng.integers(20, 90)), int(rng.integers(20, 200))
        grad = rng.integers(0, 4, size=(H, W)).astype(np.uint8)   # many equal levels
        markers = np.zeros((H, W), np.uint32)
        markers[rng.integers(0, H, 8), rng.integers(0, W, 8)] = rng.integers(1, 6, 8)
        lab, lev = run(iw, markers, grad, 8)
        _, olev = oracle.watershed(markers, grad, 8)
        np.testing.assert_array_equal(lev, olev)
        check_labels(markers, grad, lab, lev, 8)


def test_bad_label_reported(iw):
    markers = np.zeros((40, 70), np.uint32)
    markers[3, 4] = 70000
    grad = np.zeros((40, 70), np.uint8)
    with pytest.raises(iw.IwppError):
        run(iw, markers, grad, 8)
