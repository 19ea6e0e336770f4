"""GPU reconstruction-based operators against their plain definitions (bit-exact)."""
import numpy as np
import pytest

from oracle import ops
from paper_1605_00930_gb300 import synth

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


@pytest.mark.parametrize("shape", [(1, 1), (37, 200), (300, 517), (1024, 777)])
@pytest.mark.parametrize("is16", [False, True])
@pytest.mark.parametrize("conn", [4, 8])
def test_operators(iw, shape, is16, conn):
    f8 = synth.blob_field_u8(*shape, max(1, shape[0] * shape[1] // 4000), synth.rng_for(92, shape[0] + is16))
    f = synth.to_u16(f8) if is16 else f8
    g = torch.from_numpy(f).cuda()
    for h in (1, 30 * (257 if is16 else 1)):
        np.testing.assert_array_equal(iw.hmaxima(g, h, conn).cpu().numpy(), ops.hmaxima(f, h, conn))
        np.testing.assert_array_equal(iw.hdome(g, h, conn).cpu().numpy(), ops.hdome(f, h, conn))
    np.testing.assert_array_equal(iw.regional_maxima(g, conn).cpu().numpy(), ops.regional_maxima(f, conn))


def test_regional_maxima_plateaus(iw):
    rng = np.random.default_rng(93)
    for trial in range(20):
        f = rng.integers(0, 5, size=(int(rng.integers(1, 70)), int(rng.integers(1, 90)))).astype(np.uint8)
        got = iw.regional_maxima(torch.from_numpy(f).cuda(), 8).cpu().numpy()
        np.testing.assert_array_equal(got, ops.regional_maxima_flood(f, 8))
