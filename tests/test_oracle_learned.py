"""Pins for the learned-schedule oracles: per-block features against a pixel-by-pixel
brute force written independently (pure Python, integer bit lengths) and hand-worked
blocks; the MLP's backpropagation against central finite differences, its forward pass
against hand-set weights, and Adam against the update written out for one scalar."""
import math

import numpy as np
import pytest

from oracle import features, mlp
from paper_1605_00930_gb300 import synth


def _brute_block(marker, mask, op, by, bx, B=64, step=4):
    """Features of one block, pixel by pixel: every `step`-th row of the block (rows 0, step,
    ...) is summed; the edge test looks at the next row of the block, sampled or not; the
    last feature counts every pixel of the block."""
    M = int(np.iinfo(mask.dtype).max)
    H, W = mask.shape
    ys = range(by * B, min(H, by * B + B))
    xs = range(bx * B, min(W, bx * B + B))
    n = len(ys[::step]) * len(xs)
    hist = [0] * 8
    seeds = edges = 0
    sI = sI2 = sJ = sJ2 = sD = 0
    for y in ys[::step]:
        for x in xs:
            i, j = int(mask[y, x]), int(marker[y, x])
            if op == "erode":
                i, j = M - i, M - j
            d = max(i - j, 0)
            d8 = d if M == 255 else d >> 8
            hist[min(7, d8.bit_length())] += 1
            seeds += (i == j and j > 0)
            def I_at(yy, xx):
                v = int(mask[yy, xx])
                return M - v if op == "erode" else v
            gx = abs(I_at(y, x + 1) - i) if x + 1 in xs else 0
            gy = abs(I_at(y + 1, x) - i) if y + 1 in ys else 0
            edges += (gx + gy > 16 * (M // 255))
            sI += i; sI2 += i * i; sJ += j; sJ2 += j * j; sD += d
    mI, mJ = sI / n, sJ / n
    return np.array([h / n for h in hist] + [seeds / n, edges / n, mI / M,
                    math.sqrt(max(0.0, sI2 / n - mI * mI)) / M, mJ / M,
                    math.sqrt(max(0.0, sJ2 / n - mJ * mJ)) / M, sD / n / M,
                    math.log2(len(ys) * len(xs)) / 12])


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("op", ["dilate", "erode"])
def test_features_match_brute_force(dtype, op):
    field = synth.blob_field_u8(70, 130, 4, synth.rng_for(77))
    mask = field if dtype == np.uint8 else synth.to_u16(field)
    rng = np.random.default_rng(5)
    if op == "dilate":
        marker = synth.hdome_marker(mask, int(rng.integers(1, 40)) * (1 if dtype == np.uint8 else 257))
        marker[rng.random(mask.shape) < 0.1] = 0
    else:
        marker = synth.fillholes_marker(mask)
    F = features.image_features(marker, mask, op)
    nby, nbx = features.block_grid(*mask.shape)
    assert F.shape == (nby * nbx, 16)
    for by in range(nby):
        for bx in range(nbx):
            np.testing.assert_allclose(F[by * nbx + bx], _brute_block(marker, mask, op, by, bx),
                                       rtol=0, atol=1e-12)


def test_features_hand_blocks():
    # constant block, marker == mask == 7: all of d in bin 0, every pixel a seed, no edges
    m = np.full((64, 64), 7, np.uint8)
    f = features.block_features(m, m, "dilate", 0, 0)
    assert f[0] == 1.0 and f[1:8].sum() == 0 and f[8] == 1.0 and f[9] == 0.0
    assert f[10] == 7 / 255 and f[11] == 0 and f[12] == 7 / 255 and f[14] == 0 and f[15] == 1.0
    # marker 0 under mask 5: d = 5 -> bin 3 (4 <= 5 < 8); no seeds (J == 0)
    f = features.block_features(np.zeros((2, 2), np.uint8), np.full((2, 2), 5, np.uint8), "dilate", 0, 0)
    assert f[3] == 1.0 and f[8] == 0.0 and f[14] == 5 / 255 and f[15] == 2 / 12
    # a vertical step edge of height 20 > 16 between columns 0 and 1 of a 1 x 2 block
    f = features.block_features(np.zeros((1, 2), np.uint8), np.array([[0, 20]], np.uint8), "dilate", 0, 0)
    assert f[9] == 0.5
    # rows 0 and 4 of a 5 x 2 block are sampled: mask rows 0, 200, 0, 0, 100 over marker 0 give
    # d = 0 (bin 0) and 100 (bin 7, >= 64) on the sampled rows; row 0's pixels see the 200 below
    # them (edges), row 4 has no row below in the block; the unsampled 200 adds nothing else
    mask = np.array([[0, 0], [200, 200], [0, 0], [0, 0], [100, 100]], np.uint8)
    f = features.block_features(np.zeros_like(mask), mask, "dilate", 0, 0)
    assert f[0] == 0.5 and f[7] == 0.5 and f[1:7].sum() == 0
    assert f[9] == 0.5 and f[10] == 50 / 255 and f[15] == math.log2(10) / 12


def test_mlp_forward_hand_weights():
    d = {name: np.zeros(shp) for name, shp in mlp.SHAPES}
    d["W1"][0, 0] = 2.0        # h1[0] = relu(2 x0)
    d["W1"][1, 1] = -1.0       # h1[1] = relu(-x1)
    d["W2"][0, 0] = 1.0
    d["W2"][1, 1] = 3.0
    d["W3"][0, 0] = 1.0
    d["W3"][1, 1] = 1.0
    d["b3"][:] = [0.5, -0.5]
    p = mlp.pack(d)
    X = np.zeros((2, 16))
    X[0, 0], X[0, 1] = 1.5, -2.0   # h1 = (3, 2) -> h2 = (3, 6) -> y = (3.5, 5.5)
    X[1, 0], X[1, 1] = -1.0, 4.0   # h1 = (0, 0) -> y = b3
    np.testing.assert_allclose(mlp.forward(p, X), [[3.5, 5.5], [0.5, -0.5]])


def test_mlp_backprop_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = mlp.init_params(3) + rng.normal(0, 0.01, mlp.NPARAM)
    X = rng.random((7, 16))
    T = rng.normal(size=(7, 2))
    g = mlp.grad(p, X, T, (1.0, 0.25))
    idx = rng.choice(mlp.NPARAM, 200, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        e[i] = h
        fd = (mlp.loss(p + e, X, T, (1.0, 0.25)) - mlp.loss(p - e, X, T, (1.0, 0.25))) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_adam_scalar_written_out():
    p, g = np.array([1.0]), np.array([0.5])
    m, v = np.zeros(1), np.zeros(1)
    p1, m1, v1 = mlp.adam_step(p, g, m, v, 1, lr=0.1)
    # t = 1: m = 0.05, v = 0.00025, mhat = 0.5, vhat = 0.25 -> step = 0.1 * 0.5 / (0.5 + 1e-8)
    assert m1[0] == pytest.approx(0.05) and v1[0] == pytest.approx(0.00025)
    assert p1[0] == pytest.approx(1.0 - 0.1 * 0.5 / (0.5 + 1e-8), abs=1e-15)
