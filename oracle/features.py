"""Per-block features of the learned work estimator — test infrastructure only.

Plain numpy (float64) definition of the 16 inputs of the schedule MLP, computed
for every 64 x 64 block of an image (the last row / column of blocks may be
partial). These inputs are not in the paper: they follow the learned-schedule
configuration of this project, with these readings (also listed in the design doc):

  values are taken in the dilation domain: for erosion both images are
  complemented, c(x) = MAXV - x, so that d = I - J >= 0 for either operator;
  d8 = d for u8 and d >> 8 for u16;
  f[0..14] are taken over every ROW_STEP-th row of the block (its rows 0, 4, 8, ...;
           the sampled pixels), which makes them a quarter as costly to compute;
  f[0..7]  8-bin histogram of d8 as fractions of the block: bin 0 holds d8 == 0,
           bin k (1..6) holds 2^(k-1) <= d8 < 2^k, bin 7 holds d8 >= 64;
  f[8]     seed fraction: pixels with J == I and J > 0 (the marker touches the mask);
  f[9]     edge density: pixels where |I(p) - I(p + x)| + |I(p) - I(p + y)| exceeds
           16 * MAXV / 255, with a neighbour outside the block contributing 0 (p + y is
           the next row of the block, sampled or not);
  f[10..14] mean(I), std(I), mean(J), std(J), mean(d), each divided by MAXV
           (population standard deviation);
  f[15]    log2(pixels in the block, every row) / 12.

Parity status: pinned by a pixel-by-pixel brute force (tests/test_oracle_learned.py)
and hand-worked blocks.
"""
from __future__ import annotations

import numpy as np

BLOCK = 64
NFEAT = 16
ROW_STEP = 4


def _maxv(dtype) -> int:
    return int(np.iinfo(np.dtype(dtype)).max)


def block_grid(H: int, W: int, block: int = BLOCK):
    return (H + block - 1) // block, (W + block - 1) // block


def block_features(marker: np.ndarray, mask: np.ndarray, op: str, by: int, bx: int,
                   block: int = BLOCK) -> np.ndarray:
    M = _maxv(mask.dtype)
    y0, x0 = by * block, bx * block
    I = mask[y0:y0 + block, x0:x0 + block].astype(np.int64)
    J = marker[y0:y0 + block, x0:x0 + block].astype(np.int64)
    if op == "erode":
        I, J = M - I, M - J
    npix = I.size
    gx = np.zeros_like(I)
    gy = np.zeros_like(I)
    gx[:, :-1] = np.abs(I[:, 1:] - I[:, :-1])
    gy[:-1, :] = np.abs(I[1:, :] - I[:-1, :])
    # the sampled rows
    I, J, gx, gy = I[::ROW_STEP], J[::ROW_STEP], gx[::ROW_STEP], gy[::ROW_STEP]
    n = I.size
    d = np.maximum(I - J, 0)
    d8 = d if M == 255 else (d >> 8)
    bins = np.where(d8 == 0, 0, np.minimum(7, np.floor(np.log2(np.maximum(d8, 1))).astype(np.int64) + 1))
    f = np.zeros(NFEAT, dtype=np.float64)
    f[:8] = np.bincount(bins.ravel(), minlength=8)[:8] / n
    f[8] = np.mean((J == I) & (J > 0))
    f[9] = np.mean((gx + gy) > 16 * (M // 255))
    f[10] = I.mean() / M
    f[11] = I.std() / M
    f[12] = J.mean() / M
    f[13] = J.std() / M
    f[14] = d.mean() / M
    f[15] = np.log2(npix) / 12.0
    return f


def image_features(marker, mask, op, block: int = BLOCK) -> np.ndarray:
    """Features of every block of one image, blocks in row-major order."""
    nby, nbx = block_grid(*mask.shape, block)
    return np.stack([block_features(marker, mask, op, by, bx, block)
                     for by in range(nby) for bx in range(nbx)])


def batch_features(cases, block: int = BLOCK) -> np.ndarray:
    """Features of a batch: images in order, each image's blocks row-major."""
    return np.concatenate([image_features(c.marker, c.mask, c.op, block) for c in cases])
