"""Reconstruction-based operators, plain definitions — TEST INFRASTRUCTURE ONLY.

  * h-maxima:  HMAX_h(f) = R_f(max(f - h, 0)), reconstruction by dilation (Sec. 2.1.2);
  * h-dome:    f - HMAX_h(f);
  * regional maxima, twice, independently: through reconstruction (f > R_f(f - 1)) and by
    flooding every plateau (a connected set of equal pixels) and checking that all its
    outside neighbours are strictly lower. The two agreeing pins both.
"""
from __future__ import annotations

from collections import deque

import numpy as np

from . import reconstruct

NB = {4: [(-1, 0), (0, -1), (0, 1), (1, 0)],
      8: [(-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 1), (1, -1), (1, 0), (1, 1)]}


def hmaxima(f: np.ndarray, h: int, conn: int = 8) -> np.ndarray:
    marker = np.maximum(f.astype(np.int64) - int(h), 0).astype(f.dtype)
    return reconstruct(marker, f, conn, "dilate")


def hdome(f: np.ndarray, h: int, conn: int = 8) -> np.ndarray:
    return (f.astype(np.int64) - hmaxima(f, h, conn).astype(np.int64)).astype(f.dtype)


def regional_maxima(f: np.ndarray, conn: int = 8) -> np.ndarray:
    """Through reconstruction: 1 where f > R_f(f - 1)."""
    return (f > hmaxima(f, 1, conn)).astype(np.uint8)


def regional_maxima_flood(f: np.ndarray, conn: int = 8) -> np.ndarray:
    """By definition: flood each plateau; it is a regional maximum if no outside neighbour
    is higher or equal. Pure Python, for small images."""
    H, W = f.shape
    seen = np.zeros((H, W), bool)
    out = np.zeros((H, W), np.uint8)
    for y0 in range(H):
        for x0 in range(W):
            if seen[y0, x0]:
                continue
            v = f[y0, x0]
            comp, q, is_max = [], deque([(y0, x0)]), True
            seen[y0, x0] = True
            while q:
                y, x = q.popleft()
                comp.append((y, x))
                for dy, dx in NB[conn]:
                    yy, xx = y + dy, x + dx
                    if not (0 <= yy < H and 0 <= xx < W):
                        continue
                    if f[yy, xx] == v:
                        if not seen[yy, xx]:
                            seen[yy, xx] = True
                            q.append((yy, xx))
                    elif f[yy, xx] > v:
                        is_max = False
            if is_max:
                for y, x in comp:
                    out[y, x] = 1
    return out
