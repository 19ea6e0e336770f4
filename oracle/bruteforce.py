"""Brute-force reconstruction — test infrastructure only.

Algorithm 1 of Sec. 2.1.2 (the definition of reconstruction, Eq. "recon"):
repeat J <- delta_G(J_temp) ^ I, with every read taken from a copy J_temp of the
previous iterate (Jacobi order), until an iteration changes nothing. The dual,
reconstruction by erosion, repeats J <- eps_G(J_temp) v I.

The line of Algorithm 1 that forms the neighbourhood maximum is garbled in the
text ("max{J_temp(p), N_G(p)}"); it is read here as the maximum of J_temp over p
and its G-neighbours, which is how Sec. 3.1 writes the same update. Neighbours
outside the image do not exist: the shifted copies are padded with a value that
can never win the max (dilation) or the min (erosion).

This is a deliberately slow, obviously correct restatement for tiny images
(a few hundred pixels). It shares nothing with the C oracle or the CUDA path.
"""
from __future__ import annotations

import numpy as np

_OFFS4 = [(-1, 0), (0, -1), (0, 1), (1, 0)]
_OFFS8 = [(-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 1), (1, -1), (1, 0), (1, 1)]


def _neigh_extreme(J: np.ndarray, conn: int, op: str) -> np.ndarray:
    """max (dilate) or min (erode) of J over p and its in-domain G-neighbours."""
    H, W = J.shape
    big = np.int64(1 << 40)
    pad_val = -big if op == "dilate" else big
    P = np.full((H + 2, W + 2), pad_val, dtype=np.int64)
    P[1:-1, 1:-1] = J
    out = J.astype(np.int64).copy()
    for dy, dx in (_OFFS8 if conn == 8 else _OFFS4):
        sh = P[1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
        out = np.maximum(out, sh) if op == "dilate" else np.minimum(out, sh)
    return out


def reconstruct(marker: np.ndarray, mask: np.ndarray, conn: int = 8, op: str = "dilate",
                max_iters: int | None = None) -> np.ndarray:
    """Return the reconstruction of ``mask`` from ``marker`` by Algorithm 1."""
    if conn not in (4, 8):
        raise ValueError("conn must be 4 or 8")
    if op not in ("dilate", "erode"):
        raise ValueError("op must be 'dilate' or 'erode'")
    I = np.asarray(mask).astype(np.int64)
    J = np.asarray(marker).astype(np.int64).copy()
    if I.shape != J.shape or I.ndim != 2:
        raise ValueError("marker and mask must be equal-shape 2-D arrays")
    limit = max_iters if max_iters is not None else 4 * J.size + 8
    for _ in range(limit):
        J_temp = J.copy()
        ext = _neigh_extreme(J_temp, conn, op)
        J = np.minimum(ext, I) if op == "dilate" else np.maximum(ext, I)
        if np.array_equal(J, J_temp):
            return J.astype(np.asarray(marker).dtype)
    raise RuntimeError("brute force did not reach stability")
