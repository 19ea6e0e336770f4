"""Seeded synthetic inputs shaped like pathology tissue tiles.

This module builds marker/mask pairs only; it holds none of the reconstruction's
arithmetic, and both the CUDA path's tests and the CPU oracle's tests draw their
inputs from it. The paper's own inputs (brain-tumour tissue images of 4K^2-32K^2
pixels at 25-100 % tissue coverage, Sec. 5.2) are not available, so seeded
blob fields stand in for them:

  * noise-blur field: uniform{0..255} noise, 5x5 box mean with replicate edges,
    rounded as (sum + 12) // 25;
  * blob field: uniform{0..30} background; each blob has a centre uniform in the
    image, radius r ~ U[5, 40] px and peak ~ U{80..255}, with profile
    round(peak * exp(-d^2 / (2 (r/2)^2))) for d <= r and 0 beyond; the mask is
    the pixelwise maximum of background and blobs. 16-bit masks are the 8-bit
    field times 257 (0..65535);
  * markers: h-dome (marker = max(mask - h, 0)), sparse seeds (marker = 0 except
    seed pixels equal to the mask), or the fill-holes marker (mask on the four
    border lines, the maximum value elsewhere).

Every generator takes a numpy Generator; ``rng_for`` derives it from a fixed root
seed, a workload id and an image index, so every input is reproducible.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_ROOT = 160500930


def rng_for(workload_id: int, image_idx: int = 0) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([SEED_ROOT, workload_id, image_idx]))


def maxval(dtype) -> int:
    return int(np.iinfo(np.dtype(dtype)).max)


@dataclass
class Case:
    """One reconstruction problem: marker is overwritten by the result."""
    marker: np.ndarray
    mask: np.ndarray
    conn: int
    op: str  # "dilate" or "erode"

    @property
    def pixels(self) -> int:
        return int(self.mask.size)


def noise_blur_u8(H: int, W: int, rng: np.random.Generator) -> np.ndarray:
    noise = rng.integers(0, 256, size=(H, W), dtype=np.int32)
    P = np.pad(noise, 2, mode="edge").astype(np.int64)
    S = np.zeros((H + 5, W + 5), dtype=np.int64)
    S[1:, 1:] = P.cumsum(0).cumsum(1)
    box = S[5:, 5:] - S[:-5, 5:] - S[5:, :-5] + S[:-5, :-5]
    return ((box + 12) // 25).astype(np.uint8)


def blob_field_u8(H: int, W: int, nblobs: int, rng: np.random.Generator) -> np.ndarray:
    mask = rng.integers(0, 31, size=(H, W), dtype=np.uint8)
    cy = rng.uniform(0.0, H, size=nblobs)
    cx = rng.uniform(0.0, W, size=nblobs)
    rad = rng.uniform(5.0, 40.0, size=nblobs)
    peak = rng.integers(80, 256, size=nblobs)
    for k in range(nblobs):
        r = rad[k]
        y0, y1 = max(0, int(math.floor(cy[k] - r))), min(H, int(math.ceil(cy[k] + r)) + 1)
        x0, x1 = max(0, int(math.floor(cx[k] - r))), min(W, int(math.ceil(cx[k] + r)) + 1)
        if y0 >= y1 or x0 >= x1:
            continue
        yy = np.arange(y0, y1, dtype=np.float64)[:, None] + 0.5 - cy[k]
        xx = np.arange(x0, x1, dtype=np.float64)[None, :] + 0.5 - cx[k]
        d2 = yy * yy + xx * xx
        sigma2 = (r / 2.0) ** 2
        prof = np.rint(peak[k] * np.exp(-d2 / (2.0 * sigma2)))
        prof[d2 > r * r] = 0
        win = mask[y0:y1, x0:x1]
        np.maximum(win, prof.astype(np.uint8), out=win)
    return mask


def to_u16(field_u8: np.ndarray) -> np.ndarray:
    return field_u8.astype(np.uint16) * np.uint16(257)


def hdome_marker(mask: np.ndarray, h: int) -> np.ndarray:
    return np.maximum(mask.astype(np.int64) - h, 0).astype(mask.dtype)


def seeds_marker(mask: np.ndarray, nseeds: int, rng: np.random.Generator) -> np.ndarray:
    marker = np.zeros_like(mask)
    flat = rng.choice(mask.size, size=min(nseeds, mask.size), replace=False)
    marker.reshape(-1)[flat] = mask.reshape(-1)[flat]
    return marker


def fillholes_marker(mask: np.ndarray) -> np.ndarray:
    marker = np.full_like(mask, maxval(mask.dtype))
    marker[0, :] = mask[0, :]
    marker[-1, :] = mask[-1, :]
    marker[:, 0] = mask[:, 0]
    marker[:, -1] = mask[:, -1]
    return marker


def blob_count(H: int, W: int, ref_blobs: int = 2000, ref_side: int = 4096) -> int:
    """Blob count that keeps the 4096^2 / 2000-blob density at another size."""
    return max(1, int(round(ref_blobs * H * W / float(ref_side * ref_side))))


# ---- the five workloads -------------------------------------------------------

def noise_blur_case(H: int = 512, W: int = 512, h: int = 40, image_idx: int = 0) -> Case:
    """512^2 u8, 8-connectivity: mask = 5x5 blur of noise, marker = max(mask-40, 0)."""
    mask = noise_blur_u8(H, W, rng_for(1, image_idx))
    return Case(hdome_marker(mask, h), mask, 8, "dilate")


def tissue_case(H: int = 4096, W: int = 4096, conn: int = 8, nblobs: int = 2000, h: int = 30,
                image_idx: int = 0) -> Case:
    """4096^2 u8 tissue-like blob field with an h-dome marker (h = 30)."""
    mask = blob_field_u8(H, W, nblobs, rng_for(2, image_idx))
    return Case(hdome_marker(mask, h), mask, conn, "dilate")


def sparse_seed_case(H: int = 16384, W: int = 16384, nblobs: int = 2000, nseeds: int = 1000,
                     image_idx: int = 0) -> Case:
    """16384^2 u8 blob field; marker = 0 except seeds equal to the mask."""
    rng = rng_for(3, image_idx)
    mask = blob_field_u8(H, W, nblobs, rng)
    return Case(seeds_marker(mask, nseeds, rng), mask, 8, "dilate")


def porous_skiz_case(H: int = 4096, W: int = 4096, nmarkers: int = 2000, nlabels: int = 2000,
                     thresh: int = 8, image_idx: int = 0):
    """Influence-zone input: the domain is the tissue-like blob field above a low threshold
    (every blob plus ~70 % of the noisy background: a percolating porous region); markers
    are `nmarkers` uniform pixels with labels uniform in 1..nlabels. Returns (markers uint32,
    domain mask uint8)."""
    rng = rng_for(10, image_idx)
    field = blob_field_u8(H, W, blob_count(H, W), rng)
    mask = (field > thresh).astype(np.uint8)
    markers = np.zeros((H, W), np.uint32)
    markers[rng.integers(0, H, nmarkers), rng.integers(0, W, nmarkers)] = rng.integers(1, nlabels + 1, nmarkers)
    return markers, mask


def _batch_image(args) -> Case:
    """Image i of an uneven batch (its own seeded generator, so images are independent)."""
    i, n, workload_id, min_side, max_side, conn = args
    lo, hi = math.log(min_side), math.log(max_side)
    rng = rng_for(workload_id, i)
    H = int(round(math.exp(rng.uniform(lo, hi))))
    W = int(round(math.exp(rng.uniform(lo, hi))))
    is16 = bool(rng.integers(0, 2))
    field = blob_field_u8(H, W, blob_count(H, W), rng)
    mask = to_u16(field) if is16 else field
    if i < n // 2:
        h = int(rng.integers(10, 61)) * (257 if is16 else 1)
        return Case(hdome_marker(mask, h), mask, conn, "dilate")
    return Case(fillholes_marker(mask), mask, conn, "erode")


def mixed_batch(n: int = 256, workload_id: int = 4, min_side: int = 256, max_side: int = 4096,
                conn: int = 8, workers: int = 0) -> list[Case]:
    """Uneven batch: log-uniform sides, u8/u16 with p = 1/2; the first half are
    h-dome dilations (h ~ U{10..60}, x257 for u16), the second half fill-holes.
    workers > 1 generates the images in that many spawned processes (same images)."""
    jobs = [(i, n, workload_id, min_side, max_side, conn) for i in range(n)]
    if workers and workers > 1 and n > 1:
        import multiprocessing
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(max_workers=min(workers, n),
                                 mp_context=multiprocessing.get_context("spawn")) as ex:
            return list(ex.map(_batch_image, jobs, chunksize=max(1, n // (4 * workers))))
    return [_batch_image(j) for j in jobs]
