"""CPU oracle for IWPP morphological reconstruction — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
(and its ``--impl reference`` arm) may import this package. The product library
(``paper_1605_00930_gb300``) never imports it and shares no code with it.

Contents
  * ``iwpp_oracle.c`` — Vincent's hybrid reconstruction (Sec. 3.1, Algorithm 7),
    single-threaded C, built here with gcc into ``liboracle.so``.
  * ``edt_oracle.c`` — the Euclidean distance transform by Voronoi-site propagation
    (Sec. 3.2, Algorithm 8) with a FIFO, in the same library.
  * ``wshed_oracle.c`` — marker-controlled watershed by flooding as an IWPP propagation of
    (level, label) pairs, in the same library.
  * ``skiz_oracle.c`` — the geodesic skeleton by influence zones (multi-source
    breadth-first propagation of (distance, label set)), in the same library.
  * ``bruteforce.py`` — Algorithm 1 (Jacobi iteration of Eq. "recon") in numpy.
  * ``features.py`` / ``mlp.py`` — plain numpy definitions of the per-tile
    features and of the 16-64-64-2 MLP used by the learned schedule.
  * ``ops.py`` — h-maxima, h-dome and regional maxima as compositions of the
    reconstruction, and regional maxima once more by plateau flooding.

Parity status: reconstruction is pinned by brute force, hand-worked cases,
invariants, duality, threshold decomposition and the binary special case
(connected components); the distance transform by the exact transform (brute force
and scipy) as a lower bound, exactness for a single site, site validity and the
local fixed point; the watershed's levels by brute-force relaxation and the erosion
reconstruction; the SKIZ by per-marker brute-force distances and scipy's chamfer
distance transform; see tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "iwpp_oracle.c"), os.path.join(_HERE, "edt_oracle.c"),
         os.path.join(_HERE, "wshed_oracle.c"), os.path.join(_HERE, "skiz_oracle.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

DTYPES = {np.dtype(np.uint8): 0, np.dtype(np.uint16): 1}
OPS = {"dilate": 0, "erode": 1}


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (portable C11, no host-specific flags)."""
    if force or not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(s) for s in _SRCS):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp] + _SRCS)
        os.replace(tmp, _LIB)
    return _LIB


def _bind(lib):
    """Declare the C functions' signatures on a loaded oracle library."""
    lib.oracle_reconstruct.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]
    lib.oracle_reconstruct.restype = ctypes.c_int
    lib.oracle_precondition_ok.argtypes = [ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                           ctypes.c_int]
    lib.oracle_precondition_ok.restype = ctypes.c_int
    lib.oracle_edt.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                               ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]
    lib.oracle_edt.restype = ctypes.c_int
    lib.oracle_watershed.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                                     ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_uint64)]
    lib.oracle_watershed.restype = ctypes.c_int
    lib.oracle_skiz.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]
    lib.oracle_skiz.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def _check(marker: np.ndarray, mask: np.ndarray):
    if marker.shape != mask.shape or marker.ndim != 2:
        raise ValueError("marker and mask must be equal-shape 2-D arrays")
    if marker.dtype != mask.dtype or marker.dtype not in DTYPES:
        raise ValueError("marker and mask must both be uint8 or both uint16")


def reconstruct(marker: np.ndarray, mask: np.ndarray, conn: int = 8, op: str = "dilate",
                return_pops: bool = False):
    """Vincent's hybrid reconstruction of ``mask`` from ``marker`` (a new array)."""
    _check(marker, mask)
    lib = _load()
    J = np.ascontiguousarray(marker).copy()
    I = np.ascontiguousarray(mask)
    pops = ctypes.c_uint64(0)
    rc = lib.oracle_reconstruct(J.ctypes.data, I.ctypes.data, J.shape[0], J.shape[1], int(conn),
                                OPS[op], DTYPES[J.dtype], ctypes.byref(pops))
    if rc != 0:
        raise ValueError(f"oracle_reconstruct failed with code {rc}")
    return (J, int(pops.value)) if return_pops else J


def precondition_ok(marker: np.ndarray, mask: np.ndarray, op: str = "dilate") -> bool:
    _check(marker, mask)
    lib = _load()
    J = np.ascontiguousarray(marker)
    I = np.ascontiguousarray(mask)
    rc = lib.oracle_precondition_ok(J.ctypes.data, I.ctypes.data, J.shape[0], J.shape[1],
                                    OPS[op], DTYPES[J.dtype])
    if rc < 0:
        raise ValueError("bad argument")
    return rc == 1


def edt(mask: np.ndarray, conn: int = 8, return_pops: bool = False):
    """Distance transform by Voronoi-site propagation (Algorithm 8) of a 2-D mask
    (non-zero = foreground). Returns (site, d2): int64 arrays, site = y * W + x of the
    pixel's background site or -1, d2 = squared Euclidean distance to it or -1."""
    if mask.ndim != 2:
        raise ValueError("mask must be 2-D")
    lib = _load()
    fg = np.ascontiguousarray(mask != 0, dtype=np.uint8)
    site = np.empty(fg.shape, np.int64)
    d2 = np.empty(fg.shape, np.int64)
    pops = ctypes.c_uint64(0)
    rc = lib.oracle_edt(fg.ctypes.data, fg.shape[0], fg.shape[1], int(conn), site.ctypes.data, d2.ctypes.data,
                        ctypes.byref(pops))
    if rc != 0:
        raise ValueError(f"oracle_edt failed with code {rc}")
    return (site, d2, int(pops.value)) if return_pops else (site, d2)


def watershed(markers: np.ndarray, gradient: np.ndarray, conn: int = 8, return_pops: bool = False):
    """Flooding of `gradient` from labelled `markers` (uint32, 0 = none, 1..65534): returns
    (label uint32, level int32) — a label reaching each pixel at its minimax flooding level
    (which of several is order-dependent), and that level (0 / -1 where no marker reaches)."""
    if markers.shape != gradient.shape or markers.ndim != 2 or gradient.dtype not in DTYPES:
        raise ValueError("markers and a uint8/uint16 gradient of the same 2-D shape")
    lib = _load()
    mk = np.ascontiguousarray(markers, dtype=np.uint32)
    g = np.ascontiguousarray(gradient)
    label = np.empty(mk.shape, np.uint32)
    level = np.empty(mk.shape, np.int32)
    pops = ctypes.c_uint64(0)
    rc = lib.oracle_watershed(mk.ctypes.data, g.ctypes.data, DTYPES[g.dtype], mk.shape[0], mk.shape[1], int(conn),
                              label.ctypes.data, level.ctypes.data, ctypes.byref(pops))
    if rc != 0:
        raise ValueError(f"oracle_watershed failed with code {rc}")
    return (label, level, int(pops.value)) if return_pops else (label, level)


def skiz(markers: np.ndarray, mask: np.ndarray, conn: int = 8, return_pops: bool = False):
    """Geodesic influence zones of labelled `markers` (uint32, 0 = none, 1..65534) inside the
    domain mask != 0 or marker != 0: returns a dict of int32 ``dist`` (-1 = unreached) and
    uint32 ``lmin``, ``lmax`` (smallest / largest label among the nearest markers, 0 = unreached)
    and ``zone`` (the label where lmin == lmax, 0 on the skeleton and where unreached)."""
    if markers.shape != mask.shape or markers.ndim != 2:
        raise ValueError("markers and mask of the same 2-D shape")
    lib = _load()
    mk = np.ascontiguousarray(markers, dtype=np.uint32)
    m = np.ascontiguousarray(mask != 0, dtype=np.uint8)
    out = {"dist": np.empty(mk.shape, np.int32), "lmin": np.empty(mk.shape, np.uint32),
           "lmax": np.empty(mk.shape, np.uint32), "zone": np.empty(mk.shape, np.uint32)}
    pops = ctypes.c_uint64(0)
    rc = lib.oracle_skiz(mk.ctypes.data, m.ctypes.data, mk.shape[0], mk.shape[1], int(conn),
                         out["dist"].ctypes.data, out["lmin"].ctypes.data, out["lmax"].ctypes.data,
                         out["zone"].ctypes.data, ctypes.byref(pops))
    if rc != 0:
        raise ValueError(f"oracle_skiz failed with code {rc}")
    if return_pops:
        out["pops"] = int(pops.value)
    return out


def reconstruct_many(items, threads: int | None = None):
    """Reconstruct a list of (marker, mask, conn, op) tuples on ``threads`` host
    threads, one image per thread at a time (the C call releases the GIL)."""
    _load()
    threads = threads or len(os.sched_getaffinity(0))
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(lambda it: reconstruct(*it), items))
