"""Planted mistakes: each test compiles a copy of the C oracle with one plausible mistake
(a dropped term, a wrong sign, offset or condition), swaps it in for the real oracle, and
checks that the pins catch it. If a mistake survived every pin, the pins could not be trusted
to catch it in the oracle either. The mistakes are planted in the oracle, on the CPU; the
real oracle sources are not modified (a temporary copy is compiled)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from oracle import bruteforce

from .test_oracle_skiz import brute as skiz_brute
from .test_oracle_watershed import brute as wshed_brute

# (file, text of the correct code, the mistake planted in its place, which pin catches it)
MUTANTS = [
    # reconstruction (Algorithm 7)
    ("iwpp_oracle.c", "if (J[q] < J[p] && J[q] < I[q]) {", "if (0) {", "recon"),                 # no FIFO seeding
    ("iwpp_oracle.c", "J[q] = imin(J[p], I[q]);", "J[q] = J[p];", "recon"),                      # mask clamp dropped
    ("iwpp_oracle.c", "for (int half = 0; half < 2; half++) {", "for (int half = 0; half < 1; half++) {",
     "recon"),                                                                                    # half neighbourhood
    ("iwpp_oracle.c", "static const int NPLUS8[4][2] = {{-1, -1}, {-1, 0}, {-1, 1}, {0, -1}};",
     "static const int NPLUS8[4][2] = {{-1, -1}, {-1, 0}, {-1, 1}, {0, 1}};", "recon"),           # wrong offset
    ("iwpp_oracle.c", "J[q] = imax(J[p], I[q]);", "J[q] = imin(J[p], I[q]);", "recon"),         # erosion update
    ("iwpp_oracle.c", "J[p] = imin(m, I[p]);", "J[p] = m;", "recon"),                            # scan clamp dropped
    # SKIZ
    ("skiz_oracle.c", "} else if (dist_out[r] == dn) {", "} else if (0) {", "skiz"),            # no label merge
    ("skiz_oracle.c", "if (lmax_out[p] > lmax_out[r]) lmax_out[r] = lmax_out[p];", "", "skiz"),  # max label lost
    ("skiz_oracle.c", "if (!mask[r] && !markers[r]) continue; /* outside the domain */", "", "skiz"),
    ("skiz_oracle.c", "const int32_t dn = dist_out[p] + 1;", "const int32_t dn = dist_out[p] + 2;", "skiz"),
    # watershed
    ("wshed_oracle.c", "const int64_t cl = lev[p] > GRAD(r) ? lev[p] : GRAD(r), cb = lab[p];",
     "const int64_t cl = lev[p], cb = lab[p];", "wshed"),                                         # gradient ignored
    ("wshed_oracle.c", "if (markers[r]) continue;   /* markers are fixed */", "", "wshed"),
    # distance transform (Algorithm 8)
    ("edt_oracle.c", "return dy * dy + dx * dx;", "return dy * dy + dx;", "edt"),               # wrong metric
    ("edt_oracle.c", "            if (edge) {", "            if (0) {", "edt"),                  # no seeding
]


def _build_mutant(tmp_path, fname, old, new):
    src_dir = os.path.dirname(oracle.__file__)
    for f in os.listdir(src_dir):
        if f.endswith(".c"):
            shutil.copy(os.path.join(src_dir, f), tmp_path / f)
    text = (tmp_path / fname).read_text()
    assert text.count(old) >= 1, f"mutation site not found in {fname}: {old}"
    (tmp_path / fname).write_text(text.replace(old, new, 1))
    lib = tmp_path / "libmutant.so"
    srcs = [str(tmp_path / f) for f in sorted(os.listdir(tmp_path)) if f.endswith(".c")]
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", str(lib)] + srcs)
    return oracle._bind(ctypes.CDLL(str(lib)))


def _recon_pins_hold():
    rng = np.random.default_rng(7)
    for _ in range(150):
        H, W = int(rng.integers(2, 9)), int(rng.integers(2, 9))
        for op in ("dilate", "erode"):
            for conn in (4, 8):
                mask = rng.integers(0, 8, size=(H, W)).astype(np.uint8)
                if op == "dilate":
                    marker = (mask * (rng.random((H, W)) < 0.2)).astype(np.uint8)
                else:
                    marker = mask.copy()
                    marker[1:-1, 1:-1] = 255
                got = oracle.reconstruct(marker, mask, conn, op)
                if not np.array_equal(got, bruteforce.reconstruct(marker, mask, conn, op)):
                    return False
    return True


def _skiz_pins_hold():
    rng = np.random.default_rng(8)
    for _ in range(150):
        H, W = int(rng.integers(2, 10)), int(rng.integers(2, 10))
        mask = (rng.random((H, W)) < 0.75).astype(np.uint8)
        markers = np.zeros((H, W), np.uint32)
        n = int(rng.integers(1, 5))
        markers[rng.integers(0, H, n), rng.integers(0, W, n)] = rng.integers(1, 4, n)
        for conn in (4, 8):
            got, exp = oracle.skiz(markers, mask, conn), skiz_brute(markers, mask, conn)
            if any(not np.array_equal(got[k], exp[k]) for k in ("dist", "lmin", "lmax", "zone")):
                return False
    return True


def _wshed_pins_hold():
    rng = np.random.default_rng(9)
    for _ in range(60):
        H, W = int(rng.integers(2, 8)), int(rng.integers(2, 8))
        grad = rng.integers(0, 6, size=(H, W)).astype(np.uint8)
        markers = np.zeros((H, W), np.uint32)
        n = int(rng.integers(1, 4))
        markers[rng.integers(0, H, n), rng.integers(0, W, n)] = rng.integers(1, 4, n)
        for conn in (4, 8):
            lab, lev = oracle.watershed(markers, grad, conn)
            if not np.array_equal(lev, wshed_brute(markers, grad, conn)[1]):
                return False
            if not np.array_equal(lab[markers > 0], markers[markers > 0]):   # markers keep their labels
                return False
    return True


def _edt_pins_hold():
    rng = np.random.default_rng(10)
    for _ in range(40):
        H, W = int(rng.integers(2, 12)), int(rng.integers(2, 12))
        fg = np.ones((H, W), np.uint8)
        y, x = int(rng.integers(0, H)), int(rng.integers(0, W))
        fg[y, x] = 0                      # one background pixel: the transform is exact
        _, d2 = oracle.edt(fg, 8)
        yy, xx = np.mgrid[0:H, 0:W]
        if not np.array_equal(d2, (yy - y) ** 2 + (xx - x) ** 2):
            return False
    return True


PINS = {"recon": _recon_pins_hold, "skiz": _skiz_pins_hold, "wshed": _wshed_pins_hold, "edt": _edt_pins_hold}


def test_pins_hold_for_the_real_oracle():
    for name, pin in PINS.items():
        assert pin(), name


@pytest.mark.parametrize("fname,old,new,pin", MUTANTS, ids=[f"{m[0]}:{i}" for i, m in enumerate(MUTANTS)])
def test_planted_mistake_is_caught(tmp_path, monkeypatch, fname, old, new, pin):
    lib = _build_mutant(tmp_path, fname, old, new)
    monkeypatch.setattr(oracle, "_lib", lib)
    assert not PINS[pin](), f"the planted mistake in {fname} survived the {pin} pins"
