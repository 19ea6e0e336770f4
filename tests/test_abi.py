"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function that include/iwpp.h declares; host-side argument checks reject bad
calls before anything is enqueued (no GPU needed for these)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "iwpp.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"IWPP_API\s+[\w\s\*]+?\b(iwpp_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def iwpp():
    if shutil.which("nvcc") is None and not os.path.exists(
            os.path.join(ROOT, "paper_1605_00930_gb300", "libiwpp.so")):
        pytest.skip("no nvcc and no prebuilt library")
    from paper_1605_00930_gb300 import build
    build.build()
    from paper_1605_00930_gb300 import iwpp as m
    m.lib()
    return m


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["iwpp_reconstruct", "iwpp_reconstruct_plan", "iwpp_workspace_bytes", "iwpp_sync_status",
              "iwpp_default_plan"]:
        assert n in names


def test_library_exports_every_declared_symbol(iwpp):
    L = iwpp.lib()
    for name in _declared():
        assert hasattr(L, name), name
    # and the binding covers each one under the same name
    assert set(_declared()) <= set(iwpp.exported_symbols())


def test_header_constants_match_the_binding(iwpp):
    """The binding's enum values and plan layout are the header's (parsed as text)."""
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                            "iwpp.h")).read()

    def enum_value(name):
        m = re.search(r"\b" + name + r"\s*=\s*(\d+)", hdr)
        assert m, name
        return int(m.group(1))

    for name in ("IWPP_U8", "IWPP_U16", "IWPP_DILATE", "IWPP_ERODE", "IWPP_SOLVER_QUEUE",
                 "IWPP_SOLVER_REGISTER", "IWPP_SOLVER_COOP"):
        assert getattr(iwpp, name) == enum_value(name), name
    for code, name in iwpp.STATUS.items():
        assert enum_value(name) == code, name
    body = hdr[hdr.index("typedef struct {\n    int32_t tile_h"):]
    body = body[:body.index("} iwpp_plan;")]
    fields = re.findall(r"(?:int32_t|int64_t|uint16_t)\s+([a-z_]+(?:,\s*[a-z_]+)*)", body)
    names = [n.strip() for f in fields for n in f.split(",")]
    assert names == [f for f, _ in iwpp.Plan._fields_]


def test_default_plan_and_shapes(iwpp):
    p = iwpp.iwpp_default_plan()
    assert iwpp.iwpp_tile_shape_supported(p.tile_h, p.tile_w)
    assert p.sweeps >= 0 and 16 <= p.smem_queue_cap <= p.tile_h * p.tile_w
    assert (p.tile_h, p.tile_w, p.local_solver) == (64, 64, iwpp.IWPP_SOLVER_COOP)
    b = iwpp.iwpp_default_batch_plan()
    assert (b.tile_h, b.tile_w, b.local_solver) == (64, 64, iwpp.IWPP_SOLVER_COOP)
    assert iwpp.iwpp_tile_shape_supported(b.tile_h, b.tile_w)
    for shape in [(32, 32), (32, 64), (64, 64), (16, 32), (16, 64)]:
        assert iwpp.iwpp_tile_shape_supported(*shape)
    assert not iwpp.iwpp_tile_shape_supported(48, 48)


def test_host_argument_errors_return_before_any_launch(iwpp):
    buf = (ctypes.c_uint8 * 4096)()
    a = ctypes.addressof(buf)
    a16 = (a + 15) // 16 * 16
    ws = (a + 255) // 256 * 256 if a % 256 else a
    null = ctypes.c_void_p(0)
    P = ctypes.c_void_p
    # null pointers
    assert iwpp.iwpp_reconstruct(null, P(a16), 4, 4, 8, 0, 0, P(ws), 16, null) == 1
    # misaligned image
    assert iwpp.iwpp_reconstruct(P(a16 + 1), P(a16), 4, 4, 8, 0, 0, P(ws), 16, null) == 1
    # bad sizes, connectivity, op, dtype
    assert iwpp.iwpp_reconstruct(P(a16), P(a16), 0, 4, 8, 0, 0, P(ws), 16, null) == 1
    assert iwpp.iwpp_reconstruct(P(a16), P(a16), 1 << 21, 1 << 20, 8, 0, 0, P(ws), 16, null) == 1   # 2^41 px
    assert iwpp.iwpp_reconstruct(P(a16), P(a16), 1 << 31, 1, 8, 0, 0, P(ws), 16, null) == 1
    assert iwpp.iwpp_reconstruct(P(a16), P(a16), 4, 4, 6, 0, 0, P(ws), 16, null) == 1
    assert iwpp.iwpp_reconstruct(P(a16), P(a16), 4, 4, 8, 2, 0, P(ws), 16, null) == 1
    assert iwpp.iwpp_reconstruct(P(a16), P(a16), 4, 4, 8, 0, 3, P(ws), 16, null) == 1
    # bad plan
    p = iwpp.iwpp_default_plan()
    p.tile_h = 48
    assert iwpp.iwpp_reconstruct_plan(P(a16), P(a16), 4, 4, 8, 0, 0, p, P(ws), 16, null) == 1
    p = iwpp.iwpp_default_plan()
    p.smem_queue_cap = 8
    assert iwpp.iwpp_reconstruct_plan(P(a16), P(a16), 4, 4, 8, 0, 0, p, P(ws), 16, null) == 1
    # the register solver needs 16 x 64 tiles; unknown solvers, value levels beyond 16 and
    # value levels with the queue solver are rejected
    for th, tw, solver, levels in [(32, 32, 1, 0), (32, 64, 1, 0), (16, 64, 3, 0), (16, 64, 1, 17),
                                   (16, 64, 0, 4), (16, 64, 1, -1), (16, 64, 2, 0), (32, 64, 2, 0),
                                   (64, 64, 2, 4)]:
        p = iwpp.iwpp_default_plan()
        p.tile_h, p.tile_w, p.local_solver, p.value_levels = th, tw, solver, levels
        assert iwpp.iwpp_reconstruct_plan(P(a16), P(a16), 4, 4, 8, 0, 0, p, P(ws), 16, null) == 1
    # the cooperative solver takes no revisit sweeps and at most 6 CTAs per SM
    for kw in [{"revisit_sweeps": 2}, {"blocks_per_sm": 7}]:
        p = iwpp.iwpp_default_plan()
        p.tile_h, p.tile_w, p.local_solver = 64, 64, 2
        for k, v in kw.items():
            setattr(p, k, v)
        assert iwpp.iwpp_reconstruct_plan(P(a16), P(a16), 4, 4, 8, 0, 0, p, P(ws), 16, null) == 1, kw
    # missing / misaligned workspace
    assert iwpp.iwpp_reconstruct(P(a16), P(a16), 4, 4, 8, 0, 0, null, 16, null) == 3
    assert iwpp.iwpp_reconstruct(P(a16), P(a16), 4, 4, 8, 0, 0, P(ws + 16), 16, null) == 3


def test_edt_host_errors_return_before_any_launch(iwpp):
    buf = (ctypes.c_uint8 * 4096)()
    a = ctypes.addressof(buf)
    a16 = (a + 15) // 16 * 16
    ws = (a + 255) // 256 * 256 if a % 256 else a
    P, null = ctypes.c_void_p, ctypes.c_void_p(0)
    assert iwpp.iwpp_edt_workspace_bytes(40000, 10) == 0 and iwpp.iwpp_edt_workspace_bytes(0, 5) == 0
    assert iwpp.iwpp_edt_workspace_bytes(100, 100) > 0
    assert iwpp.iwpp_edt(null, P(a16), null, 4, 4, 8, P(ws), 4096, null) == 1          # no mask
    assert iwpp.iwpp_edt(P(a16), P(a16), null, 4, 4, 6, P(ws), 4096, null) == 1        # connectivity
    assert iwpp.iwpp_edt(P(a16), P(a16 + 2), null, 4, 4, 8, P(ws), 4096, null) == 1    # misaligned sites
    assert iwpp.iwpp_edt(P(a16), P(a16), null, 40000, 4, 8, P(ws), 4096, null) == 1    # too large
    assert iwpp.iwpp_edt(P(a16), P(a16), null, 4, 4, 8, null, 4096, null) == 3         # no workspace
    assert iwpp.iwpp_edt(P(a16), P(a16), null, 4, 4, 8, P(ws), 16, null) == 3          # workspace too small


def test_watershed_and_operator_host_errors(iwpp):
    buf = (ctypes.c_uint8 * 4096)()
    a = ctypes.addressof(buf)
    a16 = (a + 15) // 16 * 16
    ws = (a + 255) // 256 * 256 if a % 256 else a
    P, null = ctypes.c_void_p, ctypes.c_void_p(0)
    assert iwpp.iwpp_watershed_workspace_bytes(0, 4) == 0 and iwpp.iwpp_watershed_workspace_bytes(1 << 31, 1) == 0
    assert iwpp.iwpp_watershed_workspace_bytes(64, 64) > 0
    assert iwpp.iwpp_watershed(null, P(a16), 0, P(a16), null, 4, 4, 8, P(ws), 4096, null) == 1      # no markers
    assert iwpp.iwpp_watershed(P(a16), P(a16), 2, P(a16), null, 4, 4, 8, P(ws), 4096, null) == 1    # dtype
    assert iwpp.iwpp_watershed(P(a16), P(a16), 0, P(a16), null, 4, 4, 5, P(ws), 4096, null) == 1    # connectivity
    assert iwpp.iwpp_watershed(P(a16), P(a16), 0, P(a16 + 1), null, 4, 4, 8, P(ws), 4096, null) == 1
    assert iwpp.iwpp_watershed(P(a16), P(a16), 0, P(a16), null, 4, 4, 8, null, 4096, null) == 3
    assert iwpp.iwpp_watershed(P(a16), P(a16), 0, P(a16), null, 4, 4, 8, P(ws), 8, null) == 3
    for fn in (iwpp.iwpp_hmaxima, iwpp.iwpp_hdome):
        assert fn(null, P(a16), 4, 4, 3, 8, 0, P(ws), 4096, null) == 1
        assert fn(P(a16 + 1), P(a16), 4, 4, 3, 8, 0, P(ws), 4096, null) == 1
        assert fn(P(a16), P(a16), 4, 4, 3, 8, 7, P(ws), 4096, null) == 1
    assert iwpp.iwpp_regional_maxima(P(a16), P(a16), null, 4, 4, 8, 0, P(ws), 4096, null) == 1


def test_skiz_host_errors(iwpp):
    buf = (ctypes.c_uint8 * 4096)()
    a = ctypes.addressof(buf)
    a16 = (a + 15) // 16 * 16
    ws = (a + 255) // 256 * 256 if a % 256 else a
    P, null = ctypes.c_void_p, ctypes.c_void_p(0)
    assert iwpp.iwpp_skiz_workspace_bytes(0, 4) == 0 and iwpp.iwpp_skiz_workspace_bytes(1 << 16, 1 << 15) == 0
    assert iwpp.iwpp_skiz_workspace_bytes(64, 64) >= 64 * 64 * 8
    assert iwpp.iwpp_skiz(null, P(a16), P(a16), null, null, 4, 4, 8, P(ws), 4096, null) == 1      # no markers
    assert iwpp.iwpp_skiz(P(a16), null, P(a16), null, null, 4, 4, 8, P(ws), 4096, null) == 1      # no mask
    assert iwpp.iwpp_skiz(P(a16), P(a16), null, null, null, 4, 4, 8, P(ws), 4096, null) == 1      # no output
    assert iwpp.iwpp_skiz(P(a16), P(a16), P(a16), null, null, 4, 4, 6, P(ws), 4096, null) == 1    # connectivity
    assert iwpp.iwpp_skiz(P(a16), P(a16), P(a16 + 2), null, null, 4, 4, 8, P(ws), 4096, null) == 1
    assert iwpp.iwpp_skiz(P(a16), P(a16), P(a16), P(a16 + 1), null, 4, 4, 8, P(ws), 4096, null) == 1
    assert iwpp.iwpp_skiz(P(a16), P(a16), P(a16), null, null, 1 << 16, 1 << 15, 8, P(ws), 4096, null) == 1
    assert iwpp.iwpp_skiz(P(a16), P(a16), P(a16), null, null, 4, 4, 8, null, 4096, null) == 3
    assert iwpp.iwpp_skiz(P(a16), P(a16), P(a16), null, null, 4, 4, 8, P(ws), 64, null) == 3


def test_host_band_errors(iwpp):
    buf = (ctypes.c_uint8 * 4096)()
    a = ctypes.addressof(buf)
    ws = (a + 255) // 256 * 256 if a % 256 else a
    P, null = ctypes.c_void_p, ctypes.c_void_p(0)
    f = iwpp.iwpp_reconstruct_host
    assert iwpp.iwpp_host_workspace_bytes(0, 4, 0, 4) == 0 and iwpp.iwpp_host_workspace_bytes(4, 4, 0, 0) == 0
    assert iwpp.iwpp_host_workspace_bytes(4, 4, 2, 4) == 0
    assert f(null, P(a), 4, 4, 8, 0, 0, 2, P(ws), 4096, null, None) == 1          # no marker
    assert f(P(a), null, 4, 4, 8, 0, 0, 2, P(ws), 4096, null, None) == 1          # no mask
    assert f(P(a), P(a), 4, 4, 5, 0, 0, 2, P(ws), 4096, null, None) == 1          # connectivity
    assert f(P(a), P(a), 4, 4, 8, 2, 0, 2, P(ws), 4096, null, None) == 1          # op
    assert f(P(a), P(a), 4, 4, 8, 0, 3, 2, P(ws), 4096, null, None) == 1          # dtype
    assert f(P(a), P(a), 4, 4, 8, 0, 0, 0, P(ws), 4096, null, None) == 1          # band height
    assert f(P(a), P(a), 0, 4, 8, 0, 0, 2, P(ws), 4096, null, None) == 1          # size


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import importlib
    from paper_1605_00930_gb300 import iwpp as m
    mod = importlib.reload(m)
    monkeypatch.setattr(mod, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(mod, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        mod.lib()
    importlib.reload(m)


def test_batch_tile_count_is_host_only(iwpp):
    P = iwpp.Image
    imgs = (P * 3)()
    buf = (ctypes.c_uint8 * 64)()
    a16 = (ctypes.addressof(buf) + 15) // 16 * 16
    for i, (H, W) in enumerate([(1, 1), (33, 64), (100, 31)]):
        imgs[i] = P(a16, a16, H, W, 8, 0, 0, 0)
    p = iwpp.iwpp_default_plan()
    p.tile_h, p.tile_w, p.local_solver = 32, 32, iwpp.IWPP_SOLVER_QUEUE
    assert iwpp.iwpp_batch_tile_count(imgs, p) == 1 + 2 * 2 + 4 * 1
    imgs[1].connectivity = 6
    assert iwpp.iwpp_batch_tile_count(imgs, p) == -1


def _images(iwpp, shapes, conn=8):
    P = iwpp.Image
    imgs = (P * len(shapes))()
    buf = (ctypes.c_uint8 * 64)()
    a16 = (ctypes.addressof(buf) + 15) // 16 * 16
    for i, (H, W) in enumerate(shapes):
        imgs[i] = P(a16, a16, H, W, conn, 0, i % 2, 0)
    return imgs, buf


def test_batch_block_count_and_sched_layout_are_host_only(iwpp):
    """Feature blocks are the 64 x 64 blocks of every image (partial blocks at the right and
    bottom edges count); the scheduling workspace holds the features array at a 256-byte
    aligned offset with room for every block's 16 floats."""
    shapes = [(1, 1), (33, 64), (100, 31), (64, 65), (4096, 257), (129, 4097)]
    imgs, buf = _images(iwpp, shapes)
    nb = sum(((H + 63) // 64) * ((W + 63) // 64) for H, W in shapes)
    assert iwpp.iwpp_batch_block_count(imgs) == nb
    bp = iwpp.iwpp_default_batch_plan()
    assert (bp.tile_h, bp.tile_w) == (iwpp.FEATURE_BLOCK, iwpp.FEATURE_BLOCK)
    assert iwpp.iwpp_batch_tile_count(imgs, bp) == nb
    total = iwpp.iwpp_sched_workspace_bytes(imgs, bp)
    off = iwpp.iwpp_sched_features_offset(imgs, bp)
    assert off >= 0 and off % 256 == 0
    assert off + nb * iwpp.NFEAT * 4 <= total
    # a plan whose tiles do not divide the feature block, an empty image and an empty batch
    # are rejected
    p = iwpp.iwpp_default_batch_plan()
    p.tile_h, p.tile_w, p.local_solver = 48, 64, iwpp.IWPP_SOLVER_QUEUE
    assert iwpp.iwpp_sched_workspace_bytes(imgs, p) == 0
    assert iwpp.iwpp_sched_features_offset(imgs, p) == -1
    imgs[2].W = 0
    assert iwpp.iwpp_batch_block_count(imgs) == -1
    assert iwpp.iwpp_sched_features_offset(imgs, bp) == -1
    assert iwpp.iwpp_batch_block_count((iwpp.Image * 0)()) == -1


def test_batch_launch_count(iwpp):
    """Launch accounting of one batch call: per 32 image descriptors one table upload, then
    the tile map, scan, compaction, queue finalisation (phases 1) and the drain (phases 2);
    the learned call with features from the scan adds per 32 descriptors one schedule-table
    upload, the MLP, the sort's keys, bucket scan and scatter, and the sweeps-only pass. For
    512 images that is 21 and 42 launches, the counts the ncu launch list of the 512-image
    batch shows per call."""
    assert iwpp.iwpp_batch_launch_count(512, 3) == 21
    assert iwpp.iwpp_batch_launch_count(512, 7) == 42
    for n in (1, 31, 32, 33, 64, 65, 512, 513):
        chunks = (n + 31) // 32
        assert iwpp.iwpp_batch_launch_count(n, 1) == chunks + 4
        assert iwpp.iwpp_batch_launch_count(n, 2) == 1
        assert iwpp.iwpp_batch_launch_count(n, 3) == chunks + 5
        assert iwpp.iwpp_batch_launch_count(n, 5) == 2 * chunks + 9
        assert iwpp.iwpp_batch_launch_count(n, 7) == 2 * chunks + 10
    for n, ph in [(0, 3), (-1, 3), (5, 0), (5, 4), (5, 8)]:
        assert iwpp.iwpp_batch_launch_count(n, ph) == -1
