"""Python binding of the C ABI in include/iwpp.h (argument marshalling only).

Every step of the reconstruction runs in the CUDA library ``libiwpp.so``; this
module only passes pointers, sizes and the stream handle through ctypes. PyTorch
is used for device memory and streams. If the library is missing, every call
raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
# The in-tree build; IWPP_LIB_PATH names another build of the same library (e.g. one compiled
# with different tuning switches).
LIB_PATH = os.environ.get("IWPP_LIB_PATH") or os.path.join(_HERE, "libiwpp.so")

IWPP_U8, IWPP_U16 = 0, 1
IWPP_DILATE, IWPP_ERODE = 0, 1
STATUS = {0: "IWPP_OK", 1: "IWPP_ERR_ARG", 2: "IWPP_ERR_PRECONDITION", 3: "IWPP_ERR_WORKSPACE",
          4: "IWPP_ERR_QUEUE_FULL", 5: "IWPP_ERR_TIMEOUT", 6: "IWPP_ERR_CUDA", 7: "IWPP_ERR_INTERNAL"}
OPS = {"dilate": IWPP_DILATE, "erode": IWPP_ERODE}
IWPP_SOLVER_QUEUE, IWPP_SOLVER_REGISTER, IWPP_SOLVER_COOP = 0, 1, 2


class IwppError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {STATUS.get(code, code)}" if what else STATUS.get(code, str(code)))


class Plan(ctypes.Structure):
    _fields_ = [("tile_h", ctypes.c_int32), ("tile_w", ctypes.c_int32), ("sweeps", ctypes.c_int32),
                ("revisit_sweeps", ctypes.c_int32), ("smem_queue_cap", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("local_solver", ctypes.c_int32), ("value_levels", ctypes.c_int32),
                ("watchdog_ns", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}

    def __repr__(self):
        return f"Plan({self.as_dict()})"


class Image(ctypes.Structure):
    """iwpp_image: one image of a batch (device pointers)."""
    _fields_ = [("marker_inout", ctypes.c_void_p), ("mask", ctypes.c_void_p), ("H", ctypes.c_int64),
                ("W", ctypes.c_int64), ("connectivity", ctypes.c_int32), ("op", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()

# (name, restype, argtypes) of every exported C function
_PROTOS = [
    ("iwpp_default_plan", ctypes.c_int, [ctypes.POINTER(Plan)]),
    ("iwpp_default_batch_plan", ctypes.c_int, [ctypes.POINTER(Plan)]),
    ("iwpp_tile_shape_supported", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32]),
    ("iwpp_workspace_bytes", ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                               ctypes.POINTER(Plan)]),
    ("iwpp_reconstruct", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_size_t, ctypes.c_void_p]),
    ("iwpp_reconstruct_plan", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                             ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.POINTER(Plan), ctypes.c_void_p, ctypes.c_size_t,
                                             ctypes.c_void_p]),
    ("iwpp_scan", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                 ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Plan),
                                 ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("iwpp_drain", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                  ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Plan),
                                  ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("iwpp_batch_tile_count", ctypes.c_int64, [ctypes.POINTER(Image), ctypes.c_int, ctypes.POINTER(Plan)]),
    ("iwpp_batch_workspace_bytes", ctypes.c_size_t, [ctypes.POINTER(Image), ctypes.c_int,
                                                     ctypes.POINTER(Plan)]),
    ("iwpp_reconstruct_batch", ctypes.c_int, [ctypes.POINTER(Image), ctypes.c_int, ctypes.POINTER(Plan),
                                              ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("iwpp_reconstruct_batch_sched", ctypes.c_int, [ctypes.POINTER(Image), ctypes.c_int, ctypes.POINTER(Plan),
                                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                    ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("iwpp_reconstruct_batch_phase", ctypes.c_int, [ctypes.POINTER(Image), ctypes.c_int, ctypes.POINTER(Plan),
                                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                                    ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("iwpp_batch_launch_count", ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
    ("iwpp_reconstruct_batch_learned", ctypes.c_int, [ctypes.POINTER(Image), ctypes.c_int, ctypes.POINTER(Plan),
                                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                      ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                                      ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("iwpp_sched_features_offset", ctypes.c_int64, [ctypes.POINTER(Image), ctypes.c_int, ctypes.POINTER(Plan)]),
    ("iwpp_batch_graph_create", ctypes.c_int, [ctypes.POINTER(Image), ctypes.c_int, ctypes.POINTER(Plan),
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)]),
    ("iwpp_graph_launch", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("iwpp_graph_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("iwpp_autotune_batch", ctypes.c_int, [ctypes.POINTER(Image), ctypes.c_int, ctypes.POINTER(Plan),
                                           ctypes.c_int, ctypes.c_char_p, ctypes.c_void_p,
                                           ctypes.POINTER(ctypes.c_float)]),
    ("iwpp_batch_block_count", ctypes.c_int64, [ctypes.POINTER(Image), ctypes.c_int]),
    ("iwpp_sched_workspace_bytes", ctypes.c_size_t, [ctypes.POINTER(Image), ctypes.c_int, ctypes.POINTER(Plan)]),
    ("iwpp_batch_features", ctypes.c_int, [ctypes.POINTER(Image), ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_size_t, ctypes.c_void_p]),
    ("iwpp_mlp_forward", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    ("iwpp_mlp_train", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_uint64,
                                      ctypes.c_int64, ctypes.c_void_p]),
    ("iwpp_schedule_from_predictions", ctypes.c_int, [ctypes.POINTER(Image), ctypes.c_int, ctypes.POINTER(Plan),
                                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                      ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("iwpp_schedule_learned", ctypes.c_int, [ctypes.POINTER(Image), ctypes.c_int, ctypes.POINTER(Plan),
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_size_t, ctypes.c_void_p]),
    ("iwpp_tile_work_to_blocks", ctypes.c_int, [ctypes.POINTER(Image), ctypes.c_int, ctypes.POINTER(Plan),
                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                                ctypes.c_void_p]),
    ("iwpp_reconstruct_noalloc", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                                ctypes.POINTER(ctypes.c_int)]),
    ("iwpp_hmaxima", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                    ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                    ctypes.c_void_p]),
    ("iwpp_hdome", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                  ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                  ctypes.c_void_p]),
    ("iwpp_regional_maxima", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                            ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_size_t, ctypes.c_void_p]),
    ("iwpp_watershed_workspace_bytes", ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int64]),
    ("iwpp_watershed", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                      ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("iwpp_host_workspace_bytes", ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int64]),
    ("iwpp_reconstruct_host", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                             ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                             ctypes.POINTER(ctypes.c_int32)]),
    ("iwpp_skiz_workspace_bytes", ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int64]),
    ("iwpp_skiz", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                                 ctypes.c_size_t, ctypes.c_void_p]),
    ("iwpp_edt_workspace_bytes", ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int64]),
    ("iwpp_edt", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("iwpp_sync_status", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("iwpp_work_counters", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_uint64)]),
]


def lib():
    """Load libiwpp.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -m paper_1605_00930_gb300.build` (no CPU fallback exists)")
            L = ctypes.CDLL(LIB_PATH)
            for name, res, args in _PROTOS:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def exported_symbols():
    return [p[0] for p in _PROTOS]


# ---- thin wrappers with the C names ----------------------------------------------------

def iwpp_default_plan() -> Plan:
    """Default plan of single-image calls (64 x 64 tiles, cooperative solver)."""
    p = Plan()
    lib().iwpp_default_plan(ctypes.byref(p))
    return p


def iwpp_default_batch_plan() -> Plan:
    """Default plan of batch calls (the single-image default: 64 x 64 tiles, cooperative solver)."""
    p = Plan()
    lib().iwpp_default_batch_plan(ctypes.byref(p))
    return p


def iwpp_tile_shape_supported(th: int, tw: int) -> bool:
    return bool(lib().iwpp_tile_shape_supported(th, tw))


def iwpp_workspace_bytes(H: int, W: int, dtype: int, plan: Plan | None = None) -> int:
    return int(lib().iwpp_workspace_bytes(H, W, dtype, ctypes.byref(plan) if plan is not None else None))


def iwpp_reconstruct(marker_ptr, mask_ptr, H, W, conn, op, dtype, ws_ptr, ws_bytes, stream) -> int:
    return lib().iwpp_reconstruct(marker_ptr, mask_ptr, H, W, conn, op, dtype, ws_ptr, ws_bytes, stream)


def iwpp_reconstruct_plan(marker_ptr, mask_ptr, H, W, conn, op, dtype, plan, ws_ptr, ws_bytes,
                          stream) -> int:
    return lib().iwpp_reconstruct_plan(marker_ptr, mask_ptr, H, W, conn, op, dtype,
                                       ctypes.byref(plan) if plan is not None else None, ws_ptr,
                                       ws_bytes, stream)


def iwpp_scan(marker_ptr, mask_ptr, H, W, conn, op, dtype, plan, ws_ptr, ws_bytes, stream) -> int:
    return lib().iwpp_scan(marker_ptr, mask_ptr, H, W, conn, op, dtype,
                           ctypes.byref(plan) if plan is not None else None, ws_ptr, ws_bytes, stream)


def iwpp_drain(marker_ptr, mask_ptr, H, W, conn, op, dtype, plan, ws_ptr, ws_bytes, stream) -> int:
    return lib().iwpp_drain(marker_ptr, mask_ptr, H, W, conn, op, dtype,
                            ctypes.byref(plan) if plan is not None else None, ws_ptr, ws_bytes, stream)


def _pp(plan):
    return ctypes.byref(plan) if plan is not None else None


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def iwpp_batch_tile_count(imgs, plan: Plan | None = None) -> int:
    return int(lib().iwpp_batch_tile_count(imgs, len(imgs), _pp(plan)))


def iwpp_batch_workspace_bytes(imgs, plan: Plan | None = None) -> int:
    return int(lib().iwpp_batch_workspace_bytes(imgs, len(imgs), _pp(plan)))


def iwpp_reconstruct_batch(imgs, plan, ws_ptr, ws_bytes, stream) -> int:
    return lib().iwpp_reconstruct_batch(imgs, len(imgs), _pp(plan), ws_ptr, ws_bytes, stream)


def iwpp_reconstruct_batch_sched(imgs, plan, order_ptr, sweeps_ptr, work_ptr, ws_ptr, ws_bytes, stream) -> int:
    return lib().iwpp_reconstruct_batch_sched(imgs, len(imgs), _pp(plan), order_ptr, sweeps_ptr, work_ptr,
                                              ws_ptr, ws_bytes, stream)


def iwpp_reconstruct_batch_phase(imgs, plan, order_ptr, sweeps_ptr, work_ptr, phases, ws_ptr, ws_bytes,
                                 stream) -> int:
    return lib().iwpp_reconstruct_batch_phase(imgs, len(imgs), _pp(plan), order_ptr, sweeps_ptr, work_ptr,
                                              int(phases), ws_ptr, ws_bytes, stream)


def iwpp_batch_launch_count(n: int, phases: int = 3) -> int:
    return lib().iwpp_batch_launch_count(int(n), int(phases))


def iwpp_reconstruct_batch_learned(imgs, plan, params_ptr, order_ptr, sweeps_ptr, sws_ptr, sws_bytes, phases,
                                   ws_ptr, ws_bytes, stream) -> int:
    return lib().iwpp_reconstruct_batch_learned(imgs, len(imgs), _pp(plan), params_ptr, order_ptr, sweeps_ptr,
                                                sws_ptr, sws_bytes, int(phases), ws_ptr, ws_bytes, stream)


def iwpp_sched_features_offset(imgs, plan=None) -> int:
    return lib().iwpp_sched_features_offset(imgs, len(imgs), _pp(plan))


def iwpp_batch_graph_create(imgs, plan, order_ptr, sweeps_ptr, ws_ptr, ws_bytes):
    g = ctypes.c_void_p()
    rc = lib().iwpp_batch_graph_create(imgs, len(imgs), _pp(plan), order_ptr, sweeps_ptr, ws_ptr, ws_bytes,
                                       ctypes.byref(g))
    if rc != 0:
        raise IwppError(rc, "iwpp_batch_graph_create")
    return g


def iwpp_graph_launch(g, stream) -> int:
    return lib().iwpp_graph_launch(g, stream)


def iwpp_graph_destroy(g) -> int:
    return lib().iwpp_graph_destroy(g)


def iwpp_autotune_batch(imgs, plan: Plan, reps: int = 2, cache_path: str | None = None, stream=None):
    ms = ctypes.c_float(0)
    rc = lib().iwpp_autotune_batch(imgs, len(imgs), ctypes.byref(plan), int(reps),
                                   cache_path.encode() if cache_path else None, stream, ctypes.byref(ms))
    if rc != 0:
        raise IwppError(rc, "iwpp_autotune_batch")
    return plan, float(ms.value)


NFEAT = 16
MLP_PARAMS = 5378
FEATURE_BLOCK = 64


def _check(rc, what):
    if rc != 0:
        raise IwppError(rc, what)


def iwpp_batch_block_count(imgs) -> int:
    return int(lib().iwpp_batch_block_count(imgs, len(imgs)))


def iwpp_sched_workspace_bytes(imgs, plan=None) -> int:
    return int(lib().iwpp_sched_workspace_bytes(imgs, len(imgs), _pp(plan)))


def iwpp_batch_features(imgs, feats, sws, stream=None):
    _check(lib().iwpp_batch_features(imgs, len(imgs), _ptr(feats), _ptr(sws), sws.numel(), _stream_handle(stream)),
           "iwpp_batch_features")


def iwpp_mlp_forward(params, X, Y, stream=None):
    _check(lib().iwpp_mlp_forward(_ptr(params), _ptr(X), X.shape[0], _ptr(Y), _stream_handle(stream)),
           "iwpp_mlp_forward")


def iwpp_mlp_train(params, m, v, grad, X, T, epochs, batch, lr, w0=1.0, w1=1.0, seed=0, step0=0, stream=None):
    _check(lib().iwpp_mlp_train(_ptr(params), _ptr(m), _ptr(v), _ptr(grad), _ptr(X), _ptr(T), X.shape[0],
                                int(epochs), int(batch), float(lr), float(w0), float(w1), int(seed), int(step0),
                                _stream_handle(stream)), "iwpp_mlp_train")


def iwpp_schedule_from_predictions(imgs, plan, preds, order, sweeps, sws, stream=None):
    _check(lib().iwpp_schedule_from_predictions(imgs, len(imgs), _pp(plan), _ptr(preds), _ptr(order), _ptr(sweeps),
                                                _ptr(sws), sws.numel(), _stream_handle(stream)),
           "iwpp_schedule_from_predictions")


def iwpp_schedule_learned(imgs, plan, params, order, sweeps, sws, stream=None):
    _check(lib().iwpp_schedule_learned(imgs, len(imgs), _pp(plan), _ptr(params), _ptr(order), _ptr(sweeps),
                                       _ptr(sws), sws.numel(), _stream_handle(stream)), "iwpp_schedule_learned")


def iwpp_tile_work_to_blocks(imgs, plan, tile_work, block_work, sws, stream=None):
    _check(lib().iwpp_tile_work_to_blocks(imgs, len(imgs), _pp(plan), _ptr(tile_work), _ptr(block_work),
                                          _ptr(sws), sws.numel(), _stream_handle(stream)), "iwpp_tile_work_to_blocks")


def iwpp_reconstruct_noalloc(marker_ptr, mask_ptr, H, W, conn, op, dtype, stream, status=None) -> int:
    """C call without a caller workspace; `status` (a ctypes.c_int) receives the device status."""
    return lib().iwpp_reconstruct_noalloc(marker_ptr, mask_ptr, H, W, conn, op, dtype, stream,
                                          ctypes.byref(status) if status is not None else None)


def iwpp_sync_status(ws_ptr, stream) -> int:
    return lib().iwpp_sync_status(ws_ptr, stream)


def iwpp_hmaxima(image_ptr, out_ptr, H, W, h, conn, dtype, ws_ptr, ws_bytes, stream) -> int:
    return lib().iwpp_hmaxima(image_ptr, out_ptr, H, W, h, conn, dtype, ws_ptr, ws_bytes, stream)


def iwpp_hdome(image_ptr, out_ptr, H, W, h, conn, dtype, ws_ptr, ws_bytes, stream) -> int:
    return lib().iwpp_hdome(image_ptr, out_ptr, H, W, h, conn, dtype, ws_ptr, ws_bytes, stream)


def iwpp_regional_maxima(image_ptr, scratch_ptr, out_ptr, H, W, conn, dtype, ws_ptr, ws_bytes, stream) -> int:
    return lib().iwpp_regional_maxima(image_ptr, scratch_ptr, out_ptr, H, W, conn, dtype, ws_ptr, ws_bytes, stream)


def _op_ws(image):
    return alloc_workspace(iwpp_workspace_bytes(image.shape[0], image.shape[1], _dtype_code(image)), image.device)


def hmaxima(image, h: int, conn: int = 8, stream=None):
    """h-maxima transform of a CUDA uint8/uint16 image (a new tensor)."""
    import torch
    out = torch.empty_like(image)
    ws = _op_ws(image)
    _check(iwpp_hmaxima(ctypes.c_void_p(image.data_ptr()), ctypes.c_void_p(out.data_ptr()), image.shape[0],
                        image.shape[1], int(h), int(conn), _dtype_code(image), ctypes.c_void_p(ws.data_ptr()),
                        ws.numel(), _stream_handle(stream)), "iwpp_hmaxima")
    _check(iwpp_sync_status(ctypes.c_void_p(ws.data_ptr()), _stream_handle(stream)), "device")
    return out


def hdome(image, h: int, conn: int = 8, stream=None):
    """h-dome transform: image - hmaxima(image, h) (a new tensor)."""
    import torch
    out = torch.empty_like(image)
    ws = _op_ws(image)
    _check(iwpp_hdome(ctypes.c_void_p(image.data_ptr()), ctypes.c_void_p(out.data_ptr()), image.shape[0],
                      image.shape[1], int(h), int(conn), _dtype_code(image), ctypes.c_void_p(ws.data_ptr()),
                      ws.numel(), _stream_handle(stream)), "iwpp_hdome")
    _check(iwpp_sync_status(ctypes.c_void_p(ws.data_ptr()), _stream_handle(stream)), "device")
    return out


def regional_maxima(image, conn: int = 8, stream=None):
    """uint8 mask of the regional maxima of a CUDA uint8/uint16 image."""
    import torch
    scratch = torch.empty_like(image)
    out = torch.empty(image.shape, dtype=torch.uint8, device=image.device)
    ws = _op_ws(image)
    _check(iwpp_regional_maxima(ctypes.c_void_p(image.data_ptr()), ctypes.c_void_p(scratch.data_ptr()),
                                ctypes.c_void_p(out.data_ptr()), image.shape[0], image.shape[1], int(conn),
                                _dtype_code(image), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                _stream_handle(stream)), "iwpp_regional_maxima")
    _check(iwpp_sync_status(ctypes.c_void_p(ws.data_ptr()), _stream_handle(stream)), "device")
    return out


def iwpp_watershed_workspace_bytes(H: int, W: int) -> int:
    return int(lib().iwpp_watershed_workspace_bytes(H, W))


def iwpp_watershed(markers_ptr, grad_ptr, dtype, labels_ptr, levels_ptr, H, W, conn, ws_ptr, ws_bytes,
                   stream) -> int:
    return lib().iwpp_watershed(markers_ptr, grad_ptr, dtype, labels_ptr, levels_ptr, H, W, conn, ws_ptr, ws_bytes,
                                stream)


def watershed(markers, gradient, conn: int = 8, with_levels: bool = False, stream=None):
    """Marker-controlled watershed by flooding: markers (CUDA int32/uint32 labels, 0 =
    none) over a CUDA uint8/uint16 gradient. Returns the labels (int32), and the flooding
    levels too when asked."""
    import torch
    if markers.shape != gradient.shape:
        raise ValueError("shape mismatch")
    H, W = gradient.shape
    labels = torch.empty((H, W), dtype=torch.int32, device=gradient.device)
    levels = torch.empty((H, W), dtype=torch.int32, device=gradient.device) if with_levels else None
    ws = alloc_workspace(iwpp_watershed_workspace_bytes(H, W), gradient.device)
    mk = markers.contiguous()
    _check(iwpp_watershed(ctypes.c_void_p(mk.data_ptr()), ctypes.c_void_p(gradient.data_ptr()),
                          _dtype_code(gradient), ctypes.c_void_p(labels.data_ptr()),
                          ctypes.c_void_p(levels.data_ptr()) if levels is not None else None, H, W, int(conn),
                          ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_handle(stream)), "iwpp_watershed")
    _check(iwpp_sync_status(ctypes.c_void_p(ws.data_ptr()), _stream_handle(stream)), "device")
    return (labels, levels) if with_levels else labels


def iwpp_host_workspace_bytes(H: int, W: int, dtype: int, band_rows: int) -> int:
    return int(lib().iwpp_host_workspace_bytes(H, W, dtype, band_rows))


def iwpp_reconstruct_host(marker_ptr, mask_ptr, H, W, conn, op, dtype, band_rows, ws_ptr, ws_bytes, stream,
                          visits_ref=None) -> int:
    return lib().iwpp_reconstruct_host(marker_ptr, mask_ptr, H, W, conn, op, dtype, band_rows, ws_ptr, ws_bytes,
                                       stream, visits_ref)


class HostReconstructor:
    """Reconstruction of images in host memory, band by band (iwpp_reconstruct_host): holds
    the device workspace for H x W images of one dtype and band height."""

    def __init__(self, H: int, W: int, dtype, band_rows: int, device=None):
        import torch
        self.H, self.W, self.band_rows = int(H), int(W), int(band_rows)
        self.dtype_code = {torch.uint8: IWPP_U8, torch.uint16: IWPP_U16}[dtype]
        nbytes = iwpp_host_workspace_bytes(self.H, self.W, self.dtype_code, self.band_rows)
        if nbytes == 0:
            raise ValueError("unsupported size or band height")
        self.ws = alloc_workspace(nbytes, device)
        self.band_visits = 0

    def __call__(self, marker, mask, conn: int = 8, op: str = "dilate", stream=None) -> int:
        """marker, mask: contiguous CPU tensors (pinned for speed); marker is overwritten.
        Returns the status (0 = IWPP_OK)."""
        if marker.is_cuda or mask.is_cuda or not marker.is_contiguous() or not mask.is_contiguous():
            raise ValueError("contiguous host tensors expected")
        r = ctypes.c_int32(0)
        rc = iwpp_reconstruct_host(ctypes.c_void_p(marker.data_ptr()), ctypes.c_void_p(mask.data_ptr()), self.H,
                                   self.W, int(conn), OPS[op], self.dtype_code, self.band_rows,
                                   ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(), _stream_handle(stream),
                                   ctypes.byref(r))
        self.band_visits = int(r.value)
        return rc


def iwpp_skiz_workspace_bytes(H: int, W: int) -> int:
    return int(lib().iwpp_skiz_workspace_bytes(H, W))


def iwpp_skiz(markers_ptr, mask_ptr, zone_ptr, dist_ptr, lpair_ptr, H, W, conn, ws_ptr, ws_bytes, stream) -> int:
    return lib().iwpp_skiz(markers_ptr, mask_ptr, zone_ptr, dist_ptr, lpair_ptr, H, W, conn, ws_ptr, ws_bytes,
                           stream)


def skiz(markers, mask, conn: int = 8, with_details: bool = False, stream=None):
    """Geodesic influence zones of labelled markers (CUDA int32/uint32, 0 = none) inside the
    domain mask != 0 (CUDA uint8) or marker != 0. Returns the zone labels (int32; 0 on the
    skeleton and where unreached); with `with_details`, also the distances (int32, -1 where
    unreached) and the label pairs (min << 16 | max, int32)."""
    import torch
    if markers.shape != mask.shape or mask.dtype != torch.uint8:
        raise ValueError("markers and a uint8 mask of the same shape")
    H, W = mask.shape
    dev = mask.device
    zone = torch.empty((H, W), dtype=torch.int32, device=dev)
    dist = torch.empty((H, W), dtype=torch.int32, device=dev) if with_details else None
    lpair = torch.empty((H, W), dtype=torch.int32, device=dev) if with_details else None
    ws = alloc_workspace(iwpp_skiz_workspace_bytes(H, W), dev)
    mk, m = markers.contiguous(), mask.contiguous()
    P = ctypes.c_void_p
    _check(iwpp_skiz(P(mk.data_ptr()), P(m.data_ptr()), P(zone.data_ptr()),
                     P(dist.data_ptr()) if dist is not None else None,
                     P(lpair.data_ptr()) if lpair is not None else None, H, W, int(conn),
                     P(ws.data_ptr()), ws.numel(), _stream_handle(stream)), "iwpp_skiz")
    _check(iwpp_sync_status(P(ws.data_ptr()), _stream_handle(stream)), "device")
    return (zone, dist, lpair) if with_details else zone


def iwpp_edt_workspace_bytes(H: int, W: int) -> int:
    return int(lib().iwpp_edt_workspace_bytes(H, W))


def iwpp_edt(mask_ptr, site_ptr, dist2_ptr, H, W, conn, ws_ptr, ws_bytes, stream) -> int:
    return lib().iwpp_edt(mask_ptr, site_ptr, dist2_ptr, H, W, conn, ws_ptr, ws_bytes, stream)


class DistanceTransform:
    """Reusable distance transform (Algorithm 8) for H x W masks: holds the workspace.
    Call with a CUDA uint8 mask (non-zero = foreground) and int32 tensors for the sites
    (packed (y << 16) | x, -1 = none) and, optionally, the squared distances."""

    def __init__(self, H: int, W: int, device=None):
        import torch
        self.H, self.W = int(H), int(W)
        n = iwpp_edt_workspace_bytes(self.H, self.W)
        if n == 0:
            raise ValueError("image size not supported (1 .. 32767 per side)")
        self.ws = alloc_workspace(n, device or torch.device("cuda"))

    def __call__(self, mask, site, dist2=None, conn: int = 8, stream=None) -> int:
        for t in (mask, site) + ((dist2,) if dist2 is not None else ()):
            if tuple(t.shape) != (self.H, self.W) or not t.is_contiguous():
                raise ValueError("shape mismatch or non-contiguous tensor")
        return iwpp_edt(ctypes.c_void_p(mask.data_ptr()), ctypes.c_void_p(site.data_ptr()),
                        ctypes.c_void_p(dist2.data_ptr()) if dist2 is not None else None, self.H, self.W,
                        int(conn), ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(), _stream_handle(stream))

    def status(self, stream=None) -> int:
        return iwpp_sync_status(ctypes.c_void_p(self.ws.data_ptr()), _stream_handle(stream))

    def counters(self, stream=None):
        return iwpp_work_counters(ctypes.c_void_p(self.ws.data_ptr()), _stream_handle(stream))


def iwpp_work_counters(ws_ptr, stream):
    out = (ctypes.c_uint64 * 6)()
    rc = lib().iwpp_work_counters(ws_ptr, stream, out)
    if rc != 0:
        raise IwppError(rc, "iwpp_work_counters")
    return {"visits": int(out[0]), "pops": int(out[1]), "seeds": int(out[2]), "waves": int(out[3]),
            "idle_ns": int(out[4]), "busy_ns": int(out[5])}


# ---- torch convenience layer -----------------------------------------------------------

def _dtype_code(t):
    import torch
    if t.dtype == torch.uint8:
        return IWPP_U8
    if t.dtype == torch.uint16:
        return IWPP_U16
    raise TypeError("images must be torch.uint8 or torch.uint16")


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def alloc_workspace(nbytes: int, device=None):
    import torch
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device or "cuda")


class Reconstructor:
    """Reusable single-image reconstruction: holds a workspace sized for (H, W, dtype)."""

    def __init__(self, H: int, W: int, dtype, plan: Plan | None = None, device=None):
        import torch
        self.H, self.W = int(H), int(W)
        self.dtype_code = IWPP_U8 if dtype == torch.uint8 else IWPP_U16
        self.plan = plan
        nbytes = iwpp_workspace_bytes(self.H, self.W, self.dtype_code, plan)
        if nbytes == 0:
            raise IwppError(1, "iwpp_workspace_bytes")
        self.ws = alloc_workspace(nbytes, device)

    def __call__(self, marker, mask, conn: int = 8, op: str = "dilate", stream=None) -> int:
        """Enqueue the reconstruction (in place on ``marker``); returns the host status."""
        if marker.shape != (self.H, self.W) or mask.shape != (self.H, self.W):
            raise ValueError("shape mismatch")
        if _dtype_code(marker) != self.dtype_code or mask.dtype != marker.dtype:
            raise TypeError("dtype mismatch")
        if not (marker.is_cuda and mask.is_cuda and marker.is_contiguous() and mask.is_contiguous()):
            raise ValueError("marker and mask must be contiguous CUDA tensors")
        return iwpp_reconstruct_plan(ctypes.c_void_p(marker.data_ptr()), ctypes.c_void_p(mask.data_ptr()),
                                     self.H, self.W, int(conn), OPS[op], self.dtype_code, self.plan,
                                     ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(),
                                     _stream_handle(stream))

    def phase(self, which: str, marker, mask, conn: int = 8, op: str = "dilate", stream=None) -> int:
        """Enqueue one step of the call: which = "scan" or "drain"."""
        fn = iwpp_scan if which == "scan" else iwpp_drain
        return fn(ctypes.c_void_p(marker.data_ptr()), ctypes.c_void_p(mask.data_ptr()), self.H, self.W,
                  int(conn), OPS[op], self.dtype_code, self.plan, ctypes.c_void_p(self.ws.data_ptr()),
                  self.ws.numel(), _stream_handle(stream))

    def status(self, stream=None) -> int:
        return iwpp_sync_status(ctypes.c_void_p(self.ws.data_ptr()), _stream_handle(stream))

    def counters(self, stream=None):
        return iwpp_work_counters(ctypes.c_void_p(self.ws.data_ptr()), _stream_handle(stream))


def reconstruct(marker, mask, conn: int = 8, op: str = "dilate", plan: Plan | None = None, stream=None):
    """Reconstruct ``mask`` from ``marker`` in place on ``marker`` (torch CUDA tensors,
    uint8 or uint16, contiguous 2-D). Waits for the result and raises IwppError on
    any host- or device-side error. Returns ``marker``."""
    R = Reconstructor(marker.shape[0], marker.shape[1], marker.dtype, plan, marker.device)
    rc = R(marker, mask, conn, op, stream)
    if rc != 0:
        raise IwppError(rc, "iwpp_reconstruct")
    st = R.status(stream)
    if st != 0:
        raise IwppError(st, "device status")
    return marker


class Batch:
    """A fixed batch of (marker, mask, conn, op) torch CUDA tensors reconstructed in one
    persistent launch; holds the descriptor array and a workspace sized for it."""

    def __init__(self, items, plan: Plan | None = None, device=None):
        self.items = list(items)
        self.plan = plan
        n = len(self.items)
        self.descs = (Image * n)()
        for i, (m, I, conn, op) in enumerate(self.items):
            if m.shape != I.shape or m.dim() != 2 or m.dtype != I.dtype:
                raise ValueError(f"image {i}: marker and mask must be equal 2-D tensors")
            if not (m.is_cuda and I.is_cuda and m.is_contiguous() and I.is_contiguous()):
                raise ValueError(f"image {i}: contiguous CUDA tensors required")
            self.descs[i] = Image(m.data_ptr(), I.data_ptr(), m.shape[0], m.shape[1], int(conn), OPS[op],
                                  _dtype_code(m), 0)
        self.ntiles = iwpp_batch_tile_count(self.descs, plan)
        if self.ntiles < 1:
            raise IwppError(1, "iwpp_batch_tile_count")
        nbytes = iwpp_batch_workspace_bytes(self.descs, plan)
        if nbytes == 0:
            raise IwppError(1, "iwpp_batch_workspace_bytes")
        self.ws = alloc_workspace(nbytes, device or self.items[0][0].device)

    @property
    def pixels(self) -> int:
        return sum(int(m.numel()) for m, _, _, _ in self.items)

    def __call__(self, order=None, sweeps=None, work=None, stream=None) -> int:
        """Enqueue the batch; order (int32/uint32 [ntiles]), sweeps (uint8 [ntiles]) and work
        (int32 [2*ntiles], zeroed) are optional CUDA tensors. Returns the host status."""
        ws = ctypes.c_void_p(self.ws.data_ptr())
        if order is None and sweeps is None and work is None:
            return iwpp_reconstruct_batch(self.descs, self.plan, ws, self.ws.numel(), _stream_handle(stream))
        return iwpp_reconstruct_batch_sched(self.descs, self.plan, _ptr(order), _ptr(sweeps), _ptr(work), ws,
                                            self.ws.numel(), _stream_handle(stream))

    def phase(self, which: str, order=None, sweeps=None, work=None, stream=None) -> int:
        """Enqueue one step of the batch call: which = "scan" (table upload, reset, scan,
        queue compaction) or "drain" (the persistent kernel)."""
        phases = {"scan": 1, "drain": 2, "all": 3}[which]
        return iwpp_reconstruct_batch_phase(self.descs, self.plan, _ptr(order), _ptr(sweeps), _ptr(work), phases,
                                            ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(),
                                            _stream_handle(stream))

    def status(self, stream=None) -> int:
        return iwpp_sync_status(ctypes.c_void_p(self.ws.data_ptr()), _stream_handle(stream))

    def counters(self, stream=None):
        return iwpp_work_counters(ctypes.c_void_p(self.ws.data_ptr()), _stream_handle(stream))

    def graph(self, order=None, sweeps=None) -> "Graph":
        """Capture this batch (with an optional device schedule) into a CUDA graph."""
        g = iwpp_batch_graph_create(self.descs, self.plan, _ptr(order), _ptr(sweeps),
                                    ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel())
        return Graph(g, (order, sweeps))

    def autotune(self, reps: int = 2, cache_path: str | None = None, stream=None):
        """Pick this batch's plan with the library's autotuner (markers are restored). The
        workspace is re-sized for the chosen plan."""
        plan = Plan.from_buffer_copy(self.plan) if self.plan is not None else iwpp_default_batch_plan()
        plan, ms = iwpp_autotune_batch(self.descs, plan, reps, cache_path, _stream_handle(stream))
        self.plan = plan
        self.ntiles = iwpp_batch_tile_count(self.descs, plan)
        nbytes = iwpp_batch_workspace_bytes(self.descs, plan)
        if nbytes > self.ws.numel():
            self.ws = alloc_workspace(nbytes, self.ws.device)
        return plan, ms


class Graph:
    """An executable CUDA graph of one batch call (see iwpp_batch_graph_create)."""

    def __init__(self, handle, keepalive):
        self.handle = handle
        self._keep = keepalive

    def launch(self, stream=None) -> int:
        return iwpp_graph_launch(self.handle, _stream_handle(stream))

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                iwpp_graph_destroy(self.handle)
            except Exception:
                pass
            self.handle = None
