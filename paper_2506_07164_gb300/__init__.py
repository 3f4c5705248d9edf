"""Python binding of the GB300 Oriented FAST library (include/ofast.h).

Argument marshalling only: every step of the detection chain runs in the CUDA
kernels of ``csrc/``.  Functions carry the C names (``of_create``,
``of_detect``, ``of_detect_batch``, ``of_destroy``, ``of_inspect``,
``of_plan_levels``, ``of_last_error``, ``of_version``); device buffers are
passed as torch CUDA tensors (or raw integer device addresses), host arrays
as numpy arrays.  PyTorch provides device memory and streams, nothing else.

The shared library is built in-tree by ``build.py``.  Loading fails loudly
when it is missing: there is no CPU fallback.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from .build import LIB, build  # noqa: F401

__all__ = ["of_create", "of_destroy", "of_detect", "of_detect_batch", "of_inspect", "of_plan_levels",
           "of_time_stages", "OF_N_STAGES", "STAGE_NAMES", "of_detect_level_noalloc", "of_probe_read", "of_sync",
           "of_test_timeout", "OF_ERR_TIMEOUT", "of_autotune", "of_variant_detect", "OfVarPoint",
           "VAR_POINT_DTYPE", "of_set_tuning", "OfTuning", "of_batch_bytes",
           "of_server_create", "of_server_destroy", "of_server_submit", "of_server_poll", "of_server_stats",
           "OfServerParams", "OfServerResult", "of_tcnn_create", "of_tcnn_destroy", "of_tcnn_num_params",
           "of_tcnn_set_params", "of_tcnn_get_params", "of_tcnn_forward", "of_tcnn_loss_grad", "of_tcnn_adam",
           "of_tcnn_save", "of_tcnn_load", "of_detect_learned", "of_extract_tiles",
           "of_last_error", "of_version", "OfParams", "OfFrame", "OfKeypoint", "KEYPOINT_DTYPE",
           "OF_BUF_LEVEL", "OF_BUF_SCORE", "OF_BUF_CELLT", "OF_BUF_CAND", "OF_BUF_PMASK", "OF_BUF_LOGIT", "OfError", "load",
           "Detector", "keypoints_to_numpy"]

OF_OK, OF_ERR_ARG, OF_ERR_TOO_LARGE, OF_ERR_CUDA, OF_ERR_TIMEOUT, OF_ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5
OF_BUF_LEVEL, OF_BUF_SCORE, OF_BUF_CELLT, OF_BUF_CAND, OF_BUF_PMASK, OF_BUF_LOGIT = 0, 1, 2, 3, 4, 5


class OfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ofast error {code}: {msg}")
        self.code = code


class OfParams(C.Structure):
    _fields_ = [("max_w", C.c_int32), ("max_h", C.c_int32), ("max_levels", C.c_int32),
                ("max_features", C.c_int32), ("max_batch", C.c_int32), ("min_scale", C.c_float),
                ("fast_t_lo", C.c_int32), ("cell", C.c_int32), ("border", C.c_int32),
                ("harris_block", C.c_int32), ("orient_radius", C.c_int32), ("stream", C.c_void_p),
                ("autotune", C.c_int32), ("arena_bytes", C.c_int64)]


class OfTuning(C.Structure):
    """of_tuning: launch configuration of one batch shape.

    resize_tile_h (32/64) and resize_tma (0/1): pyramid kernel; fast_blocks_per_sm,
    nms_blocks_per_sm, fast_order, nms_order: persistent grids and tile order;
    stream_groups (1..8): frame groups on forked graph branches; fast_cell_tiles:
    0 general FAST + threshold pass, 1 cell-tile kernel, 2 cell-aligned general kernel,
    3 general FAST with per-warp pipelines + threshold pass, 4 the same on cell-row strips
    that also set the cell flags + the pass applying them (with nms_tile_h 32 the per-warp
    NMS kernel applies the flags itself and the pass only sets flags FAST leaves unset);
    fast_tile_h (32/64/128/256) and nms_tile_h (32/64/128): tile heights.  The last
    four fields report the autotuner's search (candidates, best stage times in ms)."""

    _fields_ = [("resize_tile_h", C.c_int32), ("fast_blocks_per_sm", C.c_int32),
                ("nms_blocks_per_sm", C.c_int32), ("fast_order", C.c_int32), ("nms_order", C.c_int32),
                ("resize_tma", C.c_int32), ("stream_groups", C.c_int32), ("fast_cell_tiles", C.c_int32),
                ("nms_tile_h", C.c_int32), ("fast_tile_h", C.c_int32),
                ("candidates_tried", C.c_int32), ("resize_ms", C.c_float), ("fast_ms", C.c_float),
                ("nms_ms", C.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class OfKeypoint(C.Structure):
    _fields_ = [("x", C.c_float), ("y", C.c_float), ("x_l", C.c_int32), ("y_l", C.c_int32),
                ("level", C.c_int32), ("fast_score", C.c_int32), ("response", C.c_float),
                ("angle", C.c_float), ("A", C.c_int32), ("B", C.c_int32), ("C", C.c_int32),
                ("m10", C.c_int32), ("m01", C.c_int32), ("reserved", C.c_int32), ("key", C.c_int64)]


class OfFrame(C.Structure):
    _fields_ = [("img", C.c_void_p), ("w", C.c_int32), ("h", C.c_int32), ("pitch", C.c_int32)]


class OfServerParams(C.Structure):
    _fields_ = [("max_w", C.c_int32), ("max_h", C.c_int32), ("levels", C.c_int32), ("scale", C.c_float),
                ("fast_t", C.c_int32), ("fast_t_lo", C.c_int32), ("harris_k", C.c_float),
                ("n_features", C.c_int32), ("slots", C.c_int32), ("max_batch", C.c_int32),
                ("memory_budget", C.c_int64), ("border", C.c_int32), ("cell", C.c_int32),
                ("orient_radius", C.c_int32)]


class OfServerResult(C.Structure):
    _fields_ = [("id", C.c_int64), ("tag", C.c_int64), ("w", C.c_int32), ("h", C.c_int32),
                ("count", C.c_int32), ("batch_frames", C.c_int32), ("t_submit", C.c_double),
                ("t_launch", C.c_double), ("t_done", C.c_double)]


class OfServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("queued", C.c_int64),
                ("batches", C.c_int64), ("frames_launched", C.c_int64), ("in_flight_batches", C.c_int64),
                ("slot_arena_bytes", C.c_int64), ("slot_input_bytes", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class OfVarPoint(C.Structure):
    _fields_ = [("x", C.c_int32), ("y", C.c_int32), ("A", C.c_int32), ("B", C.c_int32), ("C", C.c_int32),
                ("reserved", C.c_int32), ("key", C.c_int64)]


VAR_POINT_DTYPE = np.dtype([("x", "i4"), ("y", "i4"), ("A", "i4"), ("B", "i4"), ("C", "i4"), ("reserved", "i4"),
                            ("key", "i8")])
assert VAR_POINT_DTYPE.itemsize == C.sizeof(OfVarPoint) == 32
OF_VAR_FAST_BASELINE, OF_VAR_FAST_BINARY, OF_VAR_FAST_SM, OF_VAR_FAST_SM_BINARY = 0, 1, 2, 3
OF_VAR_HARRIS_NONE, OF_VAR_HARRIS_BASELINE, OF_VAR_HARRIS_SEP, OF_VAR_HARRIS_PARA_SEP, OF_VAR_HARRIS_SEMI_SEP = \
    -1, 0, 1, 2, 3

KEYPOINT_DTYPE = np.dtype([("x", "f4"), ("y", "f4"), ("x_l", "i4"), ("y_l", "i4"), ("level", "i4"),
                           ("fast_score", "i4"), ("response", "f4"), ("angle", "f4"), ("A", "i4"),
                           ("B", "i4"), ("C", "i4"), ("m10", "i4"), ("m01", "i4"),
                           ("reserved", "i4"), ("key", "i8")])
assert KEYPOINT_DTYPE.itemsize == C.sizeof(OfKeypoint) == 64

_lib = None


def load(path: str | None = None):
    """Load the CUDA library (must have been built by ``build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise OfError(OF_ERR_UNSUPPORTED, f"CUDA library not built: {path} (run paper_2506_07164_gb300.build())")
    L = C.CDLL(path)
    L.of_create.argtypes = [C.POINTER(OfParams)]
    L.of_create.restype = C.c_void_p
    L.of_destroy.argtypes = [C.c_void_p]
    L.of_destroy.restype = None
    L.of_detect.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float,
                            C.c_int, C.c_float, C.c_int, C.c_void_p]
    L.of_detect.restype = C.c_int
    L.of_detect_batch.argtypes = [C.c_void_p, C.POINTER(OfFrame), C.c_int, C.c_int, C.c_float, C.c_int,
                                  C.c_float, C.c_int, C.c_void_p, C.c_void_p]
    L.of_detect_batch.restype = C.c_int
    L.of_inspect.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int64,
                             C.POINTER(C.c_int32)]
    L.of_inspect.restype = C.c_int64
    L.of_plan_levels.argtypes = [C.c_int, C.c_int, C.c_int, C.c_float, C.c_int, C.POINTER(C.c_int32),
                                 C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    L.of_plan_levels.restype = C.c_int
    L.of_last_error.argtypes = []
    L.of_last_error.restype = C.c_char_p
    L.of_version.argtypes = []
    L.of_version.restype = C.c_int
    L.of_time_stages.argtypes = [C.c_void_p, C.POINTER(C.c_void_p)]
    L.of_time_stages.restype = C.c_int
    L.of_detect_level_noalloc.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                          C.c_float, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
    L.of_detect_level_noalloc.restype = C.c_int
    L.of_probe_read.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_void_p]
    L.of_probe_read.restype = C.c_int
    L.of_variant_detect.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                    C.c_float, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]
    L.of_variant_detect.restype = C.c_int
    L.of_autotune.argtypes = [C.c_void_p, C.POINTER(OfFrame), C.c_int, C.c_int, C.c_float, C.c_int, C.c_float,
                              C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(OfTuning)]
    L.of_autotune.restype = C.c_int
    L.of_set_tuning.argtypes = [C.c_void_p, C.POINTER(OfFrame), C.c_int, C.c_int, C.c_float, C.c_int, C.c_float,
                                C.c_int, C.c_void_p, C.c_void_p, C.POINTER(OfTuning)]
    L.of_set_tuning.restype = C.c_int
    L.of_server_create.argtypes = [C.POINTER(OfServerParams)]
    L.of_server_create.restype = C.c_void_p
    L.of_server_destroy.argtypes = [C.c_void_p]
    L.of_server_destroy.restype = None
    L.of_server_submit.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int64]
    L.of_server_submit.restype = C.c_int64
    L.of_server_poll.argtypes = [C.c_void_p, C.POINTER(OfServerResult), C.c_void_p, C.c_int, C.c_int]
    L.of_server_poll.restype = C.c_int
    L.of_server_stats_get.argtypes = [C.c_void_p, C.POINTER(OfServerStats)]
    L.of_server_stats_get.restype = C.c_int
    L.of_batch_bytes.argtypes = [C.POINTER(OfParams), C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_int, C.c_int,
                                 C.c_float, C.c_int]
    L.of_batch_bytes.restype = C.c_int64
    L.of_tcnn_create.argtypes = [C.c_uint64]
    L.of_tcnn_create.restype = C.c_void_p
    L.of_tcnn_destroy.argtypes = [C.c_void_p]
    L.of_tcnn_destroy.restype = None
    L.of_tcnn_num_params.argtypes = []
    L.of_tcnn_num_params.restype = C.c_int
    L.of_tcnn_set_params.argtypes = [C.c_void_p, C.c_void_p]
    L.of_tcnn_set_params.restype = C.c_int
    L.of_tcnn_get_params.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
    L.of_tcnn_get_params.restype = C.c_int
    L.of_tcnn_forward.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
    L.of_tcnn_forward.restype = C.c_int
    L.of_tcnn_loss_grad.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_float,
                                    C.POINTER(C.c_float), C.c_void_p]
    L.of_tcnn_loss_grad.restype = C.c_int
    L.of_tcnn_adam.argtypes = [C.c_void_p, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float, C.c_void_p]
    L.of_tcnn_adam.restype = C.c_int
    L.of_tcnn_save.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
    L.of_tcnn_save.restype = C.c_int64
    L.of_tcnn_load.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
    L.of_tcnn_load.restype = C.c_int
    L.of_detect_learned.argtypes = [C.c_void_p, C.POINTER(OfFrame), C.c_int, C.c_int, C.c_float, C.c_int,
                                    C.c_float, C.c_int, C.c_void_p, C.c_float, C.c_float, C.c_int, C.c_void_p,
                                    C.c_void_p, C.POINTER(C.c_int32)]
    L.of_detect_learned.restype = C.c_int
    L.of_extract_tiles.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int64, C.POINTER(C.c_int32)]
    L.of_extract_tiles.restype = C.c_int
    L.of_sync.argtypes = [C.c_void_p]
    L.of_sync.restype = C.c_int
    L.of_test_timeout.argtypes = [C.c_void_p, C.c_int64]
    L.of_test_timeout.restype = C.c_int
    _lib = L
    return L


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _check(rc: int) -> int:
    if rc < 0:
        raise OfError(rc, of_last_error())
    return rc


def of_last_error() -> str:
    return load().of_last_error().decode()


def of_version() -> int:
    return int(load().of_version())


def of_create(params: OfParams | None = None, **kw) -> int:
    """Create a handle; ``kw`` fill an OfParams (``stream`` may be a torch.cuda.Stream)."""
    p = params or OfParams()
    for k, v in kw.items():
        if k == "stream" and v is not None and not isinstance(v, int):
            v = int(v.cuda_stream)
        setattr(p, k, v)
    h = load().of_create(C.byref(p))
    if not h:
        raise OfError(OF_ERR_ARG, of_last_error())
    return h


def of_destroy(h: int) -> None:
    load().of_destroy(h)


def of_detect(h: int, img, w: int, h_px: int, pitch: int, levels: int, scale: float, fast_t: int,
              harris_k: float, n_features: int, out_kpts) -> int:
    return _check(load().of_detect(h, _ptr(img), w, h_px, pitch, levels, scale, fast_t, harris_k,
                                   n_features, _ptr(out_kpts)))


def of_detect_batch(h: int, frames, levels: int, scale: float, fast_t: int, harris_k: float,
                    n_features: int, out_kpts, out_counts) -> int:
    """``frames``: sequence of (img, w, h, pitch) with img a device tensor or address."""
    arr = (OfFrame * len(frames))()
    for i, (img, w, hh, pitch) in enumerate(frames):
        arr[i] = OfFrame(_ptr(img), w, hh, pitch)
    return _check(load().of_detect_batch(h, arr, len(frames), levels, scale, fast_t, harris_k,
                                         n_features, _ptr(out_kpts), _ptr(out_counts)))


def of_inspect(h: int, what: int, frame: int, level: int, dst=None, dst_bytes: int = 0):
    """Returns (byte size, dims[4])."""
    dims = (C.c_int32 * 4)()
    n = _check(int(load().of_inspect(h, what, frame, level, _ptr(dst), dst_bytes, dims)))
    return n, list(dims)


OF_N_STAGES = 5
STAGE_NAMES = ("pyramid", "fast", "nms_harris", "select", "orient")


def of_time_stages(h: int, events) -> int:
    """Record 6 events around the 5 stages of the next detect call.

    ``events``: raw cudaEvent_t handles, or torch.cuda.Event(enable_timing=True)
    objects that have been recorded once (torch creates them lazily)."""
    hs = [e if isinstance(e, int) else int(e.cuda_event) for e in events]
    if len(hs) != OF_N_STAGES + 1:
        raise ValueError("need OF_N_STAGES + 1 events")
    arr = (C.c_void_p * len(hs))(*hs)
    return _check(load().of_time_stages(h, arr))


def of_detect_level_noalloc(img, w: int, h: int, pitch: int, fast_t: int, fast_t_lo: int,
                            harris_k: float, n_features: int, out_kpts, out_count, stream=None) -> int:
    """Single-level detect whose scratch is the library's static device array.

    For callers that cannot allocate device memory (graph capture, real-time
    loops, hosts that own all allocations).  Asynchronous on ``stream``."""
    s = None if stream is None else (stream if isinstance(stream, int) else int(stream.cuda_stream))
    return _check(load().of_detect_level_noalloc(_ptr(img), w, h, pitch, fast_t, fast_t_lo, harris_k,
                                                 n_features, _ptr(out_kpts), _ptr(out_count), s))


def of_probe_read(buf, nbytes: int, reps: int, sink, stream=None) -> None:
    """Read nbytes of a device buffer reps times (bandwidth probe; see include/ofast.h). Asynchronous."""
    s = None if stream is None else (stream if isinstance(stream, int) else int(stream.cuda_stream))
    _check(load().of_probe_read(_ptr(buf), nbytes, reps, _ptr(sink), s))


def of_variant_detect(fast_variant: int, harris_variant: int, img, w: int, h: int, pitch: int, fast_t: int,
                      border: int, harris_k: float, out_points, out_count, capacity: int, stream=None) -> None:
    """One of the paper's ablation variants (Table 2) on one level (see include/ofast.h). Asynchronous."""
    s = None if stream is None else (stream if isinstance(stream, int) else int(stream.cuda_stream))
    _check(load().of_variant_detect(fast_variant, harris_variant, _ptr(img), w, h, pitch, fast_t, border, harris_k,
                                    _ptr(out_points), _ptr(out_count), capacity, s))


def of_autotune(h: int, frames, levels: int, scale: float, fast_t: int, harris_k: float, n_features: int,
                out_kpts, out_counts, reps: int = 3) -> OfTuning:
    """Tune the launch configuration of this batch shape (see include/ofast.h); returns the choice."""
    arr = (OfFrame * len(frames))()
    for i, (img, w, hh, pitch) in enumerate(frames):
        arr[i] = OfFrame(_ptr(img), w, hh, pitch)
    t = OfTuning()
    _check(load().of_autotune(h, arr, len(frames), levels, scale, fast_t, harris_k, n_features, _ptr(out_kpts),
                              _ptr(out_counts), reps, C.byref(t)))
    return t


def of_set_tuning(h: int, frames, levels: int, scale: float, fast_t: int, harris_k: float, n_features: int,
                  out_kpts, out_counts, tuning: OfTuning) -> None:
    """Fix the launch configuration of this batch shape (see include/ofast.h)."""
    arr = (OfFrame * len(frames))()
    for i, (img, w, hh, pitch) in enumerate(frames):
        arr[i] = OfFrame(_ptr(img), w, hh, pitch)
    _check(load().of_set_tuning(h, arr, len(frames), levels, scale, fast_t, harris_k, n_features, _ptr(out_kpts),
                                _ptr(out_counts), C.byref(tuning)))


def of_batch_bytes(params: OfParams, sizes, levels: int, scale: float, n_features: int) -> int:
    """Scratch bytes for a batch of frames with the given (w, h) sizes (host-only)."""
    n = len(sizes)
    ws = (C.c_int32 * n)(*[w for w, _ in sizes])
    hs = (C.c_int32 * n)(*[h for _, h in sizes])
    return _check(int(load().of_batch_bytes(C.byref(params), ws, hs, n, levels, scale, n_features)))


# Records a server writes per polled result (its n_features; 1000 when left 0).
_server_features: dict = {}


def of_server_create(**kw) -> int:
    p = OfServerParams()
    for k, v in kw.items():
        setattr(p, k, v)
    s = load().of_server_create(C.byref(p))
    if not s:
        raise OfError(OF_ERR_ARG, of_last_error())
    _server_features[s] = p.n_features or 1000
    return s


def of_server_destroy(s: int) -> None:
    load().of_server_destroy(s)
    _server_features.pop(s, None)


def of_server_submit(s: int, img: np.ndarray, tag: int = 0) -> int:
    """img: 2-D uint8 numpy array (rows may be strided)."""
    assert img.dtype == np.uint8 and img.ndim == 2 and img.strides[1] == 1
    return _check(int(load().of_server_submit(s, img.ctypes.data, img.shape[1], img.shape[0], img.strides[0], tag)))


_poll_local = threading.local()


def of_server_poll(s: int, max_results: int, n_features: int, wait_ms: int = 0, keypoints: bool = True):
    """Returns a list of (OfServerResult, keypoints ndarray or None).  The
    keypoints land in a buffer the calling thread keeps per (max_results,
    n_features) and are copied out per result; keypoints=False returns the
    results only."""
    nf = _server_features.get(s)
    if keypoints and nf is not None and n_features != nf:
        # The server writes result i's records at i * its own n_features.
        raise ValueError(f"n_features {n_features} differs from the server's {nf}")
    res = (OfServerResult * max_results)()
    kp = None
    if keypoints:
        bufs = getattr(_poll_local, "bufs", None)
        if bufs is None:
            bufs = _poll_local.bufs = {}
        kp = bufs.get((max_results, n_features))
        if kp is None:
            kp = bufs[(max_results, n_features)] = np.empty(max_results * n_features, KEYPOINT_DTYPE)
    n = _check(load().of_server_poll(s, res, kp.ctypes.data if kp is not None else None, max_results, wait_ms))
    out = []
    for i in range(n):
        c = res[i].count
        out.append((res[i], kp[i * n_features: i * n_features + max(c, 0)].copy() if kp is not None else None))
    return out


def of_server_stats(s: int) -> dict:
    st = OfServerStats()
    _check(load().of_server_stats_get(s, C.byref(st)))
    return st.as_dict()


# ------------------------------------------------------------ tile-proposal network
def _sp(stream):
    return None if stream is None else (stream if isinstance(stream, int) else int(stream.cuda_stream))


def of_tcnn_create(seed: int = 0) -> int:
    n = load().of_tcnn_create(seed)
    if not n:
        raise OfError(OF_ERR_CUDA, of_last_error())
    return n


def of_tcnn_destroy(net: int) -> None:
    load().of_tcnn_destroy(net)


def of_tcnn_num_params() -> int:
    return int(load().of_tcnn_num_params())


def of_tcnn_set_params(net: int, params: np.ndarray) -> None:
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert p.size == of_tcnn_num_params()
    _check(load().of_tcnn_set_params(net, p.ctypes.data))


def of_tcnn_get_params(net: int, which: int = 0) -> np.ndarray:
    out = np.zeros(of_tcnn_num_params(), np.float32)
    _check(load().of_tcnn_get_params(net, which, out.ctypes.data))
    return out


def of_tcnn_forward(net: int, tiles, n: int, logits, stream=None) -> None:
    _check(load().of_tcnn_forward(net, _ptr(tiles), n, _ptr(logits), _sp(stream)))


def of_tcnn_loss_grad(net: int, tiles, labels, n: int, pos_weight: float = 1.0, stream=None) -> float:
    loss = C.c_float()
    _check(load().of_tcnn_loss_grad(net, _ptr(tiles), _ptr(labels), n, pos_weight, C.byref(loss), _sp(stream)))
    return float(loss.value)


def of_tcnn_adam(net: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                 weight_decay: float = 0.0, stream=None) -> None:
    _check(load().of_tcnn_adam(net, lr, beta1, beta2, eps, weight_decay, _sp(stream)))


def of_tcnn_save(net: int) -> bytes:
    n = _check(int(load().of_tcnn_save(net, None, 0)))
    buf = (C.c_uint8 * n)()
    _check(int(load().of_tcnn_save(net, buf, n)))
    return bytes(buf)


def of_tcnn_load(net: int, data: bytes) -> None:
    buf = (C.c_uint8 * len(data)).from_buffer_copy(data)
    _check(load().of_tcnn_load(net, buf, len(data)))


def of_detect_learned(h: int, frames, levels: int, scale: float, fast_t: int, harris_k: float,
                      n_features: int, net: int, threshold: float, min_confidence: float, dilate: int,
                      out_kpts, out_counts, want_stats: bool = True):
    arr = (OfFrame * len(frames))()
    for i, (img, w, hh, pitch) in enumerate(frames):
        arr[i] = OfFrame(_ptr(img), w, hh, pitch)
    st = (C.c_int32 * 3)()
    _check(load().of_detect_learned(h, arr, len(frames), levels, scale, fast_t, harris_k, n_features, net,
                                    threshold, min_confidence, dilate, _ptr(out_kpts), _ptr(out_counts),
                                    st if want_stats else None))
    return {"tiles": st[0], "proposed": st[1], "fallback_images": st[2]} if want_stats else None


def of_extract_tiles(h: int, frame: int, level: int, dst=None, cap_tiles: int = 0):
    grid = (C.c_int32 * 2)()
    n = _check(load().of_extract_tiles(h, frame, level, _ptr(dst), cap_tiles, grid))
    return n, (grid[0], grid[1])


def of_sync(h: int) -> int:
    """Wait for the handle's work; raises OfError(OF_ERR_TIMEOUT) if a device wait expired."""
    return _check(load().of_sync(h))


def of_test_timeout(h: int, limit_us: int) -> int:
    """Run the bounded-wait failure path on the GPU; returns the raw code (OF_ERR_TIMEOUT expected)."""
    return int(load().of_test_timeout(h, limit_us))


def of_plan_levels(W: int, H: int, levels: int, scale: float, n_features: int):
    ws = (C.c_int32 * levels)()
    hs = (C.c_int32 * levels)()
    q = (C.c_int32 * levels)()
    rc = load().of_plan_levels(W, H, levels, scale, n_features, ws, hs, q)
    if rc != 0:
        raise OfError(rc, "bad plan arguments")
    return list(ws), list(hs), list(q)


def keypoints_to_numpy(t) -> np.ndarray:
    """A uint8 torch tensor holding of_keypoint records -> structured numpy array."""
    b = t.detach().to("cpu").contiguous().numpy().view(np.uint8).reshape(-1)
    return b.view(KEYPOINT_DTYPE)


class Detector:
    """Convenience owner of a handle and its output buffers (torch CUDA tensors)."""

    def __init__(self, max_w: int, max_h: int, max_levels: int = 8, max_features: int = 1000,
                 max_batch: int = 1, fast_t_lo: int = 0, min_scale: float = 1.2, border: int = 19,
                 cell: int = 30, orient_radius: int = 15, stream=None, device="cuda"):
        """stream: a torch.cuda.Stream (default: the current stream of `device`)."""
        import torch

        self.torch = torch
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            if stream is None:
                stream = torch.cuda.current_stream(self.device)
            self.stream = stream
            self.h = of_create(max_w=max_w, max_h=max_h, max_levels=max_levels,
                               max_features=max_features, max_batch=max_batch, fast_t_lo=fast_t_lo,
                               min_scale=min_scale, border=border, cell=cell,
                               orient_radius=orient_radius, stream=stream)
        self.max_features = max_features
        self.max_batch = max_batch
        self.out = torch.empty(max_batch * max(max_features, 1) * 64, dtype=torch.uint8, device=self.device)
        self.counts = torch.zeros(max_batch, dtype=torch.int32, device=self.device)

    def close(self):
        if self.h:
            of_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def detect(self, img, levels=8, scale=1.2, fast_t=20, harris_k=0.04, n_features=1000) -> np.ndarray:
        """One frame (2-D uint8 CUDA tensor, rows may be strided) -> numpy keypoints."""
        assert img.dtype == self.torch.uint8 and img.is_cuda and img.dim() == 2 and img.stride(1) == 1
        n = of_detect(self.h, img, img.shape[1], img.shape[0], img.stride(0), levels, scale, fast_t,
                      harris_k, n_features, self.out)
        return keypoints_to_numpy(self.out[: n * 64])

    def detect_batch(self, imgs, levels=8, scale=1.2, fast_t=20, harris_k=0.04, n_features=1000):
        """Queue a batch (list of 2-D uint8 CUDA tensors); returns (records tensor, counts tensor)."""
        frames = [(im, im.shape[1], im.shape[0], im.stride(0)) for im in imgs]
        of_detect_batch(self.h, frames, levels, scale, fast_t, harris_k, n_features, self.out, self.counts)
        return self.out, self.counts

    def autotune(self, imgs, levels=8, scale=1.2, fast_t=20, harris_k=0.04, n_features=1000, reps=3):
        """Tune this batch shape (a list of 2-D uint8 CUDA tensors); returns an OfTuning."""
        frames = [(im, im.shape[1], im.shape[0], im.stride(0)) for im in imgs]
        return of_autotune(self.h, frames, levels, scale, fast_t, harris_k, n_features, self.out, self.counts, reps)

    def set_tuning(self, imgs, tuning: OfTuning, levels=8, scale=1.2, fast_t=20, harris_k=0.04, n_features=1000):
        """Fix the launch configuration of this batch shape (a list of 2-D uint8 CUDA tensors)."""
        frames = [(im, im.shape[1], im.shape[0], im.stride(0)) for im in imgs]
        of_set_tuning(self.h, frames, levels, scale, fast_t, harris_k, n_features, self.out, self.counts, tuning)

    def batch_results(self, n_frames: int, n_features: int):
        """Per-frame numpy keypoints of the last batch (synchronises)."""
        recs = keypoints_to_numpy(self.out[: n_frames * n_features * 64])
        cnt = self.counts[:n_frames].cpu().numpy()
        return [recs[i * n_features: i * n_features + int(cnt[i])] for i in range(n_frames)]

    def inspect(self, what: int, frame: int = 0, level: int = 0):
        n, dims = of_inspect(self.h, what, frame, level)
        buf = self.torch.empty(max(n, 1), dtype=self.torch.uint8, device=self.device)
        n, dims = of_inspect(self.h, what, frame, level, buf, n)
        return buf[:n].cpu().numpy(), dims
