"""Plain CPU oracle for Oriented FAST over an image pyramid (arXiv 2506.07164).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use it; the product library never does.

The arithmetic lives in ``ofast_oracle.c`` (plain single-threaded C, float64
where floating point appears, built with ``-ffp-contract=off``).  This module
compiles it with gcc on first use and wraps each function for numpy arrays.
It shares no code with the CUDA path.

Every function here is pinned by ``tests/test_oracle_pins.py`` against brute
force, closed forms, the Fig. 6 cases and library routines.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ofast_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libofast_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc; returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Keypoint(C.Structure):
    _fields_ = [("x", C.c_double), ("y", C.c_double), ("x_l", C.c_int32), ("y_l", C.c_int32),
                ("level", C.c_int32), ("fast_score", C.c_int32), ("key", C.c_int64),
                ("response", C.c_double), ("angle", C.c_double), ("A", C.c_int32),
                ("B", C.c_int32), ("C", C.c_int32), ("m10", C.c_int32), ("m01", C.c_int32)]


class Config(C.Structure):
    _fields_ = [("border", C.c_int), ("cell", C.c_int), ("block", C.c_int), ("radius", C.c_int),
                ("t_hi", C.c_int), ("t_lo", C.c_int)]


KEYPOINT_DTYPE = np.dtype([("x", "f8"), ("y", "f8"), ("x_l", "i4"), ("y_l", "i4"), ("level", "i4"),
                           ("fast_score", "i4"), ("key", "i8"), ("response", "f8"), ("angle", "f8"),
                           ("A", "i4"), ("B", "i4"), ("C", "i4"), ("m10", "i4"), ("m01", "i4")],
                          align=True)
assert KEYPOINT_DTYPE.itemsize == C.sizeof(Keypoint)

_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_I32 = C.POINTER(C.c_int32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.ora_level_sizes.argtypes = [C.c_int, C.c_int, C.c_int, C.c_float, _i32p, _i32p, _f64p]
            L.ora_resize.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, _u8p, C.c_int, C.c_int, C.c_int]
            L.ora_ring_masks.argtypes = [_i32p, C.c_int, C.c_int, C.POINTER(C.c_uint32),
                                         C.POINTER(C.c_uint32)]
            L.ora_has_arc9.argtypes = [C.c_uint32]
            L.ora_has_arc9.restype = C.c_int
            L.ora_is_corner.argtypes = [_i32p, C.c_int, C.c_int]
            L.ora_is_corner.restype = C.c_int
            L.ora_fast_score.argtypes = [_i32p, C.c_int]
            L.ora_fast_score.restype = C.c_int
            L.ora_score_map.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, C.c_int, _u8p]
            L.ora_cell_thresh.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                          C.c_int, _u8p]
            L.ora_nms.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, C.c_int, _u8p, _i32p, C.c_int]
            L.ora_nms.restype = C.c_int
            L.ora_harris_sums.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, C.c_int, _I32, _I32, _I32]
            L.ora_k_fraction.argtypes = [C.c_float, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
            L.ora_k_fraction.restype = C.c_int
            L.ora_harris_key.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int64, C.c_int64]
            L.ora_harris_key.restype = C.c_int64
            L.ora_harris_response.argtypes = [C.c_int64, C.c_int64, C.c_int]
            L.ora_harris_response.restype = C.c_double
            L.ora_orient.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, C.c_int, _I32, _I32,
                                     C.POINTER(C.c_double)]
            L.ora_level_quotas.argtypes = [C.c_int, C.c_int, C.c_float, _i32p]
            L.ora_rank_sort.argtypes = [_i64p, _i32p, _i32p, C.c_int]
            L.ora_detect.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float,
                                     C.POINTER(Config), C.c_float, C.c_int, C.c_void_p, C.c_int,
                                     _i32p]
            L.ora_detect.restype = C.c_int
            L.ora_pyramid_level.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float,
                                            C.c_int, _u8p, _I32, _I32]
            L.ora_pyramid_level.restype = C.c_int
            _lib = L
    return _lib


def _img(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint8)
    if a.ndim != 2:
        raise ValueError("expected a 2-D uint8 image")
    return a


# ---------------------------------------------------------------- pyramid
def level_sizes(W: int, H: int, levels: int, scale: float):
    ws = np.zeros(levels, np.int32)
    hs = np.zeros(levels, np.int32)
    sl = np.zeros(levels, np.float64)
    lib().ora_level_sizes(W, H, levels, scale, ws, hs, sl)
    return ws, hs, sl


def resize(src: np.ndarray, dw: int, dh: int) -> np.ndarray:
    src = _img(src)
    out = np.zeros((dh, dw), np.uint8)
    lib().ora_resize(src, src.shape[1], src.shape[0], src.shape[1], out, dw, dh, dw)
    return out


def pyramid_level(img: np.ndarray, levels: int, scale: float, level: int) -> np.ndarray:
    img = _img(img)
    ws, hs, _ = level_sizes(img.shape[1], img.shape[0], levels, scale)
    out = np.zeros(max(1, int(ws[level]) * int(hs[level])), np.uint8)
    w, h = C.c_int32(), C.c_int32()
    rc = lib().ora_pyramid_level(img, img.shape[1], img.shape[0], img.shape[1], levels, scale,
                                 level, out, C.byref(w), C.byref(h))
    if rc != 0:
        return np.zeros((0, 0), np.uint8)
    return out[: w.value * h.value].reshape(h.value, w.value)


# ------------------------------------------------------------------- FAST
def ring_masks(ring, center: int, t: int):
    r = np.ascontiguousarray(ring, dtype=np.int32)
    b, d = C.c_uint32(), C.c_uint32()
    lib().ora_ring_masks(r, int(center), int(t), C.byref(b), C.byref(d))
    return b.value, d.value


def has_arc9(mask16: int) -> bool:
    return bool(lib().ora_has_arc9(int(mask16) & 0xFFFF))


def is_corner(ring, center: int, t: int) -> bool:
    return bool(lib().ora_is_corner(np.ascontiguousarray(ring, dtype=np.int32), int(center), int(t)))


def fast_score(ring, center: int) -> int:
    return int(lib().ora_fast_score(np.ascontiguousarray(ring, dtype=np.int32), int(center)))


def score_map(img: np.ndarray, border: int) -> np.ndarray:
    img = _img(img)
    h, w = img.shape
    out = np.zeros((h, w), np.uint8)
    lib().ora_score_map(img, w, h, w, border, out)
    return out


def cell_thresh(score: np.ndarray, border: int, cell: int, t_hi: int, t_lo: int) -> np.ndarray:
    score = _img(score)
    h, w = score.shape
    rw, rh = w - 2 * border, h - 2 * border
    if rw <= 0 or rh <= 0:
        return np.zeros((0, 0), np.uint8)
    ncx, ncy = -(-rw // cell), -(-rh // cell)
    T = np.zeros((ncy, ncx), np.uint8)
    lib().ora_cell_thresh(score, w, h, border, cell, t_hi, t_lo, T)
    return T


def nms(score: np.ndarray, border: int, cell: int, T: np.ndarray) -> np.ndarray:
    """Survivors of strict 3x3 NMS in raster order, as an (n, 2) int32 array of (x, y)."""
    score = _img(score)
    h, w = score.shape
    T = np.ascontiguousarray(T, dtype=np.uint8)
    if T.size == 0:
        return np.zeros((0, 2), np.int32)
    cap = w * h
    xy = np.zeros(2 * cap, np.int32)
    n = lib().ora_nms(score, w, h, border, cell, T.reshape(-1), xy, cap)
    return xy[: 2 * n].reshape(n, 2)


# ----------------------------------------------------------------- Harris
def harris_sums(img: np.ndarray, x: int, y: int, block: int = 7):
    img = _img(img)
    A, B, Cc = C.c_int32(), C.c_int32(), C.c_int32()
    lib().ora_harris_sums(img, img.shape[1], int(x), int(y), block, C.byref(A), C.byref(B), C.byref(Cc))
    return A.value, B.value, Cc.value


def k_fraction(k: float):
    n, d = C.c_int64(), C.c_int64()
    rc = lib().ora_k_fraction(k, C.byref(n), C.byref(d))
    if rc != 0:
        raise ValueError(f"harris k={k} not representable")
    return n.value, d.value


def harris_key(A: int, B: int, Cc: int, num: int, den: int) -> int:
    return int(lib().ora_harris_key(A, B, Cc, num, den))


def harris_response(key: int, den: int, block: int = 7) -> float:
    return float(lib().ora_harris_response(key, den, block))


# ------------------------------------------------------------ orientation
def orient(img: np.ndarray, x: int, y: int, radius: int = 15):
    img = _img(img)
    a, b, th = C.c_int32(), C.c_int32(), C.c_double()
    lib().ora_orient(img, img.shape[1], int(x), int(y), radius, C.byref(a), C.byref(b), C.byref(th))
    return a.value, b.value, th.value


# ------------------------------------------------------------ quotas, rank
def level_quotas(N: int, L: int, scale: float) -> np.ndarray:
    n = np.zeros(L, np.int32)
    lib().ora_level_quotas(N, L, scale, n)
    return n


def rank_sort(key, x, y):
    key = np.ascontiguousarray(key, dtype=np.int64).copy()
    x = np.ascontiguousarray(x, dtype=np.int32).copy()
    y = np.ascontiguousarray(y, dtype=np.int32).copy()
    lib().ora_rank_sort(key, x, y, len(key))
    return key, x, y


# --------------------------------------------------------------- pipeline
def detect(img: np.ndarray, levels: int = 1, scale: float = 1.2, fast_t: int = 20, fast_t_lo: int | None = None,
           harris_k: float = 0.04, n_features: int = 500, border: int = 19, cell: int = 30,
           block: int = 7, radius: int = 15, with_counts: bool = False):
    """The whole chain for one frame; returns a structured array (KEYPOINT_DTYPE)."""
    img = _img(img)
    h, w = img.shape
    cfg = Config(border, cell, block, radius, fast_t, fast_t if fast_t_lo is None else fast_t_lo)
    cap = max(1, n_features)
    out = np.zeros(cap, KEYPOINT_DTYPE)
    counts = np.zeros(levels, np.int32)
    n = lib().ora_detect(img, w, h, w, levels, scale, C.byref(cfg), harris_k, n_features,
                         out.ctypes.data, cap, counts)
    if n < 0:
        raise ValueError("oracle rejected the arguments")
    if with_counts:
        return out[:n], counts
    return out[:n]
