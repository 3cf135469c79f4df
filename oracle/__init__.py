"""Reference oracle for the resampling path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path (the CUDA library and
its Python binding) never imports it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain single-threaded C, built with
``-O2 -ffp-contract=off``); this module only builds it and marshals numpy
arrays. Every function takes and returns contiguous HWC arrays; views, pitches
and planar layouts are the caller's business.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, hand-worked cases, an exact-rational brute force, and library
routines that compute the same special case).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_u8p = ctypes.POINTER(ctypes.c_uint8)
_f32p = ctypes.POINTER(ctypes.c_float)
_f64p = ctypes.POINTER(ctypes.c_double)
_lp = ctypes.POINTER(ctypes.c_long)
_L = ctypes.c_long


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99", "-Wall",
             "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.oracle_resize_u8.argtypes = [_u8p, _L, _L, _L, _u8p, _L, _L, ctypes.c_int, _u8p]
            lib.oracle_resize_f64.argtypes = [_u8p, _L, _L, _L, _f64p, _L, _L, ctypes.c_int,
                                              _f64p, _f64p, _u8p]
            lib.oracle_warp_u8.argtypes = [_u8p, _L, _L, _L, _f32p, _u8p, _L, _L, ctypes.c_int, _u8p]
            lib.oracle_warp_f64.argtypes = [_u8p, _L, _L, _L, _f32p, _f64p, _L, _L, ctypes.c_int,
                                            _f64p, _f64p, _u8p]
            lib.oracle_rgb_to_gray_u8.argtypes = [_u8p, _L, _L, _u8p]
            lib.oracle_warp_point.argtypes = [_f32p, _L, _L, _f32p, _f32p, _lp, _lp, _lp, _lp]
            lib.oracle_resize_point.argtypes = [_L, _L, _L, _lp, _lp, _lp, _f64p]
            lib.oracle_resize_nearest_u8.argtypes = [_u8p, _L, _L, _L, _u8p, _L, _L]
            lib.oracle_warp_persp_u8.argtypes = [_u8p, _L, _L, _L, _f32p, _u8p, _L, _L, ctypes.c_int, _u8p]
            lib.oracle_warp_persp_f64.argtypes = [_u8p, _L, _L, _L, _f32p, _f64p, _L, _L, ctypes.c_int,
                                                  _f64p, _f64p, _u8p]
            lib.oracle_persp_point.argtypes = [_f32p, _L, _L, _f32p, _f32p, _lp, _lp, _lp, _lp]
            lib.oracle_warp_ex_u8.argtypes = [_u8p, _L, _L, _L, _f32p, ctypes.c_int, ctypes.c_int, _u8p, _L, _L,
                                              ctypes.c_int, _u8p]
            lib.oracle_warp_ex_f64.argtypes = [_u8p, _L, _L, _L, _f32p, ctypes.c_int, ctypes.c_int, _f64p, _L,
                                               _L, ctypes.c_int, _f64p, _f64p, _u8p]
            lib.oracle_flip_h_u8.argtypes = [_u8p, _L, _L, _L, _u8p]
            lib.oracle_sobel.argtypes = [_u8p, _L, _L, _L, _f32p, _u8p]
            lib.oracle_resize_area_u8.argtypes = [_u8p, _L, _L, _L, _u8p, _L, _L]
            lib.oracle_resize_area_f64.argtypes = [_u8p, _L, _L, _L, _f64p, _L, _L, _f64p, _f64p]
            for f in (lib.oracle_resize_u8, lib.oracle_resize_f64, lib.oracle_warp_u8,
                      lib.oracle_warp_f64, lib.oracle_rgb_to_gray_u8, lib.oracle_warp_point,
                      lib.oracle_resize_point):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _src(img):
    img = np.ascontiguousarray(img, dtype=np.uint8)
    if img.ndim == 2:
        img = img[:, :, None]
    if img.ndim != 3 or img.shape[2] not in (1, 3):
        raise ValueError("oracle: source must be H x W x C with C in (1, 3)")
    return img


def _norm(C, mean, std):
    m = np.zeros(3) if mean is None else np.asarray(mean, dtype=np.float64).reshape(-1)
    s = np.ones(3) if std is None else np.asarray(std, dtype=np.float64).reshape(-1)
    m = np.ascontiguousarray(np.resize(m, 3))
    s = np.ascontiguousarray(np.resize(s, 3))
    return m, s


def _touched(H, W, want):
    return np.zeros((H, W), dtype=np.uint8) if want else None


def resize_u8(img, h, w, gray=False, touched=False):
    """Bilinear resize to h x w, u8 fixed point. Returns out (and the touched bitmap)."""
    src = _src(img)
    H, W, C = src.shape
    out = np.zeros((h, w, 1 if gray else C), dtype=np.uint8)
    t = _touched(H, W, touched)
    rc = _load().oracle_resize_u8(_p(src, _u8p), H, W, C, _p(out, _u8p), h, w, int(gray), _p(t, _u8p))
    if rc != 0:
        raise ValueError("oracle_resize_u8: bad arguments")
    return (out, t) if touched else out


def resize_f64(img, h, w, gray=False, mean=None, std=None, touched=False):
    """Bilinear resize to h x w of p/255, normalised, in double (HWC out)."""
    src = _src(img)
    H, W, C = src.shape
    m, s = _norm(C, mean, std)
    out = np.zeros((h, w, 1 if gray else C), dtype=np.float64)
    t = _touched(H, W, touched)
    rc = _load().oracle_resize_f64(_p(src, _u8p), H, W, C, _p(out, _f64p), h, w, int(gray),
                                   _p(m, _f64p), _p(s, _f64p), _p(t, _u8p))
    if rc != 0:
        raise ValueError("oracle_resize_f64: bad arguments")
    return (out, t) if touched else out


def _mat(M, n=6):
    M = np.ascontiguousarray(np.asarray(M, dtype=np.float32).reshape(n))
    return M


_BORDERS = {"zero": 0, "replicate": 1}


def _warp_ex_u8(img, M, h, w, persp, border, gray, touched):
    src = _src(img)
    H, W, C = src.shape
    Mf = _mat(M, 9 if persp else 6)
    out = np.zeros((h, w, 1 if gray else C), dtype=np.uint8)
    t = _touched(H, W, touched)
    rc = _load().oracle_warp_ex_u8(_p(src, _u8p), H, W, C, _p(Mf, _f32p), int(persp), _BORDERS[border],
                                   _p(out, _u8p), h, w, int(gray), _p(t, _u8p))
    if rc != 0:
        raise ValueError("oracle_warp_ex_u8: bad arguments")
    return (out, t) if touched else out


def _warp_ex_f64(img, M, h, w, persp, border, gray, mean, std, touched):
    src = _src(img)
    H, W, C = src.shape
    Mf = _mat(M, 9 if persp else 6)
    m, s = _norm(C, mean, std)
    out = np.zeros((h, w, 1 if gray else C), dtype=np.float64)
    t = _touched(H, W, touched)
    rc = _load().oracle_warp_ex_f64(_p(src, _u8p), H, W, C, _p(Mf, _f32p), int(persp), _BORDERS[border],
                                    _p(out, _f64p), h, w, int(gray), _p(m, _f64p), _p(s, _f64p), _p(t, _u8p))
    if rc != 0:
        raise ValueError("oracle_warp_ex_f64: bad arguments")
    return (out, t) if touched else out


def warp_u8(img, M, h, w, gray=False, touched=False, border="zero"):
    """Affine warp (M: 2x3 destination->source, fp32), zero or replicated border, u8 fixed point."""
    if border != "zero":
        return _warp_ex_u8(img, M, h, w, False, border, gray, touched)
    src = _src(img)
    H, W, C = src.shape
    Mf = _mat(M)
    out = np.zeros((h, w, 1 if gray else C), dtype=np.uint8)
    t = _touched(H, W, touched)
    rc = _load().oracle_warp_u8(_p(src, _u8p), H, W, C, _p(Mf, _f32p), _p(out, _u8p), h, w,
                                int(gray), _p(t, _u8p))
    if rc != 0:
        raise ValueError("oracle_warp_u8: bad arguments")
    return (out, t) if touched else out


def warp_f64(img, M, h, w, gray=False, mean=None, std=None, touched=False, border="zero"):
    """Affine warp of p/255 in double (fp32 coordinate), zero or replicated border, normalised."""
    if border != "zero":
        return _warp_ex_f64(img, M, h, w, False, border, gray, mean, std, touched)
    src = _src(img)
    H, W, C = src.shape
    Mf = _mat(M)
    m, s = _norm(C, mean, std)
    out = np.zeros((h, w, 1 if gray else C), dtype=np.float64)
    t = _touched(H, W, touched)
    rc = _load().oracle_warp_f64(_p(src, _u8p), H, W, C, _p(Mf, _f32p), _p(out, _f64p), h, w,
                                 int(gray), _p(m, _f64p), _p(s, _f64p), _p(t, _u8p))
    if rc != 0:
        raise ValueError("oracle_warp_f64: bad arguments")
    return (out, t) if touched else out


def rgb_to_gray_u8(img):
    """Standalone BT.601 gray of an H x W x 3 u8 image (14-bit weights)."""
    src = _src(img)
    H, W, C = src.shape
    if C != 3:
        raise ValueError("rgb_to_gray_u8: source must have 3 channels")
    out = np.zeros((H, W, 1), dtype=np.uint8)
    rc = _load().oracle_rgb_to_gray_u8(_p(src, _u8p), H, W, _p(out, _u8p))
    if rc != 0:
        raise ValueError("oracle_rgb_to_gray_u8: bad arguments")
    return out


def resize_nearest_u8(img, h, w):
    """Nearest-neighbour resize (half-pixel centres) of an H x W x C u8 image to h x w."""
    src = _src(img)
    H, W, C = src.shape
    out = np.zeros((h, w, C), dtype=np.uint8)
    rc = _load().oracle_resize_nearest_u8(_p(src, _u8p), H, W, C, _p(out, _u8p), h, w)
    if rc != 0:
        raise ValueError("oracle_resize_nearest_u8: bad arguments")
    return out


def resize_area_u8(img, h, w):
    """Area (overlap-weighted mean) downscale of an H x W x C u8 image to h x w (h <= H, w <= W)."""
    src = _src(img)
    H, W, C = src.shape
    out = np.zeros((h, w, C), dtype=np.uint8)
    rc = _load().oracle_resize_area_u8(_p(src, _u8p), H, W, C, _p(out, _u8p), h, w)
    if rc != 0:
        raise ValueError("oracle_resize_area_u8: bad arguments")
    return out


def resize_area_f64(img, h, w, mean=None, std=None):
    """Area downscale of p/255 in double, normalised."""
    src = _src(img)
    H, W, C = src.shape
    m, s = _norm(C, mean, std)
    out = np.zeros((h, w, C), dtype=np.float64)
    rc = _load().oracle_resize_area_f64(_p(src, _u8p), H, W, C, _p(out, _f64p), h, w, _p(m, _f64p), _p(s, _f64p))
    if rc != 0:
        raise ValueError("oracle_resize_area_f64: bad arguments")
    return out


def sobel(img):
    """Sobel 3x3 magnitude (replicated border, normalised kernels) of an H x W x C u8 image
    (C = 3: of its u8 gray): (f32 H x W x 1, u8 H x W x 1)."""
    src = _src(img)
    H, W, C = src.shape
    f = np.zeros((H, W, 1), dtype=np.float32)
    u = np.zeros((H, W, 1), dtype=np.uint8)
    rc = _load().oracle_sobel(_p(src, _u8p), H, W, C, _p(f, _f32p), _p(u, _u8p))
    if rc != 0:
        raise ValueError("oracle_sobel: bad arguments")
    return f, u


def flip_h_u8(img):
    """Horizontal flip of an H x W x C u8 image."""
    src = _src(img)
    H, W, C = src.shape
    out = np.zeros((H, W, C), dtype=np.uint8)
    rc = _load().oracle_flip_h_u8(_p(src, _u8p), H, W, C, _p(out, _u8p))
    if rc != 0:
        raise ValueError("oracle_flip_h_u8: bad arguments")
    return out


def warp_persp_u8(img, M, h, w, gray=False, touched=False, border="zero"):
    """Perspective warp (M: 3x3 destination->source, fp32), zero or replicated border, u8 fixed point."""
    if border != "zero":
        return _warp_ex_u8(img, M, h, w, True, border, gray, touched)
    src = _src(img)
    H, W, C = src.shape
    Mf = _mat(M, 9)
    out = np.zeros((h, w, 1 if gray else C), dtype=np.uint8)
    t = _touched(H, W, touched)
    rc = _load().oracle_warp_persp_u8(_p(src, _u8p), H, W, C, _p(Mf, _f32p), _p(out, _u8p), h, w,
                                      int(gray), _p(t, _u8p))
    if rc != 0:
        raise ValueError("oracle_warp_persp_u8: bad arguments")
    return (out, t) if touched else out


def warp_persp_f64(img, M, h, w, gray=False, mean=None, std=None, touched=False, border="zero"):
    """Perspective warp of p/255 in double (fp32 coordinate), zero or replicated border, normalised."""
    if border != "zero":
        return _warp_ex_f64(img, M, h, w, True, border, gray, mean, std, touched)
    src = _src(img)
    H, W, C = src.shape
    Mf = _mat(M, 9)
    m, s = _norm(C, mean, std)
    out = np.zeros((h, w, 1 if gray else C), dtype=np.float64)
    t = _touched(H, W, touched)
    rc = _load().oracle_warp_persp_f64(_p(src, _u8p), H, W, C, _p(Mf, _f32p), _p(out, _f64p), h, w,
                                       int(gray), _p(m, _f64p), _p(s, _f64p), _p(t, _u8p))
    if rc != 0:
        raise ValueError("oracle_warp_persp_f64: bad arguments")
    return (out, t) if touched else out


def persp_point(M, x, y):
    """(ok, sx, sy, x0, qx, y0, qy) of output pixel (x, y) under the 3x3 map M."""
    Mf = _mat(M, 9)
    sx, sy = ctypes.c_float(), ctypes.c_float()
    x0, qx, y0, qy = ctypes.c_long(), ctypes.c_long(), ctypes.c_long(), ctypes.c_long()
    ok = _load().oracle_persp_point(_p(Mf, _f32p), x, y, ctypes.byref(sx), ctypes.byref(sy),
                                    ctypes.byref(x0), ctypes.byref(qx), ctypes.byref(y0),
                                    ctypes.byref(qy))
    return bool(ok), sx.value, sy.value, x0.value, qx.value, y0.value, qy.value


def warp_point(M, x, y):
    """(ok, sx, sy, x0, qx, y0, qy) of output pixel (x, y) under M."""
    Mf = _mat(M)
    sx, sy = ctypes.c_float(), ctypes.c_float()
    x0, qx, y0, qy = ctypes.c_long(), ctypes.c_long(), ctypes.c_long(), ctypes.c_long()
    ok = _load().oracle_warp_point(_p(Mf, _f32p), x, y, ctypes.byref(sx), ctypes.byref(sy),
                                   ctypes.byref(x0), ctypes.byref(qx), ctypes.byref(y0),
                                   ctypes.byref(qy))
    return bool(ok), sx.value, sy.value, x0.value, qx.value, y0.value, qy.value


def resize_point(i, n_in, n_out):
    """(i0, i1, q, frac) of output index i along one resize axis."""
    i0, i1, q = ctypes.c_long(), ctypes.c_long(), ctypes.c_long()
    fr = ctypes.c_double()
    rc = _load().oracle_resize_point(i, n_in, n_out, ctypes.byref(i0), ctypes.byref(i1),
                                     ctypes.byref(q), ctypes.byref(fr))
    if rc != 0:
        raise ValueError("resize_point: bad arguments")
    return i0.value, i1.value, q.value, fr.value


def touched_bytes(bitmap, C, row_bytes=None, sector=None):
    """Unique source bytes read (pixel granular), or unique `sector`-byte sectors x sector."""
    bm = np.asarray(bitmap, dtype=bool)
    if sector is None:
        return int(bm.sum()) * C
    H, W = bm.shape
    row_bytes = W * C if row_bytes is None else row_bytes
    ys, xs = np.nonzero(bm)
    off = ys.astype(np.int64) * row_bytes + xs.astype(np.int64) * C
    return int(np.unique(np.concatenate([off // sector, (off + C - 1) // sector])).size) * sector
