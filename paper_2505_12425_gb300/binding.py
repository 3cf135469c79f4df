"""Thin Python binding of the C ABI in include/kr.h (ctypes).

Argument marshalling only: every function here builds the C descriptors from
torch tensors (device memory, shapes, strides) and calls the library entry of
the same name; all resampling work runs in the library's CUDA kernels. There
is no CPU fallback: if libkr.so is missing or has no GPU to run on, the call
raises.

Image tensors:
  * u8 / f32 HWC: shape (H, W, C), (N, H, W, C) or (H, W) for C = 1; the last
    two strides must be (C, 1) -- rows may be padded and images may be views;
  * f32 CHW (destinations): shape (C, H, W) or (N, C, H, W), last stride 1,
    selected with layout="chw".
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkr.so")

KR_U8, KR_F32 = 0, 1
KR_HWC, KR_CHW = 0, 1
KR_GRAY, KR_NORMALIZE, KR_BORDER_REPLICATE = 1, 2, 4
KR_OP_RESIZE, KR_OP_WARP, KR_OP_GRAY = 0, 1, 2

STATUS = {0: "KR_OK", 1: "KR_ERR_INVALID_ARG", 2: "KR_ERR_UNSUPPORTED", 3: "KR_ERR_ALIAS",
          4: "KR_ERR_CUDA", 5: "KR_ERR_NO_SPACE", 6: "KR_ERR_TIMEOUT"}


class KrError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


class KrImage(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("height", ctypes.c_int32), ("width", ctypes.c_int32),
                ("channels", ctypes.c_int32), ("dtype", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("batch", ctypes.c_int32), ("pitch", ctypes.c_int64), ("plane_stride", ctypes.c_int64),
                ("batch_stride", ctypes.c_int64)]


class KrPost(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_uint32), ("mean", ctypes.c_float * 3), ("std", ctypes.c_float * 3)]


class KrWork(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("src", KrImage), ("dst", KrImage), ("M", ctypes.c_float * 6),
                ("post", KrPost)]


class KrBatchOpts(ctypes.Structure):
    _fields_ = [("tile_config", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("use_graph", ctypes.c_int32)]


class KrRequest(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("src_index", ctypes.c_int32), ("out_h", ctypes.c_int32),
                ("out_w", ctypes.c_int32), ("M", ctypes.c_float * 6), ("t_arrival", ctypes.c_double)]


class KrServeConfig(ctypes.Structure):
    _fields_ = [("pool", ctypes.POINTER(KrImage)), ("pool_n", ctypes.c_int32), ("out_arena", ctypes.c_void_p),
                ("out_arena_bytes", ctypes.c_size_t), ("hbm_budget_bytes", ctypes.c_size_t),
                ("max_batch", ctypes.c_int32), ("streams", ctypes.c_int32), ("policy", ctypes.c_int32),
                ("workspaces", ctypes.c_void_p), ("ws_bytes_each", ctypes.c_size_t),
                ("retain_outputs", ctypes.c_int32), ("direct_px", ctypes.c_int64)]


class KrServeResult(ctypes.Structure):
    _fields_ = [("t_admit", ctypes.c_double), ("t_launch", ctypes.c_double), ("t_done", ctypes.c_double),
                ("out_offset", ctypes.c_int64), ("status", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None


def load():
    """Load libkr.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        S = ctypes.c_int
        lib.kr_resize_bilinear.argtypes = [P(KrImage), P(KrImage), P(KrPost), ctypes.c_void_p]
        lib.kr_warp_affine.argtypes = [P(KrImage), P(KrImage), P(ctypes.c_float), P(KrPost), ctypes.c_void_p]
        lib.kr_rgb_to_gray.argtypes = [P(KrImage), P(KrImage), ctypes.c_void_p]
        lib.kr_resize_nearest.argtypes = [P(KrImage), P(KrImage), ctypes.c_void_p]
        lib.kr_sobel.argtypes = [P(KrImage), P(KrImage), ctypes.c_int32, ctypes.c_void_p]
        lib.kr_resize_area.argtypes = [P(KrImage), P(KrImage), P(KrPost), ctypes.c_void_p]
        lib.kr_warp_perspective.argtypes = [P(KrImage), P(KrImage), P(ctypes.c_float), P(KrPost), ctypes.c_void_p]
        lib.kr_flip_horizontal.argtypes = [P(KrImage), P(KrImage), ctypes.c_void_p]
        lib.kr_batch_workspace_size.argtypes = [ctypes.c_int32]
        lib.kr_batch_workspace_size.restype = ctypes.c_size_t
        lib.kr_batch_submit.argtypes = [P(KrWork), ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t,
                                        P(KrBatchOpts), ctypes.c_void_p]
        lib.kr_batch_submit_noalloc.argtypes = [P(KrWork), ctypes.c_int32, P(KrBatchOpts), ctypes.c_void_p]
        lib.kr_serve_run.argtypes = [P(KrRequest), ctypes.c_int32, P(KrServeConfig), P(KrServeResult)]
        lib.kr_device_errors.argtypes = [P(ctypes.c_uint32), ctypes.c_int32]
        lib.kr_debug_set_stage_wait_ns.argtypes = [ctypes.c_uint64]
        lib.kr_debug_set_fault.argtypes = [ctypes.c_int32, ctypes.c_int32]
        lib.kr_tile_config_count.argtypes = []
        lib.kr_tile_config_count.restype = ctypes.c_int32
        lib.kr_tile_config_shape.argtypes = [ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_int32)]
        lib.kr_autotune_batch.argtypes = [P(KrWork), ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t,
                                          ctypes.c_void_p, P(ctypes.c_int32), P(ctypes.c_int32)]
        lib.kr_autotune_save.argtypes = [ctypes.c_char_p]
        lib.kr_autotune_load.argtypes = [ctypes.c_char_p]
        lib.kr_status_string.argtypes = [S]
        lib.kr_status_string.restype = ctypes.c_char_p
        lib.kr_last_error.argtypes = []
        lib.kr_last_error.restype = ctypes.c_char_p
        lib.kr_shutdown.argtypes = []
        lib.kr_shutdown.restype = None
        for f in ("kr_resize_bilinear", "kr_warp_affine", "kr_warp_perspective", "kr_rgb_to_gray", "kr_resize_nearest",
                  "kr_flip_horizontal", "kr_sobel", "kr_resize_area", "kr_batch_submit",
                  "kr_batch_submit_noalloc", "kr_serve_run", "kr_device_errors", "kr_debug_set_stage_wait_ns",
                  "kr_debug_set_fault",
                  "kr_tile_config_shape", "kr_autotune_batch", "kr_autotune_save", "kr_autotune_load"):
            getattr(lib, f).restype = S
        _lib = lib
        return lib


def _check(st: int, where: str):
    if st != 0:
        detail = load().kr_last_error().decode() if st == 4 else ""
        raise KrError(st, where, detail)


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def image(t: torch.Tensor, layout: str = "hwc") -> KrImage:
    """A kr_image_t describing tensor t (see the module docstring for accepted shapes)."""
    if t.dtype == torch.uint8:
        dt, es = KR_U8, 1
    elif t.dtype == torch.float32:
        dt, es = KR_F32, 4
    else:
        raise TypeError(f"unsupported dtype {t.dtype}")
    im = KrImage()
    im.data = t.data_ptr()
    im.dtype = dt
    st = t.stride()
    if layout == "hwc":
        if t.dim() == 2:
            n, (h, w), c = 1, t.shape, 1
            if st[1] != 1:
                raise ValueError("pixels of a row must be contiguous")
            pitch, bstride = st[0], 0
        elif t.dim() in (3, 4):
            shp = t.shape if t.dim() == 4 else (1, *t.shape)
            sts = st if t.dim() == 4 else (0, *st)
            n, h, w, c = shp
            if sts[3] != 1 or (c > 1 and sts[2] != c):
                raise ValueError("HWC tensors need strides (..., C, 1)")
            pitch, bstride = sts[1], sts[0]
        else:
            raise ValueError("HWC image must be 2-D, 3-D or 4-D")
        im.layout, im.plane_stride = KR_HWC, 0
    elif layout == "chw":
        shp = t.shape if t.dim() == 4 else (1, *t.shape)
        sts = st if t.dim() == 4 else (0, *st)
        n, c, h, w = shp
        if sts[3] != 1:
            raise ValueError("CHW tensors need a unit last stride")
        pitch, bstride = sts[2], sts[0]
        im.layout, im.plane_stride = KR_CHW, sts[1] * es
    else:
        raise ValueError(layout)
    im.height, im.width, im.channels, im.batch = h, w, c, n
    im.pitch = pitch * es
    im.batch_stride = bstride * es
    return im


def post(gray: bool = False, mean=None, std=None, border: str = "zero") -> KrPost:
    if border not in ("zero", "replicate"):
        raise ValueError(f"border must be 'zero' or 'replicate', got {border!r}")
    p = KrPost()
    p.flags = (KR_GRAY if gray else 0) | (KR_NORMALIZE if (mean is not None or std is not None) else 0) | \
        (KR_BORDER_REPLICATE if border == "replicate" else 0)
    m = (0.0, 0.0, 0.0) if mean is None else tuple(float(v) for v in mean)
    s = (1.0, 1.0, 1.0) if std is None else tuple(float(v) for v in std)
    for i in range(3):
        p.mean[i] = m[i] if len(m) > i else m[0]
        p.std[i] = s[i] if len(s) > i else s[0]
    return p


def kr_resize_bilinear(src, dst, gray=False, mean=None, std=None, dst_layout="hwc", stream=None):
    """Bilinear resize of u8 HWC `src` into pre-allocated `dst` (its size is the output size)."""
    lib = load()
    s, d, p = image(src), image(dst, dst_layout), post(gray, mean, std)
    _check(lib.kr_resize_bilinear(ctypes.byref(s), ctypes.byref(d), ctypes.byref(p), _stream(stream)),
           "kr_resize_bilinear")


def _mats(M, n, k=6):
    import numpy as np
    a = np.ascontiguousarray(np.asarray(M, dtype=np.float32).reshape(-1))
    if a.size != k * n:
        raise ValueError(f"need {n} matrices of {k} floats, got {a.size / k}")
    return a


def kr_warp_affine(src, dst, M, gray=False, mean=None, std=None, dst_layout="hwc", stream=None, border="zero"):
    """Affine warp (M: (N,) 2x3 destination->source maps) of u8 HWC `src` into `dst`."""
    lib = load()
    s, d, p = image(src), image(dst, dst_layout), post(gray, mean, std, border)
    a = _mats(M, s.batch)
    _check(lib.kr_warp_affine(ctypes.byref(s), ctypes.byref(d),
                              a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(p),
                              _stream(stream)), "kr_warp_affine")


def kr_warp_perspective(src, dst, M, gray=False, mean=None, std=None, dst_layout="hwc", stream=None,
                        border="zero"):
    """Perspective warp (M: (N,) 3x3 destination->source maps) of u8 HWC `src` into `dst`."""
    lib = load()
    s, d, p = image(src), image(dst, dst_layout), post(gray, mean, std, border)
    a = _mats(M, s.batch, 9)
    _check(lib.kr_warp_perspective(ctypes.byref(s), ctypes.byref(d),
                                   a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(p),
                                   _stream(stream)), "kr_warp_perspective")


def kr_rgb_to_gray(src, dst, stream=None):
    """BT.601 gray of u8 HWC RGB `src` into u8 `dst` of the same size."""
    lib = load()
    s, d = image(src), image(dst)
    _check(lib.kr_rgb_to_gray(ctypes.byref(s), ctypes.byref(d), _stream(stream)), "kr_rgb_to_gray")


def kr_resize_nearest(src, dst, stream=None):
    """Nearest-neighbour resize (half-pixel centres) of u8 HWC `src` into u8 `dst`."""
    lib = load()
    s, d = image(src), image(dst)
    _check(lib.kr_resize_nearest(ctypes.byref(s), ctypes.byref(d), _stream(stream)), "kr_resize_nearest")


def kr_flip_horizontal(src, dst, stream=None):
    """Horizontal flip of u8 HWC `src` into `dst` of the same size (not in place)."""
    lib = load()
    s, d = image(src), image(dst)
    _check(lib.kr_flip_horizontal(ctypes.byref(s), ctypes.byref(d), _stream(stream)), "kr_flip_horizontal")


def kr_resize_area(src, dst, mean=None, std=None, dst_layout="hwc", stream=None):
    """Area (overlap-weighted mean) downscale of u8 HWC `src` into `dst` (u8, or f32 normalised)."""
    lib = load()
    s, d, p = image(src), image(dst, dst_layout), post(False, mean, std)
    _check(lib.kr_resize_area(ctypes.byref(s), ctypes.byref(d), ctypes.byref(p), _stream(stream)), "kr_resize_area")


def kr_sobel(src, dst, ksize=3, stream=None):
    """Sobel 3x3 magnitude of u8 HWC `src` (RGB: of its gray) into single-channel u8 or f32 `dst`."""
    lib = load()
    s, d = image(src), image(dst)
    _check(lib.kr_sobel(ctypes.byref(s), ctypes.byref(d), int(ksize), _stream(stream)), "kr_sobel")


def work_item(op, src, dst, M=None, gray=False, mean=None, std=None, dst_layout="hwc", border="zero") -> KrWork:
    """One kr_work_t (batch == 1 images)."""
    w = KrWork()
    w.op = op
    w.src = image(src)
    w.dst = image(dst, dst_layout)
    if M is not None:
        a = _mats(M, 1)
        for i in range(6):
            w.M[i] = float(a[i])
    w.post = post(gray, mean, std, border)
    return w


def work_array(items) -> ctypes.Array:
    arr = (KrWork * len(items))()
    for i, it in enumerate(items):
        arr[i] = it
    return arr


def kr_batch_workspace_size(max_items: int) -> int:
    return int(load().kr_batch_workspace_size(max_items))


def kr_batch_submit(items, workspace: torch.Tensor, tile_config: int = -1, ctas_per_sm: int = 0,
                    use_graph: bool = False, stream=None):
    """Run kr_work_t items (a list or a ctypes array) in one persistent launch."""
    lib = load()
    arr = items if isinstance(items, ctypes.Array) else work_array(items)
    o = KrBatchOpts(tile_config, ctas_per_sm, 1 if use_graph else 0)
    _check(lib.kr_batch_submit(arr, len(arr), ctypes.c_void_p(workspace.data_ptr()),
                               workspace.numel() * workspace.element_size(), ctypes.byref(o),
                               _stream(stream)), "kr_batch_submit")


KR_BATCH_NOALLOC_MAX_ITEMS = 1024


def kr_batch_submit_noalloc(items, tile_config: int = -1, ctas_per_sm: int = 0, stream=None):
    """kr_batch_submit without a workspace: for callers that may not allocate device memory
    when they submit (the work list goes into a fixed device array inside the library)."""
    lib = load()
    arr = items if isinstance(items, ctypes.Array) else work_array(items)
    o = KrBatchOpts(tile_config, ctas_per_sm, 0)
    _check(lib.kr_batch_submit_noalloc(arr, len(arr), ctypes.byref(o), _stream(stream)),
           "kr_batch_submit_noalloc")


def kr_tile_config_count() -> int:
    return int(load().kr_tile_config_count())


def kr_tile_config_shape(i: int):
    tw, th = ctypes.c_int32(), ctypes.c_int32()
    _check(load().kr_tile_config_shape(i, ctypes.byref(tw), ctypes.byref(th)), "kr_tile_config_shape")
    return tw.value, th.value


def kr_autotune_batch(items, workspace: torch.Tensor, stream=None):
    lib = load()
    arr = items if isinstance(items, ctypes.Array) else work_array(items)
    cfg, ctas = ctypes.c_int32(), ctypes.c_int32()
    _check(lib.kr_autotune_batch(arr, len(arr), ctypes.c_void_p(workspace.data_ptr()),
                                 workspace.numel() * workspace.element_size(), _stream(stream),
                                 ctypes.byref(cfg), ctypes.byref(ctas)), "kr_autotune_batch")
    return cfg.value, ctas.value


def kr_autotune_save(path: str):
    _check(load().kr_autotune_save(path.encode()), "kr_autotune_save")


def kr_autotune_load(path: str):
    _check(load().kr_autotune_load(path.encode()), "kr_autotune_load")


def kr_status_string(status: int) -> str:
    return load().kr_status_string(status).decode()


def kr_shutdown():
    load().kr_shutdown()


def kr_device_errors(clear: bool = True) -> int:
    """Device error flags of the single-image kernels (bit 0: a TMA wait ran out)."""
    v = ctypes.c_uint32()
    _check(load().kr_device_errors(ctypes.byref(v), 1 if clear else 0), "kr_device_errors")
    return v.value


# sites of kr_debug_set_fault
KR_FAULT_SUBMIT, KR_FAULT_EVENT, KR_FAULT_ADMIT = 1, 2, 3
KR_STAGE_WAIT_NS_DEFAULT = 2_000_000_000


def kr_debug_set_stage_wait_ns(ns: int):
    """Bound of the tile kernels' first wait for a staged box (0: give up at once)."""
    _check(load().kr_debug_set_stage_wait_ns(int(ns)), "kr_debug_set_stage_wait_ns")


def kr_debug_set_fault(site: int, period: int):
    """Make a host-side step of kr_serve_run fail every period-th time (0: never)."""
    _check(load().kr_debug_set_fault(int(site), int(period)), "kr_debug_set_fault")


def requests_array(reqs) -> ctypes.Array:
    """kr_request_t array from objects with op, src_index, h, w, M, t_arrival."""
    arr = (KrRequest * len(reqs))()
    for i, r in enumerate(reqs):
        arr[i].op = int(r.op)
        arr[i].src_index = int(r.src_index)
        arr[i].out_h = int(r.h)
        arr[i].out_w = int(r.w)
        m = [float(v) for v in r.M.reshape(-1)]
        for k in range(6):
            arr[i].M[k] = m[k]
        arr[i].t_arrival = float(r.t_arrival)
    return arr


def kr_serve_run(reqs, pool, arena: torch.Tensor, budget_bytes: int = 8 << 30, max_batch: int = 64,
                 streams: int = 4, policy: int = 0, retain_outputs: bool = False, direct_px: int = 0):
    """Serve `reqs` (see inputs.request_stream) over the device image `pool` (list of u8 HWC
    tensors); outputs are carved from the device tensor `arena`. Returns the kr_serve_result_t
    array (seconds from the start of the run; byte offsets into the arena)."""
    lib = load()
    arr = reqs if isinstance(reqs, ctypes.Array) else requests_array(reqs)
    imgs = (KrImage * len(pool))()
    for i, t in enumerate(pool):
        imgs[i] = image(t)
    ws = None
    ws_each = 0
    if policy in (0, 2):
        ws_each = kr_batch_workspace_size(max_batch)
        ws_each = (ws_each + 255) // 256 * 256
        ws = torch.empty(ws_each * streams, dtype=torch.uint8, device=arena.device)
    cfg = KrServeConfig(imgs, len(pool), ctypes.c_void_p(arena.data_ptr()), arena.numel() * arena.element_size(),
                        budget_bytes, max_batch, streams, policy,
                        ctypes.c_void_p(ws.data_ptr() if ws is not None else 0), ws_each,
                        1 if retain_outputs else 0, direct_px)
    res = (KrServeResult * len(arr))()
    torch.cuda.synchronize()
    _check(lib.kr_serve_run(arr, len(arr), ctypes.byref(cfg), res), "kr_serve_run")
    return res
