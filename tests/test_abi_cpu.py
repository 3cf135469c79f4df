"""C-ABI checks that need no GPU: the library loads, exports every entry point
that include/kr.h declares, and rejects bad arguments on the host before
anything is enqueued (so no CUDA call is made on these paths)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

import __graft_entry__ as ge
from paper_2505_12425_gb300 import binding as kr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    ge.build()
    return kr.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "kr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kr_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layouts_match_header():
    assert ctypes.sizeof(kr.KrImage) == 56
    assert kr.KrImage.pitch.offset == 32
    assert ctypes.sizeof(kr.KrPost) == 28
    assert ctypes.sizeof(kr.KrWork) == 4 + 4 + 56 + 56 + 24 + 28 + 4


def _img(data=0x10000, h=4, w=5, c=3, dtype=kr.KR_U8, layout=kr.KR_HWC, batch=1, pitch=None,
         plane=0, bstride=0):
    im = kr.KrImage()
    im.data = data
    im.height, im.width, im.channels = h, w, c
    im.dtype, im.layout, im.batch = dtype, layout, batch
    es = 4 if dtype == kr.KR_F32 else 1
    im.pitch = pitch if pitch is not None else (w * es if layout == kr.KR_CHW else w * c * es)
    im.plane_stride = plane
    im.batch_stride = bstride
    return im


def _resize(lib, s, d, p=None):
    return lib.kr_resize_bilinear(ctypes.byref(s), ctypes.byref(d), ctypes.byref(p) if p else None, None)


@pytest.mark.parametrize("bad", [
    dict(data=0), dict(h=0), dict(w=-1), dict(c=2), dict(c=4), dict(dtype=7), dict(pitch=14),
    dict(batch=0), dict(batch=65536, bstride=60), dict(h=70000)])
def test_resize_rejects_bad_source(lib, bad):
    s = _img(**bad)
    d = _img(data=0x900000, h=2, w=2)
    assert _resize(lib, s, d) == 1


def test_resize_rejects_alias_and_mismatches(lib):
    s = _img(data=0x10000, h=10, w=10)
    assert _resize(lib, s, _img(data=0x10000 + 30, h=2, w=2)) == 3          # overlap
    assert _resize(lib, s, _img(data=0x900000, h=2, w=2, c=1)) == 1         # channel mismatch
    g = kr.post(gray=True)
    assert _resize(lib, _img(c=1), _img(data=0x900000, c=1), g) == 1        # gray needs RGB
    n = kr.post(mean=(0.5, 0.5, 0.5), std=(0.2, 0.2, 0.2))
    assert _resize(lib, s, _img(data=0x900000), n) == 1                     # normalise needs f32
    z = kr.post(mean=(0.5, 0.5, 0.5), std=(0.0, 1.0, 1.0))
    assert _resize(lib, s, _img(data=0x900000, dtype=kr.KR_F32), z) == 1    # std 0
    assert _resize(lib, s, _img(data=0x900000, layout=kr.KR_CHW, plane=4 * 20)) == 2  # CHW u8
    assert _resize(lib, _img(dtype=kr.KR_F32), _img(data=0x900000)) == 2    # f32 source
    assert _resize(lib, _img(batch=2, bstride=60), _img(data=0x900000, batch=3, bstride=60)) == 1
    # destination images of a batch may not overlap
    assert _resize(lib, _img(batch=2, bstride=60), _img(data=0x900000, batch=2, bstride=10)) == 1
    # unaligned f32 destination
    assert _resize(lib, s, _img(data=0x900002, dtype=kr.KR_F32)) == 1
    bad_flags = kr.KrPost()
    bad_flags.flags = 8
    assert _resize(lib, s, _img(data=0x900000), bad_flags) == 1


def test_warp_rejects_nonfinite_matrix(lib):
    s, d = _img(), _img(data=0x900000)
    p = kr.post()
    for M in ([float("nan"), 0, 0, 0, 1, 0], [1, 0, float("inf"), 0, 1, 0]):
        a = (ctypes.c_float * 6)(*M)
        assert lib.kr_warp_affine(ctypes.byref(s), ctypes.byref(d), a, ctypes.byref(p), None) == 1
    assert lib.kr_warp_affine(ctypes.byref(s), ctypes.byref(d), None, ctypes.byref(p), None) == 1


def test_replicate_border_is_for_warps_only(lib):
    s, d = _img(), _img(data=0x900000)
    p = kr.post(border="replicate")
    assert _resize(lib, s, d, p) == 1
    with pytest.raises(ValueError):
        kr.post(border="reflect")


def test_perspective_rejects_bad_maps(lib):
    s, d, p = _img(), _img(data=0x900000), kr.KrPost()
    assert lib.kr_warp_perspective(ctypes.byref(s), ctypes.byref(d), None, ctypes.byref(p), None) == 1
    for k in (0, 5, 8):
        M = [1, 0, 0, 0, 1, 0, 0, 0, 1]
        M[k] = float("nan")
        a = (ctypes.c_float * 9)(*M)
        assert lib.kr_warp_perspective(ctypes.byref(s), ctypes.byref(d), a, ctypes.byref(p), None) == 1
    a = (ctypes.c_float * 9)(1, 0, 0, 0, 1, 0, 0, 0, 1)
    assert lib.kr_warp_perspective(ctypes.byref(s), ctypes.byref(_img(data=0x10001)), a, ctypes.byref(p), None) == 3


def test_area_rejects_upscale_and_gray(lib):
    s = _img(h=4, w=5)
    assert lib.kr_resize_area(ctypes.byref(s), ctypes.byref(_img(data=0x900000, h=5, w=5)), None, None) == 1
    p = kr.post(gray=True)
    d = _img(data=0x900000, h=2, w=2, c=1)
    assert lib.kr_resize_area(ctypes.byref(s), ctypes.byref(d), ctypes.byref(p), None) == 2


def test_area_footprint_too_wide_is_unsupported(lib):
    # one output column over 65535 source columns: two ring slots of its footprint row exceed
    # the shared-memory budget, reported before anything is launched
    s = _img(h=1, w=65535)
    d = _img(data=0x900000, h=1, w=1)
    assert lib.kr_resize_area(ctypes.byref(s), ctypes.byref(d), None, None) == 2


def test_sobel_rejects_bad_arguments(lib):
    s = _img()
    d = _img(data=0x900000, c=1)
    assert lib.kr_sobel(ctypes.byref(s), ctypes.byref(d), 5, None) == 2          # only 3 x 3
    assert lib.kr_sobel(ctypes.byref(s), ctypes.byref(_img(data=0x900000, c=3)), 3, None) == 1
    assert lib.kr_sobel(ctypes.byref(s), ctypes.byref(_img(data=0x900000, c=1, w=4)), 3, None) == 1
    assert lib.kr_sobel(ctypes.byref(s), ctypes.byref(_img(data=0x10001, c=1)), 3, None) == 3


def test_gathers_reject_bad_shapes(lib):
    s = _img()
    for f in (lib.kr_resize_nearest, lib.kr_flip_horizontal):
        assert f(ctypes.byref(s), ctypes.byref(_img(data=0x900000, c=1)), None) == 1       # channels differ
        assert f(ctypes.byref(s), ctypes.byref(_img(data=0x10001, c=3)), None) == 3        # overlap
        assert f(None, ctypes.byref(_img(data=0x900000, c=3)), None) == 1
    assert lib.kr_flip_horizontal(ctypes.byref(s), ctypes.byref(_img(data=0x900000, c=3, w=4)), None) == 1
    f32 = _img(data=0x900000, c=3, dtype=kr.KR_F32)
    assert lib.kr_resize_nearest(ctypes.byref(s), ctypes.byref(f32), None) == 2


def test_gray_rejects_bad_shapes(lib):
    s = _img()
    assert lib.kr_rgb_to_gray(ctypes.byref(s), ctypes.byref(_img(data=0x900000, c=3)), None) == 1
    assert lib.kr_rgb_to_gray(ctypes.byref(s), ctypes.byref(_img(data=0x900000, c=1, w=4)), None) == 1
    assert lib.kr_rgb_to_gray(ctypes.byref(s), ctypes.byref(_img(data=0x10001, c=1)), None) == 3


def test_batch_host_checks(lib):
    assert lib.kr_batch_workspace_size(1) >= 512 + 128
    assert lib.kr_batch_workspace_size(256) == 512 + 256 * 128 + ((257 * 4 + 15) // 16) * 16
    items = (kr.KrWork * 2)()
    # n == 0 is a no-op
    assert lib.kr_batch_submit(items, 0, None, 0, None, None) == 0
    # too small a workspace
    assert lib.kr_batch_submit(items, 2, ctypes.c_void_p(0x1000), 16, None, None) == 5
    # invalid item (zero-initialised descriptors)
    ws = lib.kr_batch_workspace_size(2)
    assert lib.kr_batch_submit(items, 2, ctypes.c_void_p(0x1000), ws, None, None) == 1
    # bad option
    o = kr.KrBatchOpts(99, 0, 0)
    assert lib.kr_batch_submit(items, 2, ctypes.c_void_p(0x1000), ws, ctypes.byref(o), None) == 1
    assert lib.kr_tile_config_count() >= 2
    tw, th = ctypes.c_int32(), ctypes.c_int32()
    assert lib.kr_tile_config_shape(0, ctypes.byref(tw), ctypes.byref(th)) == 0 and tw.value % 32 == 0
    assert lib.kr_tile_config_shape(99, ctypes.byref(tw), ctypes.byref(th)) == 1


def test_status_strings(lib):
    for s in range(7):
        assert lib.kr_status_string(s)
    assert lib.kr_status_string(99) == b"unknown status"


def test_autotune_cache_roundtrip(lib, tmp_path):
    p = tmp_path / "tune.json"
    p.write_text('{"entries": [\n  {"key": "GPU|n2^3|px2^20|ops2", "tile_config": 1, "ctas_per_sm": 2}\n]}\n')
    assert lib.kr_autotune_load(str(p).encode()) == 0
    q = tmp_path / "out.json"
    assert lib.kr_autotune_save(str(q).encode()) == 0
    assert '"tile_config": 1' in q.read_text() and "GPU|n2^3|px2^20|ops2" in q.read_text()
    bad = tmp_path / "bad.json"
    bad.write_text('{"entries": [{"key": "x", "tile_config": 42, "ctas_per_sm": 1}]}')
    assert lib.kr_autotune_load(str(bad).encode()) == 1
    lib.kr_shutdown()
