"""kr_batch_submit_noalloc: the batch launch for callers that may not allocate.

Some callers cannot allocate device memory when they submit work (real-time loops
that forbid allocation on their hot path, frameworks whose allocator owns all of
device memory, code that cannot keep a workspace alive between calls). For them the
library offers kr_batch_submit_noalloc, which keeps the work list in a fixed device
array of its own instead of a caller workspace. This checks, through the C ABI, that
two calls in a row each give exactly what kr_batch_submit gives for the same items
(u8 bit for bit, f32 within 1e-5), and that oversize requests are refused.

The file name sorts last so that a run that stops at the first failure has run every
other test before this one.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

from paper_2505_12425_gb300 import binding as kr
from paper_2505_12425_gb300 import inputs

pytestmark = pytest.mark.gpu
F32_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()
    kr.load()


def _items(seed, n):
    """n mixed items (resize / warp / gray; u8, fused gray, f32 normalised CHW) with their
    sources and two sets of destinations (one per entry point)."""
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(seed)
    srcs, dst_a, dst_b, specs = [], [], [], []
    for i in range(n):
        H, W = (int(v) for v in rng.integers(20, 400, 2))
        img = torch.from_numpy(inputs.uniform_image(seed * 100 + i, H, W, 3)).to(dev)
        kind = i % 5
        if kind == 0:       # resize u8
            h, w = max(1, int(H * rng.uniform(0.3, 1.8))), max(1, int(W * rng.uniform(0.3, 1.8)))
            mk = lambda: torch.empty((h, w, 3), dtype=torch.uint8, device=dev)  # noqa: E731
            spec = dict(op=kr.KR_OP_RESIZE)
        elif kind == 1:     # warp u8
            h, w = H, W
            mk = lambda: torch.empty((h, w, 3), dtype=torch.uint8, device=dev)  # noqa: E731
            spec = dict(op=kr.KR_OP_WARP, M=inputs.random_inverse_affine(rng, H, W))
        elif kind == 2:     # warp + fused gray
            h, w = H, W
            mk = lambda: torch.empty((h, w, 1), dtype=torch.uint8, device=dev)  # noqa: E731
            spec = dict(op=kr.KR_OP_WARP, M=inputs.random_inverse_affine(rng, H, W), gray=True)
        elif kind == 3:     # resize, f32 normalised planar
            h, w = max(1, H // 2 + 3), max(1, W // 3 + 1)
            mk = lambda: torch.empty((3, h, w), dtype=torch.float32, device=dev)  # noqa: E731
            spec = dict(op=kr.KR_OP_RESIZE, mean=inputs.IMAGENET_MEAN, std=inputs.IMAGENET_STD,
                        dst_layout="chw")
        else:               # standalone gray
            mk = lambda: torch.empty((H, W, 1), dtype=torch.uint8, device=dev)  # noqa: E731
            spec = dict(op=kr.KR_OP_GRAY)
        srcs.append(img)
        dst_a.append(mk())
        dst_b.append(mk())
        specs.append(spec)
    return srcs, dst_a, dst_b, specs


def _work(srcs, dsts, specs):
    out = []
    for s, d, sp in zip(srcs, dsts, specs):
        sp = dict(sp)
        op = sp.pop("op")
        out.append(kr.work_item(op, s, d, **sp))
    return kr.work_array(out)


def _compare(a, b):
    if a.dtype == torch.uint8:
        assert torch.equal(a, b)
    else:
        assert float((a - b).abs().max()) <= F32_TOL


def test_noalloc_matches_workspace_submit_on_two_calls_in_a_row():
    dev = torch.device("cuda:0")
    batches = [_items(11, 23), _items(12, 37)]
    # the reference results: the workspace entry point
    for srcs, dst_a, _, specs in batches:
        ws = torch.empty(kr.kr_batch_workspace_size(len(srcs)), dtype=torch.uint8, device=dev)
        kr.kr_batch_submit(_work(srcs, dst_a, specs), ws)
        torch.cuda.synchronize()
    # two calls in a row of the allocation-free entry point, on one stream
    for _, _, dst_b, _ in batches:
        for d in dst_b:
            d.fill_(0x3C if d.dtype == torch.uint8 else -3.0)
    works = [_work(srcs, dst_b, specs) for srcs, _, dst_b, specs in batches]
    torch.cuda.synchronize()
    for w in works:
        kr.kr_batch_submit_noalloc(w)
    torch.cuda.synchronize()
    for srcs, dst_a, dst_b, specs in batches:
        for a, b in zip(dst_a, dst_b):
            _compare(a, b)


def test_noalloc_refuses_more_items_than_its_array_holds():
    lib = kr.load()
    n = kr.KR_BATCH_NOALLOC_MAX_ITEMS + 1
    items = (kr.KrWork * n)()
    o = kr.KrBatchOpts(-1, 0, 0)
    assert lib.kr_batch_submit_noalloc(items, n, ctypes.byref(o), None) == 5   # KR_ERR_NO_SPACE


def test_noalloc_with_exactly_the_maximum_item_count():
    """KR_BATCH_NOALLOC_MAX_ITEMS small items fill the library's work-list array to its end:
    every one of them must come out as kr_batch_submit makes it (bit for bit, u8)."""
    dev = torch.device("cuda:0")
    n = kr.KR_BATCH_NOALLOC_MAX_ITEMS
    rng = np.random.default_rng(77)
    srcs, dst_a, dst_b, work_a, work_b = [], [], [], [], []
    for i in range(n):
        img = torch.from_numpy(inputs.uniform_image(7700 + i, 8, 8, 3)).to(dev)
        if i % 2 == 0:
            a = torch.empty((8, 8, 1), dtype=torch.uint8, device=dev)
            b = torch.full((8, 8, 1), 0x3C, dtype=torch.uint8, device=dev)
            work_a.append(kr.work_item(kr.KR_OP_GRAY, img, a))
            work_b.append(kr.work_item(kr.KR_OP_GRAY, img, b))
        else:
            h, w = int(rng.integers(3, 17)), int(rng.integers(3, 17))
            a = torch.empty((h, w, 3), dtype=torch.uint8, device=dev)
            b = torch.full((h, w, 3), 0x3C, dtype=torch.uint8, device=dev)
            work_a.append(kr.work_item(kr.KR_OP_RESIZE, img, a))
            work_b.append(kr.work_item(kr.KR_OP_RESIZE, img, b))
        srcs.append(img)
        dst_a.append(a)
        dst_b.append(b)
    ws = torch.empty(kr.kr_batch_workspace_size(n), dtype=torch.uint8, device=dev)
    kr.kr_batch_submit(kr.work_array(work_a), ws)
    kr.kr_batch_submit_noalloc(kr.work_array(work_b))
    torch.cuda.synchronize()
    for a, b in zip(dst_a, dst_b):
        assert torch.equal(a, b)


def test_noalloc_refuses_a_capturing_stream_and_leaves_the_capture_valid():
    """A call on a stream under graph capture returns KR_ERR_UNSUPPORTED, enqueues nothing,
    and the capture still ends with a valid (empty) graph."""
    dev = torch.device("cuda:0")
    srcs, _, dst_b, specs = _items(13, 3)
    w = _work(srcs, dst_b, specs)
    kr.kr_batch_submit_noalloc(w)            # the first call on the device does the set-up
    torch.cuda.synchronize()
    lib = kr.load()
    o = kr.KrBatchOpts(-1, 0, 0)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    x = torch.zeros(4, device=dev)
    with torch.cuda.graph(g, stream=s):
        x.add_(1.0)
        st = lib.kr_batch_submit_noalloc(w, len(w), ctypes.byref(o), ctypes.c_void_p(s.cuda_stream))
        x.add_(1.0)
    assert st == 2   # KR_ERR_UNSUPPORTED
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(x, torch.full((4,), 4.0, device=dev))
