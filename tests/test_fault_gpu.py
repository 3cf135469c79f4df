"""Failure paths, exercised without faulting a GPU.

Device side: the tile kernels' first wait for a staged source box is given a zero bound
(kr_debug_set_stage_wait_ns(0)), so every staged tile records the timeout flag, waits with
the full bound for its copies to land and is abandoned. The kernels must return, the flag
must be readable, nothing outside the destination may change (every tile of these resizes is
staged, so nothing inside it changes either), and once the bound is back the same call must
be exact again.

Host side: kr_serve_run with injected failures (kr_debug_set_fault) of its launches, its
completion events and its arena allocations must finish, leave every request either
completed (its output equal to the request run alone) or dropped with its own status, and
never half-reported.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_2505_12425_gb300 import binding as kr
from paper_2505_12425_gb300 import inputs

pytestmark = pytest.mark.gpu
GUARD = 0xA5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()
    kr.load()


def dev():
    return torch.device("cuda:0")


def guarded(h, w, C, g=64):
    """An h x w x C u8 destination inside a buffer with g guard bytes (and g/3 guard rows)
    around it, everything filled with GUARD. Returns (buffer, view)."""
    pitch = w * C + 2 * g
    rows = h + 2 * (g // 3)
    buf = torch.full((rows * pitch,), GUARD, dtype=torch.uint8, device=dev())
    off = (g // 3) * pitch + g
    view = torch.as_strided(buf, (h, w, C), (pitch, C, 1), storage_offset=off)
    return buf, view


def pitched(img):
    """A device copy of img whose rows start 64-byte aligned (staged by bulk row copies in
    the ragged kernels)."""
    H, W, C = img.shape
    pitch = (W * C + 63) // 64 * 64
    buf = torch.zeros((H * pitch,), dtype=torch.uint8, device=dev())
    v = torch.as_strided(buf, (H, W, C), (pitch, C, 1))
    v.copy_(torch.from_numpy(img).to(dev()))
    return v


@pytest.fixture
def zero_first_wait():
    kr.kr_device_errors(clear=True)
    kr.kr_debug_set_stage_wait_ns(0)
    try:
        yield
    finally:
        kr.kr_debug_set_stage_wait_ns(kr.KR_STAGE_WAIT_NS_DEFAULT)


def test_single_image_wait_that_runs_out(zero_first_wait):
    img = inputs.noise_gradient_image(42, 1080, 1920, 3)
    src = torch.from_numpy(img).to(dev())
    buf, dst = guarded(720, 1280, 3)
    kr.kr_resize_bilinear(src, dst)
    torch.cuda.synchronize()
    assert kr.kr_device_errors() & kr_timeout_bit()
    assert bool((buf == GUARD).all())           # every tile abandoned, nothing written anywhere
    kr.kr_debug_set_stage_wait_ns(kr.KR_STAGE_WAIT_NS_DEFAULT)
    kr.kr_resize_bilinear(src, dst)
    torch.cuda.synchronize()
    assert kr.kr_device_errors() == 0
    np.testing.assert_array_equal(dst.cpu().numpy(), oracle.resize_u8(img, 720, 1280))
    inner = torch.zeros_like(buf, dtype=torch.bool)
    torch.as_strided(inner, dst.shape, dst.stride(), dst.storage_offset()).fill_(True)
    assert bool((buf[~inner] == GUARD).all())    # the guard bands around it are intact


def kr_timeout_bit():
    return 1   # KR_DEVERR_TMA_TIMEOUT


@pytest.mark.parametrize("tile_config", [0, 1])
def test_ragged_wait_that_runs_out(zero_first_wait, tile_config):
    rng = np.random.default_rng(8)
    imgs, srcs, bufs, dsts, work = [], [], [], [], []
    for i in range(6):
        H, W = int(rng.integers(100, 400)), int(rng.integers(100, 400))
        img = inputs.uniform_image(900 + i, H, W, 3)
        h, w = max(8, H * 2 // 3), max(8, W * 3 // 4)
        buf, d = guarded(h, w, 3)
        s = pitched(img)
        imgs.append(img)
        srcs.append(s)
        bufs.append(buf)
        dsts.append(d)
        work.append(kr.work_item(kr.KR_OP_RESIZE, s, d))
    ws = torch.empty(kr.kr_batch_workspace_size(len(work)), dtype=torch.uint8, device=dev())
    arr = kr.work_array(work)
    kr.kr_batch_submit(arr, ws, tile_config=tile_config)
    torch.cuda.synchronize()
    assert kr.kr_device_errors() & kr_timeout_bit()
    for buf in bufs:
        assert bool((buf == GUARD).all())
    kr.kr_debug_set_stage_wait_ns(kr.KR_STAGE_WAIT_NS_DEFAULT)
    kr.kr_batch_submit(arr, ws, tile_config=tile_config)
    torch.cuda.synchronize()
    assert kr.kr_device_errors() == 0
    for img, d, buf in zip(imgs, dsts, bufs):
        np.testing.assert_array_equal(d.cpu().numpy(), oracle.resize_u8(img, d.shape[0], d.shape[1]))
        inner = torch.zeros_like(buf, dtype=torch.bool)
        torch.as_strided(inner, d.shape, d.stride(), d.storage_offset()).fill_(True)
        assert bool((buf[~inner] == GUARD).all())


def _pool(n=6, seed=31):
    out = []
    for i, (H, W) in enumerate(inputs.pool_sizes(seed, n)):
        H, W = max(8, H // 4), max(8, W // 4)
        out.append(torch.from_numpy(inputs.uniform_image(seed * 100 + i, H, W, 3)).to(dev()))
    return out


def _requests(pool, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for r in inputs.request_stream(seed, 20000.0, 0.004, pool=len(pool)):
        H, W = pool[r.src_index].shape[:2]
        if r.op == inputs.OP_RESIZE:
            k = rng.uniform(0.25, 2.0)
            r.h, r.w = max(1, round(k * H)), max(1, round(k * W))
        elif r.op == inputs.OP_WARP:
            r.h, r.w = H, W
            r.M = inputs.random_inverse_affine(rng, H, W)
        else:
            r.h, r.w = H, W
        reqs.append(r)
    return reqs


def _alone(r, src):
    dC = 1 if r.op == inputs.OP_GRAY else 3
    out = torch.empty((r.h, r.w, dC), dtype=torch.uint8, device=src.device)
    if r.op == inputs.OP_RESIZE:
        kr.kr_resize_bilinear(src, out)
    elif r.op == inputs.OP_WARP:
        kr.kr_warp_affine(src, out, r.M)
    else:
        kr.kr_rgb_to_gray(src, out)
    return out


@pytest.mark.parametrize("policy", [0, 1, 2])
@pytest.mark.parametrize("site", [kr.KR_FAULT_SUBMIT, kr.KR_FAULT_EVENT, kr.KR_FAULT_ADMIT])
def test_serving_with_injected_host_failures(site, policy):
    pool = _pool()
    reqs = _requests(pool, 40 + policy)
    assert len(reqs) >= 30
    arena = torch.empty(1 << 30, dtype=torch.uint8, device=dev())
    kr.kr_debug_set_fault(site, 3)
    try:
        res = kr.kr_serve_run(reqs, pool, arena, budget_bytes=1 << 30, max_batch=8, streams=2, policy=policy,
                              retain_outputs=True, direct_px=3000 if policy == 2 else 0)
    finally:
        kr.kr_debug_set_fault(site, 0)
    dropped = 0
    for i, r in enumerate(reqs):
        if res[i].status == 0:
            assert res[i].t_done >= res[i].t_launch >= res[i].t_admit >= 0
            dC = 1 if r.op == inputs.OP_GRAY else 3
            off = int(res[i].out_offset)
            got = arena[off:off + r.h * r.w * dC].view(r.h, r.w, dC)
            assert torch.equal(got, _alone(r, pool[r.src_index])), i
        else:
            dropped += 1
            assert res[i].status == 4          # KR_ERR_CUDA: the injected launch failure
            assert res[i].t_done == -1.0 and res[i].out_offset == -1 and res[i].t_launch == -1.0
    if site == kr.KR_FAULT_SUBMIT:
        assert 0 < dropped < len(reqs)
    else:
        assert dropped == 0                    # events: waited for; admission: retried
