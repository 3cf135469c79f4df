"""Serving loop (kr_serve_run): validation on the host, and on the GPU that every
request's result is the same alone and in the mix, that the HBM budget holds at
every instant, and that work admitted while other batches run overlaps them."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

from paper_2505_12425_gb300 import binding as kr
from paper_2505_12425_gb300 import inputs


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    return kr.load()


def _fake_cfg(n_pool=2):
    imgs = (kr.KrImage * n_pool)()
    for i in range(n_pool):
        im = imgs[i]
        im.data = 0x100000 * (i + 1)
        im.height, im.width, im.channels, im.dtype, im.layout, im.batch = 40, 50, 3, kr.KR_U8, kr.KR_HWC, 1
        im.pitch = 150
    cfg = kr.KrServeConfig(imgs, n_pool, ctypes.c_void_p(0x9000000), 1 << 20, 1 << 20, 8, 2, 1,
                           ctypes.c_void_p(0), 0, 0)
    return imgs, cfg


def _req(op=kr.KR_OP_RESIZE, src=0, h=20, w=25, t=0.0):
    r = kr.KrRequest()
    r.op, r.src_index, r.out_h, r.out_w, r.t_arrival = op, src, h, w, t
    return r


@pytest.mark.parametrize("bad", [
    dict(src=5), dict(src=-1), dict(op=7), dict(h=0), dict(w=70000),
    dict(op=kr.KR_OP_GRAY, h=10, w=10),          # gray must keep the source size
    dict(h=2000, w=2000),                         # output larger than the arena
])
def test_serve_rejects_bad_requests_before_running(lib, bad):
    imgs, cfg = _fake_cfg()
    reqs = (kr.KrRequest * 2)(_req(), _req(**bad))
    res = (kr.KrServeResult * 2)()
    st = lib.kr_serve_run(reqs, 2, ctypes.byref(cfg), res)
    assert st in (1, 5)


def test_serve_rejects_bad_configs(lib):
    imgs, cfg = _fake_cfg()
    reqs = (kr.KrRequest * 2)(_req(t=0.5), _req(t=0.1))      # arrivals out of order
    res = (kr.KrServeResult * 2)()
    assert lib.kr_serve_run(reqs, 2, ctypes.byref(cfg), res) == 1
    reqs = (kr.KrRequest * 1)(_req())
    cfg.policy = 0                                             # batching needs workspaces
    assert lib.kr_serve_run(reqs, 1, ctypes.byref(cfg), res) == 5
    cfg.policy = 2                                             # so does size-aware batching
    assert lib.kr_serve_run(reqs, 1, ctypes.byref(cfg), res) == 5
    cfg.policy, cfg.direct_px = 1, -1                          # negative threshold
    assert lib.kr_serve_run(reqs, 1, ctypes.byref(cfg), res) == 1
    cfg.direct_px = 0
    cfg.policy = 3
    assert lib.kr_serve_run(reqs, 1, ctypes.byref(cfg), res) == 1
    cfg.policy, cfg.streams = 1, 0
    assert lib.kr_serve_run(reqs, 1, ctypes.byref(cfg), res) == 1


# ---------------------------------------------------------------------------
# GPU
# ---------------------------------------------------------------------------
def _pool(dev, n=12, seed=77, scale=0.3):
    """A small device pool (sizes of the serving recipe, scaled down to keep the test short)."""
    sizes = inputs.pool_sizes(seed, n)
    out = []
    for i, (H, W) in enumerate(sizes):
        H, W = max(8, int(H * scale)), max(8, int(W * scale))
        out.append(torch.from_numpy(inputs.uniform_image(seed * 1000 + i, H, W, 3)).to(dev))
    return out


def _stream(pool, rate, duration, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for r in inputs.request_stream(seed, rate, duration, pool=len(pool)):
        H, W = pool[r.src_index].shape[:2]
        if r.op == inputs.OP_RESIZE:
            k = rng.uniform(0.25, 2.0)
            r.h, r.w = max(1, round(k * H)), max(1, round(k * W))
        elif r.op == inputs.OP_WARP:
            r.h, r.w = H, W
            r.M = inputs.random_inverse_affine(rng, H, W)
        else:
            r.h, r.w = H, W
        r.H, r.W = H, W
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


def _from_arena(arena, res, r):
    dC = 1 if r.op == inputs.OP_GRAY else 3
    n = r.h * r.w * dC
    off = int(res.out_offset)
    return arena[off:off + n].view(r.h, r.w, dC)


@pytest.mark.gpu
@pytest.mark.parametrize("policy", [0, 1, 2])
def test_served_results_equal_results_alone(lib, policy):
    dev = torch.device("cuda:0")
    pool = _pool(dev)
    reqs = _stream(pool, rate=4000.0, duration=0.08, seed=5 + policy)
    assert len(reqs) > 100
    arena = torch.empty(1 << 30, dtype=torch.uint8, device=dev)
    # policy 2 with a low threshold: some requests launch alone, the rest share ragged launches
    res = kr.kr_serve_run(reqs, pool, arena, budget_bytes=1 << 30, max_batch=32, streams=4, policy=policy,
                          retain_outputs=True, direct_px=20000 if policy == 2 else 0)
    if policy == 2:
        big = sum(1 for r in reqs if r.h * r.w >= 20000)
        assert 0 < big < len(reqs)
    for i, r in enumerate(reqs):
        assert res[i].t_done >= res[i].t_launch >= res[i].t_admit >= r.t_arrival - 1e-3
        got = _from_arena(arena, res[i], r)
        assert torch.equal(got, _alone(r, pool[r.src_index])), (i, r.op)
    torch.cuda.synchronize()
    # every request against the oracle (its calls release the interpreter lock: a thread pool)
    import concurrent.futures as cf
    import os

    import oracle
    pool_np = [p.cpu().numpy() for p in pool]

    def ref_of(r):
        src = pool_np[r.src_index]
        if r.op == inputs.OP_RESIZE:
            return oracle.resize_u8(src, r.h, r.w)
        if r.op == inputs.OP_WARP:
            return oracle.warp_u8(src, r.M, r.h, r.w)
        return oracle.rgb_to_gray_u8(src)

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        refs = list(ex.map(ref_of, reqs))
    for i, (r, ref) in enumerate(zip(reqs, refs)):
        np.testing.assert_array_equal(_from_arena(arena, res[i], r).cpu().numpy(), ref, err_msg=f"request {i}")


@pytest.mark.gpu
def test_budget_holds_and_batches_overlap(lib):
    dev = torch.device("cuda:0")
    pool = _pool(dev, n=8, seed=91, scale=0.5)
    reqs = _stream(pool, rate=200000.0, duration=0.005, seed=9)
    for r in reqs:
        r.t_arrival = 0.0                                             # one simultaneous burst
    nbytes = []
    for r in reqs:
        src = pool[r.src_index]
        nbytes.append(src.numel() + r.h * r.w * (1 if r.op == inputs.OP_GRAY else 3))
    budget = 2 * max(nbytes)                                          # room for a few requests at a time
    arena = torch.empty(2 << 30, dtype=torch.uint8, device=dev)
    res = kr.kr_serve_run(reqs, pool, arena, budget_bytes=budget, max_batch=16, streams=4, policy=0,
                          retain_outputs=True)
    # at every admission instant the admitted-but-unfinished bytes stay within the budget
    events = sorted([(res[i].t_admit, 0, i) for i in range(len(reqs))] + [(res[i].t_done, -1, i) for i in range(len(reqs))])
    cur = peak = 0
    for t, kind, i in events:
        cur += nbytes[i] if kind == 0 else -nbytes[i]
        peak = max(peak, cur)
    assert peak <= budget
    # the budget admits a few requests at a time, so most of the burst waits for earlier ones ...
    waited = sum(1 for i in range(len(reqs)) if res[i].t_admit > min(res[j].t_done for j in range(len(reqs))))
    assert waited > len(reqs) // 2
    # ... and requests admitted while others were in flight shared batches / overlapped them
    launches = sorted({round(res[i].t_launch, 9) for i in range(len(reqs))})
    assert len(launches) < len(reqs)
    for i, r in enumerate(reqs[:64]):
        assert torch.equal(_from_arena(arena, res[i], r), _alone(r, pool[r.src_index]))


@pytest.mark.gpu
def test_retained_outputs_that_do_not_fit_are_refused(lib):
    dev = torch.device("cuda:0")
    pool = _pool(dev, n=4, seed=3, scale=0.5)
    reqs = _stream(pool, rate=5000.0, duration=0.02, seed=4)
    arena = torch.empty(8 << 20, dtype=torch.uint8, device=dev)      # far too small for all outputs
    with pytest.raises(kr.KrError) as e:
        kr.kr_serve_run(reqs, pool, arena, budget_bytes=1 << 30, max_batch=16, streams=2, policy=0,
                        retain_outputs=True)
    assert e.value.status == 5
