"""GPU parity of the ragged batch launch (kr_batch_submit).

Every item of a batch must equal the matching single-image call bit for bit
(u8 and f32 alike: same tile engine, same arithmetic) and the oracle (bit-exact
u8, <= 1e-5 f32), for every tile configuration, with and without CUDA-graph
replay, and for back-to-back submits that reuse the staging ring.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_2505_12425_gb300 import binding as kr
from paper_2505_12425_gb300 import inputs

pytestmark = pytest.mark.gpu
F32_TOL = 1e-5
MEAN, STD = inputs.IMAGENET_MEAN, inputs.IMAGENET_STD


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()
    kr.load()


def dev():
    return torch.device("cuda:0")


def make_mixed(seed, n, lo=8, hi=300):
    """n items cycling through every (op, output kind) the batch path runs."""
    kinds = [("resize", "u8"), ("warp", "u8"), ("gray", "u8"), ("resize", "u8g"), ("warp", "f32chw"),
             ("resize", "f32"), ("warp", "u8g"), ("resize", "f32g"), ("warp", "c1"), ("resize", "c1f32")]
    rng = np.random.default_rng(seed)
    items = []
    for i in range(n):
        op, kind = kinds[i % len(kinds)]
        H, W = (int(v) for v in np.exp(rng.uniform(np.log(lo), np.log(hi), 2)).round())
        C = 1 if kind.startswith("c1") else 3
        img = inputs.uniform_image(seed * 1000 + i, H, W, C)
        if op == "gray":
            h, w, M = H, W, None
        elif op == "resize":
            k = rng.uniform(0.25, 2.0)
            h, w, M = max(1, round(k * H)), max(1, round(k * W)), None
        else:
            k = rng.uniform(0.5, 1.5)
            h, w = max(1, round(k * H)), max(1, round(k * W))
            M = inputs.random_inverse_affine(rng, H, W, h, w, k)
        items.append(dict(op=op, kind=kind, img=img, h=h, w=w, M=M, C=C))
    return items


def alloc_dst(it):
    h, w, C, kind = it["h"], it["w"], it["C"], it["kind"]
    if it["op"] == "gray" or kind in ("u8g",):
        return torch.empty((h, w, 1), dtype=torch.uint8, device=dev()), "hwc"
    if kind in ("u8", "c1"):
        return torch.empty((h, w, C), dtype=torch.uint8, device=dev()), "hwc"
    if kind == "f32chw":
        return torch.empty((3, h, w), dtype=torch.float32, device=dev()), "chw"
    if kind == "f32g":
        return torch.empty((h, w, 1), dtype=torch.float32, device=dev()), "hwc"
    return torch.empty((h, w, C), dtype=torch.float32, device=dev()), "hwc"


def post_of(it):
    kind = it["kind"]
    gray = kind in ("u8g", "f32g")
    norm = kind in ("f32chw", "f32g")
    return dict(gray=gray, mean=MEAN if norm else None, std=STD if norm else None)


def work_of(it, src, dst, layout):
    op = {"resize": kr.KR_OP_RESIZE, "warp": kr.KR_OP_WARP, "gray": kr.KR_OP_GRAY}[it["op"]]
    return kr.work_item(op, src, dst, M=it["M"], dst_layout=layout, **post_of(it))


def single_call(it, src, dst, layout):
    p = post_of(it)
    if it["op"] == "gray":
        kr.kr_rgb_to_gray(src, dst)
    elif it["op"] == "resize":
        kr.kr_resize_bilinear(src, dst, dst_layout=layout, **p)
    else:
        kr.kr_warp_affine(src, dst, it["M"], dst_layout=layout, **p)


def oracle_of(it):
    img, h, w, p = it["img"], it["h"], it["w"], post_of(it)
    kind = it["kind"]
    if it["op"] == "gray":
        return oracle.rgb_to_gray_u8(img)
    f32 = kind.startswith("f32") or kind == "c1f32" or kind == "f32"
    if it["op"] == "resize":
        if f32:
            return oracle.resize_f64(img, h, w, gray=p["gray"], mean=p["mean"], std=p["std"])
        return oracle.resize_u8(img, h, w, gray=p["gray"])
    if f32:
        return oracle.warp_f64(img, it["M"], h, w, gray=p["gray"], mean=p["mean"], std=p["std"])
    return oracle.warp_u8(img, it["M"], h, w, gray=p["gray"])


def as_hwc(t, layout):
    a = t.cpu().numpy()
    return a.transpose(1, 2, 0) if layout == "chw" else a


def to_src(img, pitched):
    """The image on the device: contiguous, or inside rows of a 64-byte multiple pitch whose
    padding holds 0xC3 (16-byte aligned rows: staged by bulk row copies)."""
    t = torch.from_numpy(img).to(dev())
    if not pitched:
        return t
    H, W, C = img.shape
    pitch = (W * C + 63) // 64 * 64
    buf = torch.full((H * pitch,), 0xC3, dtype=torch.uint8, device=dev())
    v = torch.as_strided(buf, (H, W, C), (pitch, C, 1))
    v.copy_(t)
    return v


def run_batch(items, tile_config=-1, use_graph=False, ctas=0, pitched=False):
    srcs = [to_src(it["img"], pitched) for it in items]
    dsts = [alloc_dst(it) for it in items]
    work = kr.work_array([work_of(it, s, d, l) for it, s, (d, l) in zip(items, srcs, dsts)])
    ws = torch.empty(kr.kr_batch_workspace_size(len(items)), dtype=torch.uint8, device=dev())
    for d, _ in dsts:
        d.fill_(0x5A if d.dtype == torch.uint8 else -7.0)
    kr.kr_batch_submit(work, ws, tile_config=tile_config, use_graph=use_graph, ctas_per_sm=ctas)
    torch.cuda.synchronize()
    return srcs, dsts


@pytest.mark.parametrize("pitched", [False, True])
def test_mixed_batch_matches_oracle_and_single_calls(pitched):
    items = make_mixed(1, 40)
    srcs, dsts = run_batch(items, pitched=pitched)
    for it, s, (d, l) in zip(items, srcs, dsts):
        ref = oracle_of(it)
        got = as_hwc(d, l)
        if d.dtype == torch.uint8:
            np.testing.assert_array_equal(got, ref)
        else:
            assert np.abs(got - ref).max() <= F32_TOL
        single = torch.empty_like(d)
        single_call(it, s, single, l)
        torch.cuda.synchronize()
        assert torch.equal(single, d), (it["op"], it["kind"])


@pytest.mark.parametrize("pitched", [False, True])
@pytest.mark.parametrize("use_graph", [False, True])
def test_every_tile_config(use_graph, pitched):
    items = make_mixed(2, 20)
    ref = None
    for cfg in range(kr.kr_tile_config_count()):
        for _ in range(2):      # second pass replays the graph
            _, dsts = run_batch(items, tile_config=cfg, use_graph=use_graph, pitched=pitched)
        outs = [d.cpu() for d, _ in dsts]
        if ref is None:
            ref = outs
            for it, (d, l) in zip(items, dsts):
                got, exp = as_hwc(d, l), oracle_of(it)
                if d.dtype == torch.uint8:
                    np.testing.assert_array_equal(got, exp)
                else:
                    assert np.abs(got - exp).max() <= F32_TOL
        else:
            for a, b in zip(ref, outs):
                assert torch.equal(a, b), cfg


def test_back_to_back_submits_reuse_staging():
    """Ten batches enqueued without a sync in between (graph replays with changing
    work lists): each must come out right."""
    ws = torch.empty(kr.kr_batch_workspace_size(8), dtype=torch.uint8, device=dev())
    jobs = []
    for b in range(10):
        items = make_mixed(100 + b, 3 + b % 6)
        srcs = [torch.from_numpy(it["img"]).to(dev()) for it in items]
        dsts = [alloc_dst(it) for it in items]
        work = kr.work_array([work_of(it, s, d, l) for it, s, (d, l) in zip(items, srcs, dsts)])
        jobs.append((items, srcs, dsts, work))
    torch.cuda.synchronize()
    for items, srcs, dsts, work in jobs:
        kr.kr_batch_submit(work, ws, use_graph=True)
    torch.cuda.synchronize()
    for items, srcs, dsts, work in jobs:
        for it, (d, l) in zip(items, dsts):
            got, exp = as_hwc(d, l), oracle_of(it)
            if d.dtype == torch.uint8:
                np.testing.assert_array_equal(got, exp)
            else:
                assert np.abs(got - exp).max() <= F32_TOL


def test_autotune_picks_a_valid_config():
    items = make_mixed(3, 16)
    srcs = [torch.from_numpy(it["img"]).to(dev()) for it in items]
    dsts = [alloc_dst(it) for it in items]
    work = kr.work_array([work_of(it, s, d, l) for it, s, (d, l) in zip(items, srcs, dsts)])
    ws = torch.empty(kr.kr_batch_workspace_size(len(items)), dtype=torch.uint8, device=dev())
    cfg, ctas = kr.kr_autotune_batch(work, ws)
    assert 0 <= cfg < kr.kr_tile_config_count() and ctas >= 1
    kr.kr_batch_submit(work, ws)          # uses the cached choice
    torch.cuda.synchronize()
    for it, (d, l) in zip(items, dsts):
        if d.dtype == torch.uint8:
            np.testing.assert_array_equal(as_hwc(d, l), oracle_of(it))


def test_workspace_too_small_is_rejected():
    items = make_mixed(4, 3)
    srcs = [torch.from_numpy(it["img"]).to(dev()) for it in items]
    dsts = [alloc_dst(it) for it in items]
    work = kr.work_array([work_of(it, s, d, l) for it, s, (d, l) in zip(items, srcs, dsts)])
    ws = torch.empty(64, dtype=torch.uint8, device=dev())
    with pytest.raises(kr.KrError) as e:
        kr.kr_batch_submit(work, ws)
    assert e.value.status == 5


@pytest.mark.parametrize("pitched", [False, True])
def test_ragged_256_warps_full_size(pitched):
    """256 warps, sides log-uniform 64..2048, output scale 0.25-2x: every item of the batch
    equals its single-image launch and the oracle (the oracle's calls run on a thread pool:
    they release the interpreter lock)."""
    import concurrent.futures as cf
    import os
    spec = inputs.ragged_batch(1003, 256)
    imgs, srcs, dsts, work = [], [], [], []
    for it in spec:
        img = inputs.uniform_image(it.seed, it.H, it.W, 3)
        imgs.append(img)
        s = to_src(img, pitched)
        d = torch.empty((it.h, it.w, 3), dtype=torch.uint8, device=dev())
        srcs.append(s)
        dsts.append(d)
        work.append(kr.work_item(kr.KR_OP_WARP, s, d, M=it.M))
    ws = torch.empty(kr.kr_batch_workspace_size(256), dtype=torch.uint8, device=dev())
    kr.kr_batch_submit(kr.work_array(work), ws, use_graph=True)
    torch.cuda.synchronize()
    for i, (it, s, d) in enumerate(zip(spec, srcs, dsts)):
        single = torch.empty_like(d)
        kr.kr_warp_affine(s, single, it.M)
        torch.cuda.synchronize()
        assert torch.equal(single, d), i
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        refs = list(ex.map(lambda k: oracle.warp_u8(imgs[k], spec[k].M, spec[k].h, spec[k].w), range(len(spec))))
    for i, ref in enumerate(refs):
        np.testing.assert_array_equal(dsts[i].cpu().numpy(), ref, err_msg=f"item {i}")
