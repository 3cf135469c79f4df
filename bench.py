"""Benchmark of the resampling path on GB300.

One step = every operation of the path over a batch of 32 synthetic 1920x1080x3
u8 video frames (inputs larger than L2: 199 MB of sources per step), each
operation one launch over the whole batch through the C ABI:

  resize -> 1280x720: u8 | u8 + fused gray | f32 | f32 + normalise, planar CHW
  warp_affine -> 1920x1080 (per-frame inverse map): u8 | u8 + fused gray | f32
  rgb_to_gray (standalone)

Metric: output Gpixel/s of the whole step (all ranks), plus the HBM roofline of
the dominant kernel (algorithmic bytes = output bytes + unique source bytes
read, from tests/golden/bench_touched.json, over its CUDA-event duration), the
oracle timed on the host cores, the end-to-end rate through the public API
with pinned host buffers, a ragged-batch comparison (256 warps in one
persistent graph-replayed launch vs 256 per-image launches) and SM clocks
sampled during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {gb300,reference}]

Under torchrun each rank runs its own copy of the workload (weak scaling); the
step time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2505_12425_gb300 import inputs  # noqa: E402
from paper_2505_12425_gb300.sharding import max_over_ranks  # noqa: E402

METRIC = "Gpixel/s and HBM GB/s %peak for resize/warp; p50/p99 latency batched vs per-image"
UNIT = "Gpixel/s"
WORKLOAD = "32 x 1920x1080x3 u8 frames: resize->1280x720 (u8, u8+gray, f32, f32 norm CHW), " \
           "warp_affine->1920x1080 (u8, u8+gray, f32), rgb_to_gray"
MEAN, STD = inputs.IMAGENET_MEAN, inputs.IMAGENET_STD
RS_H, RS_W = 720, 1280


def op_table():
    """(name, output pixels per image, output bytes per image) of the step's operations."""
    H, W = inputs.BENCH_H, inputs.BENCH_W
    r, w = RS_H * RS_W, H * W
    return [
        ("resize_u8", r, 3 * r), ("resize_gray_u8", r, r), ("resize_f32", r, 12 * r),
        ("resize_norm_f32_chw", r, 12 * r), ("warp_u8", w, 3 * w), ("warp_gray_u8", w, w),
        ("warp_f32", w, 12 * w), ("rgb_to_gray", w, w),
    ]


def kernel_source_sha() -> str:
    """Hash of the sources of the per-operation kernels (the tile engine and its launcher)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2505_12425_gb300", "csrc")
    for f in ("kr_device.cuh", "kr_quad.cuh", "kr_tile.cuh", "kr_kernels.cu"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


NOMINAL_HBM_GBS = 8000.0   # the chip's nominal HBM bandwidth (~8 TB/s), beside the measured copy


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def load_traffic(op):
    """ncu dram bytes per launch of `op`, if captured from the current kernel source."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get("per_op", {}).get(op)
    if not e or d.get("kernel_source_sha") != kernel_source_sha():
        return None
    return e.get("dram_bytes_per_launch")


# ---------------------------------------------------------------------------
# Clock sampling (nvidia-smi) during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, out_dir: str | None = None):
        self.proc = None
        out_dir = out_dir or tempfile.mkdtemp(prefix="kr_clocks_")
        self.path = os.path.join(out_dir, f"clocks_rank{gpu_index}.csv")
        self.idx = gpu_index

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if not self.proc:
            return None
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        mx = float(rows[0][2])
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, v in zip(names, r[5:9]):
                if v.strip() == "Active":
                    reasons.add(k)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].strip()[:1].isdigit())
                if any(r[3].strip()[:1].isdigit() for r in rows) else None}


# ---------------------------------------------------------------------------
# The GPU arm
# ---------------------------------------------------------------------------
class Step:
    """Prepared C-ABI calls of one step (descriptors built once)."""

    def __init__(self, torch, kr, dev, imgs_dev, Ms):
        self.torch, self.kr = torch, kr
        n, H, W = imgs_dev.shape[0], inputs.BENCH_H, inputs.BENCH_W
        e = lambda *s, dt=torch.uint8: torch.empty(*s, dtype=dt, device=dev)  # noqa: E731
        f32 = torch.float32
        self.src = imgs_dev
        self.outs = {
            "resize_u8": e((n, RS_H, RS_W, 3)), "resize_gray_u8": e((n, RS_H, RS_W, 1)),
            "resize_f32": e((n, RS_H, RS_W, 3), dt=f32), "resize_norm_f32_chw": e((n, 3, RS_H, RS_W), dt=f32),
            "warp_u8": e((n, H, W, 3)), "warp_gray_u8": e((n, H, W, 1)), "warp_f32": e((n, H, W, 3), dt=f32),
            "rgb_to_gray": e((n, H, W, 1)),
        }
        lib = kr.load()
        self.lib = lib
        self.Ms = np.ascontiguousarray(Ms.reshape(-1), dtype=np.float32)
        self.Mp = self.Ms.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        s = kr.image(imgs_dev)
        self._keep = []

        def call_resize(name, layout="hwc", **p):
            d, pp = kr.image(self.outs[name], layout), kr.post(**p)
            self._keep += [d, pp]
            return lambda st: lib.kr_resize_bilinear(ctypes.byref(s), ctypes.byref(d), ctypes.byref(pp), st)

        def call_warp(name, **p):
            d, pp = kr.image(self.outs[name]), kr.post(**p)
            self._keep += [d, pp]
            return lambda st: lib.kr_warp_affine(ctypes.byref(s), ctypes.byref(d), self.Mp, ctypes.byref(pp), st)

        def call_gray(name):
            d = kr.image(self.outs[name])
            self._keep.append(d)
            return lambda st: lib.kr_rgb_to_gray(ctypes.byref(s), ctypes.byref(d), st)

        self._keep.append(s)
        self.calls = [
            ("resize_u8", call_resize("resize_u8")),
            ("resize_gray_u8", call_resize("resize_gray_u8", gray=True)),
            ("resize_f32", call_resize("resize_f32")),
            ("resize_norm_f32_chw", call_resize("resize_norm_f32_chw", "chw", mean=MEAN, std=STD)),
            ("warp_u8", call_warp("warp_u8")),
            ("warp_gray_u8", call_warp("warp_gray_u8", gray=True)),
            ("warp_f32", call_warp("warp_f32")),
            ("rgb_to_gray", call_gray("rgb_to_gray")),
        ]

    # The step's operations are independent: run_split issues the instruction-bound u8 kinds on
    # one stream and the f32 kinds and rgb_to_gray, which move the most bytes, on another, so that
    # their CTAs share the SMs.
    SPLITS = {
        2: (("warp_u8", "resize_u8", "warp_gray_u8", "resize_gray_u8"),
            ("warp_f32", "resize_f32", "resize_norm_f32_chw", "rgb_to_gray")),
        3: (("warp_u8", "resize_gray_u8", "rgb_to_gray"), ("warp_gray_u8", "resize_u8"),
            ("warp_f32", "resize_f32", "resize_norm_f32_chw")),
        4: (("warp_u8", "resize_u8"), ("warp_gray_u8", "resize_gray_u8"), ("warp_f32", "rgb_to_gray"),
            ("resize_f32", "resize_norm_f32_chw")),
    }
    SPLIT = SPLITS[2]

    def run_split(self, main, sides):
        """One step on the torch stream `main` and the streams `sides` (forked from and joined back
        into main), split as SPLITS[1 + len(sides)]."""
        torch = self.torch
        if not hasattr(self, "_fork"):
            self._fork = torch.cuda.Event()
            self._joins = [torch.cuda.Event() for _ in range(3)]
            self._by_name = dict(self.calls)
        self._fork.record(main)
        for sd in sides:
            sd.wait_event(self._fork)
        for names, s in zip(self.SPLITS[1 + len(sides)], [main] + list(sides)):
            h = ctypes.c_void_p(s.cuda_stream)
            for name in names:
                st = self._by_name[name](h)
                if st != 0:
                    raise RuntimeError(f"{name}: status {st} {self.lib.kr_last_error().decode()}")
        for sd, ev in zip(sides, self._joins):
            ev.record(sd)
            main.wait_event(ev)

    def run(self, stream_handle, events=None):
        for i, (name, c) in enumerate(self.calls):
            if events is not None:
                events[i][0].record()
            st = c(stream_handle)
            if st != 0:
                raise RuntimeError(f"{name}: status {st} {self.lib.kr_last_error().decode()}")
            if events is not None:
                events[i][1].record()


def pitched(torch, img, dev, align=64):
    """A device copy of an HWC u8 image whose rows start `align`-byte aligned (pitched, as a
    resident image pool lays frames out in HBM; the row padding is never read)."""
    H, W, C = img.shape
    pitch = (W * C + align - 1) // align * align
    buf = torch.empty((H * pitch,), dtype=torch.uint8, device=dev)
    v = torch.as_strided(buf, (H, W, C), (pitch, C, 1))
    v.copy_(torch.from_numpy(img).to(dev))
    return v


def ragged_compare(torch, kr, dev, peak=None, reps=20, autotune=True):
    """256 warps (sides log-uniform 64..2048, output 0.25-2x, pitched sources): one persistent
    graph-replayed launch vs 256 per-image launches. Returns a summary dict."""
    spec = inputs.ragged_batch(1003, 256)
    srcs, dsts, work = [], [], []
    for it in spec:
        s = pitched(torch, inputs.uniform_image(it.seed, it.H, it.W, 3), dev)
        d = torch.empty((it.h, it.w, 3), dtype=torch.uint8, device=dev)
        srcs.append(s)
        dsts.append(d)
        work.append(kr.work_item(kr.KR_OP_WARP, s, d, M=it.M))
    arr = kr.work_array(work)
    ws = torch.empty(kr.kr_batch_workspace_size(len(arr)), dtype=torch.uint8, device=dev)
    # autotune: the tuner's pick for this batch class (else tile configuration 0 at its default
    # residency, a fixed launch for profiling)
    cfg, ctas = kr.kr_autotune_batch(arr, ws) if autotune else (0, 0)
    out_px = sum(it.h * it.w for it in spec)
    lib = kr.load()
    single = []
    for it, s, d in zip(spec, srcs, dsts):
        si, di, pp = kr.image(s), kr.image(d), kr.post()
        M = np.ascontiguousarray(it.M.reshape(-1), dtype=np.float32)
        single.append((si, di, pp, M, M.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    opts = kr.KrBatchOpts(-1, 0, 1) if autotune else kr.KrBatchOpts(0, 0, 1)

    def batched():
        r = lib.kr_batch_submit(arr, len(arr), ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.byref(opts), st)
        assert r == 0, r

    def per_image():
        for si, di, pp, _, Mp in single:
            r = lib.kr_warp_affine(ctypes.byref(si), ctypes.byref(di), Mp, ctypes.byref(pp), st)
            assert r == 0, r

    res = {}
    for name, fn in (("batched", batched), ("per_image", per_image)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        times = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            times.append(a.elapsed_time(b))
        times.sort()
        res[name] = {"ms_p50": round(statistics.median(times), 4),
                     "ms_p99": round(times[min(len(times) - 1, int(0.99 * len(times)))], 4),
                     "gpx_s": round(out_px / (statistics.median(times) * 1e-3) / 1e9, 3)}
    t = json.load(open(os.path.join(ROOT, "tests", "golden", "bench_touched.json")))["extra"]["ragged_256_warps_u8"]
    alg = sum(t["touched_bytes"]) + sum(t["out_bytes"])
    alg_sec = sum(t["touched_sector_bytes"]) + sum(t["out_bytes"])
    for name in ("batched", "per_image"):
        gbs = alg / (res[name]["ms_p50"] * 1e-3) / 1e9
        res[name]["GB_s"] = round(gbs, 1)
        if peak:
            res[name]["frac_of_measured_hbm"] = round(gbs / peak, 3)
            res[name]["frac_of_measured_hbm_sector"] = round(alg_sec / (res[name]["ms_p50"] * 1e-3) / 1e9 / peak, 3)
    res.update({"alg_bytes": alg, "alg_sector_bytes": alg_sec,
                "items": 256, "out_px": out_px, "tile_config": list(kr.kr_tile_config_shape(cfg)),
                "ctas_per_sm": ctas, "launches_batched": 1, "launches_per_image": 256,
                "speedup_p50": round(res["per_image"]["ms_p50"] / res["batched"]["ms_p50"], 3)})
    return res


SERVE_RATES = (2000, 5000, 10000, 20000, 40000, 80000, 160000, 200000, 210000, 220000, 225000, 230000, 235000,
               240000, 250000, 260000, 280000, 320000)
SERVE_STREAMS = 8            # launches in flight (the best of 2/4/8/16 for both per-image and size-aware)
SERVE_DIRECT_PX = 1 << 18    # size-aware threshold: requests of at least this many output pixels launch alone


def serving_compare(torch, kr, dev, rates=SERVE_RATES, seconds=1.0, grid=False):
    """Poisson request streams (sizes log-uniform 320..3840 x 240..2160, op uniform over
    resize / warp / gray) over a device-resident pool of 64 pitched images, 8 GB in-flight budget:
    continuous batching (policy 0) vs one launch per request (policy 1) vs size-aware continuous
    batching (policy 2: requests of at least 2^18 output pixels launch alone at once, the smaller
    ones share ragged launches on free slots), 8 streams each. Offered rates step
    finely between the last rate every policy keeps up with and saturation. grid: also every
    (max_batch, streams) of {16, 32, 64} x {2, 4, 8} for the two batching policies (streams only
    for per-image launches) at the rates around saturation."""
    sizes = inputs.pool_sizes(1004, 64)
    pool = [pitched(torch, inputs.uniform_image(5000 + i, H, W, 3), dev) for i, (H, W) in enumerate(sizes)]
    arena = torch.empty(8 << 30, dtype=torch.uint8, device=dev)
    out = {"pool_images": 64, "budget_bytes": 8 << 30, "seconds_per_rate": seconds, "streams": SERVE_STREAMS,
           "max_batch": 64, "size_aware_direct_px": SERVE_DIRECT_PX, "runs": []}
    for rate in rates:
        # the highest rates run for a shorter time (the stream and its host-side arrays scale with it)
        dur = seconds if rate <= 80000 else seconds * 80000 / rate * 2
        reqs = inputs.request_stream(1004, float(rate), dur, pool=64)
        px = sum(r.h * r.w for r in reqs)
        for policy in (0, 1, 2):
            res = kr.kr_serve_run(reqs, pool, arena, budget_bytes=8 << 30, max_batch=64, streams=SERVE_STREAMS,
                                  policy=policy, direct_px=SERVE_DIRECT_PX if policy == 2 else 0)
            lat = np.array([res[i].t_done - r.t_arrival for i, r in enumerate(reqs)]) * 1e3
            t_end = max(res[i].t_done for i in range(len(reqs)))
            nb = len({round(res[i].t_launch, 9) for i in range(len(reqs))})
            out["runs"].append({
                "rate": rate, "policy": ("batched", "per_image", "size_aware")[policy], "requests": len(reqs),
                "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
                "p999_ms": round(float(np.percentile(lat, 99.9)), 3),
                "gpx_s": round(px / t_end / 1e9, 3), "launches": nb, "mean_batch": round(len(reqs) / nb, 2)})
    if grid:
        for rate in (200000, 220000, 240000):
            dur = seconds * 80000 / rate * 2
            reqs = inputs.request_stream(1004, float(rate), dur, pool=64)
            px = sum(r.h * r.w for r in reqs)
            for policy in (0, 1, 2):
                for streams in (2, 4, 8):
                    for mb in ((16, 32, 64) if policy != 1 else (64,)):
                        res = kr.kr_serve_run(reqs, pool, arena, budget_bytes=8 << 30, max_batch=mb, streams=streams,
                                              policy=policy, direct_px=SERVE_DIRECT_PX if policy == 2 else 0)
                        lat = np.array([res[i].t_done - r.t_arrival for i, r in enumerate(reqs)]) * 1e3
                        t_end = max(res[i].t_done for i in range(len(reqs)))
                        out["runs"].append({
                            "rate": rate, "policy": ("batched", "per_image", "size_aware")[policy],
                            "streams": streams, "max_batch": mb, "requests": len(reqs),
                            "p50_ms": round(float(np.percentile(lat, 50)), 3),
                            "p99_ms": round(float(np.percentile(lat, 99)), 3), "gpx_s": round(px / t_end / 1e9, 3)})
    best = {}
    for slo in (2.0, 5.0, 10.0, 20.0):
        for pol in ("batched", "per_image", "size_aware"):
            ok = [r for r in out["runs"] if r["policy"] == pol and r["p99_ms"] <= slo]
            top = max(ok, key=lambda r: r["gpx_s"], default=None)
            best[f"{pol}_gpx_s_at_p99<={slo:g}ms"] = top["gpx_s"] if top else None
            if top and "streams" in top:
                best[f"{pol}_config_at_p99<={slo:g}ms"] = {"streams": top["streams"], "max_batch": top["max_batch"],
                                                           "rate": top["rate"]}
    out["best"] = best
    return out


def next_rows(torch, kr, dev, imgs_dev, peak, reps=50):
    """The widening rows on the same frames, each one launch over the batch: nearest-neighbour
    resize -> 1280x720, horizontal flip, perspective warp (per-frame homographies, u8), Sobel
    3x3 magnitude of the frames' gray (f32 out), the u8 affine warp with the replicated border,
    area downscales (-> 1280x720 u8; 16 x 3840x2160 -> 224x224 normalised planar f32).
    Algorithmic bytes = output + distinct source pixels read (nearest: distinct source rows x
    distinct source columns; flip, Sobel, area: every pixel; warps: the oracle's touched bitmaps)."""
    n, H, W, C = imgs_dev.shape
    lib = kr.load()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    s = kr.image(imgs_dev)
    P = np.ascontiguousarray(inputs.bench_homographies(n).reshape(-1), dtype=np.float32)
    Pp = P.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    pp = kr.post()
    prep = kr.post(border="replicate")
    # the strong-downscale case: 16 uniform 3840x2160 frames -> 224x224 normalised, planar
    src4k = torch.from_numpy(np.stack([inputs.uniform_image(700 + i, 2160, 3840, 3) for i in range(16)])).to(dev)
    s4k = kr.image(src4k)
    pnorm = kr.post(mean=MEAN, std=STD)
    A = np.ascontiguousarray(inputs.bench_matrices(n).reshape(-1), dtype=np.float32)
    Ap = A.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    outs = {"resize_nearest_u8": torch.empty((n, RS_H, RS_W, C), dtype=torch.uint8, device=dev),
            "flip_u8": torch.empty((n, H, W, C), dtype=torch.uint8, device=dev),
            "warp_persp_u8": torch.empty((n, H, W, C), dtype=torch.uint8, device=dev),
            "sobel_f32": torch.empty((n, H, W, 1), dtype=torch.float32, device=dev),
            "warp_u8_replicate": torch.empty((n, H, W, C), dtype=torch.uint8, device=dev),
            "resize_area_u8": torch.empty((n, RS_H, RS_W, C), dtype=torch.uint8, device=dev),
            "resize_area_16x4k_224_f32_chw": torch.empty((16, 3, 224, 224), dtype=torch.float32, device=dev)}
    ds = {k: kr.image(v, "chw" if k.endswith("chw") else "hwc") for k, v in outs.items()}
    d224 = ds["resize_area_16x4k_224_f32_chw"]
    calls = {"resize_nearest_u8": lambda: lib.kr_resize_nearest(ctypes.byref(s), ctypes.byref(ds["resize_nearest_u8"]), st),
             "flip_u8": lambda: lib.kr_flip_horizontal(ctypes.byref(s), ctypes.byref(ds["flip_u8"]), st),
             "warp_persp_u8": lambda: lib.kr_warp_perspective(ctypes.byref(s), ctypes.byref(ds["warp_persp_u8"]), Pp,
                                                              ctypes.byref(pp), st),
             "sobel_f32": lambda: lib.kr_sobel(ctypes.byref(s), ctypes.byref(ds["sobel_f32"]), 3, st),
             "warp_u8_replicate": lambda: lib.kr_warp_affine(ctypes.byref(s), ctypes.byref(ds["warp_u8_replicate"]),
                                                             Ap, ctypes.byref(prep), st),
             "resize_area_u8": lambda: lib.kr_resize_area(ctypes.byref(s), ctypes.byref(ds["resize_area_u8"]),
                                                          ctypes.byref(pp), st),
             "resize_area_16x4k_224_f32_chw": lambda: lib.kr_resize_area(ctypes.byref(s4k), ctypes.byref(d224),
                                                                         ctypes.byref(pnorm), st)}
    rows = len({((2 * y + 1) * H) // (2 * RS_H) for y in range(RS_H)})
    cols = len({((2 * x + 1) * W) // (2 * RS_W) for x in range(RS_W)})
    touched = json.load(open(os.path.join(ROOT, "tests", "golden", "bench_touched.json")))["per_op"]
    alg = {"resize_nearest_u8": n * (RS_H * RS_W * C + rows * cols * C), "flip_u8": n * 2 * H * W * C,
           "warp_persp_u8": n * H * W * C + sum(touched["warp_persp_u8"]["touched_bytes"][:n]),
           "sobel_f32": n * H * W * (C + 4),
           "warp_u8_replicate": n * H * W * C + sum(touched["warp_u8_replicate"]["touched_bytes"][:n]),
           "resize_area_u8": n * (H * W * C + RS_H * RS_W * C),
           "resize_area_16x4k_224_f32_chw": 16 * (2160 * 3840 * 3 + 224 * 224 * 3 * 4)}
    res = {}
    for name, fn in calls.items():
        for _ in range(3):
            assert fn() == 0
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b) / reps
        gbs = alg[name] / (ms * 1e-3) / 1e9
        o = outs[name]
        opx = o.shape[0] * (o.shape[2] * o.shape[3] if name.endswith("chw") else o.shape[1] * o.shape[2])
        res[name] = {"ms": round(ms, 4), "alg_bytes": alg[name], "GB_s": round(gbs, 1),
                     "frac_of_measured_hbm": round(gbs / peak, 3), "gpx_s": round(opx / (ms * 1e-3) / 1e9, 1)}
    return res


def l2_flush(torch, dev, buf=[]):
    """Write a buffer twice the size of L2 so that the next launch reads from HBM."""
    if not buf:
        buf.append(torch.empty(256 << 20, dtype=torch.uint8, device=dev))
    buf[0].fill_(1)


def small_and_strong_downscale(torch, kr, dev, peak, reps=30):
    """The two other resize workloads, bilinear:
    c1  640x480 -> 320x240 u8 over 256 distinct uniform frames (295 MB of sources and
        outputs, more than L2): one launch per frame (launch-bound: the work of a launch is
        1.15 MB) and one launch over all 256 frames;
    c3  16 uniform 3840x2160 -> 224x224 normalised planar f32 NCHW, one launch, L2 flushed
        before every timed launch (its touched bytes would otherwise stay in L2).
    Algorithmic bytes = output + the source bytes the taps read (the oracle's bitmaps,
    tests/golden/bench_touched.json), pixel- and 32-byte-sector-granular."""
    lib = kr.load()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    extra = json.load(open(os.path.join(ROOT, "tests", "golden", "bench_touched.json")))["extra"]
    out = {}
    # c1
    n1 = 256
    src = torch.from_numpy(inputs.uniform_batch(1000, n1, 480, 640)).to(dev)
    dst = torch.empty((n1, 240, 320, 3), dtype=torch.uint8, device=dev)
    pp = kr.post()
    sb, db = kr.image(src), kr.image(dst)
    singles = [(kr.image(src[i]), kr.image(dst[i])) for i in range(n1)]
    t1 = extra["c1_resize_u8_640x480_to_320x240"]
    per_frame = 240 * 320 * 3 + t1["touched_bytes"]
    per_frame_sec = 240 * 320 * 3 + t1["touched_sector_bytes"]

    def one_per_frame():
        for a, b in singles:
            assert lib.kr_resize_bilinear(ctypes.byref(a), ctypes.byref(b), ctypes.byref(pp), st) == 0

    def one_launch():
        assert lib.kr_resize_bilinear(ctypes.byref(sb), ctypes.byref(db), ctypes.byref(pp), st) == 0

    for name, fn, launches in (("per_frame_launches", one_per_frame, n1), ("one_launch", one_launch, 1)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b) / reps
        gbs = n1 * per_frame / (ms * 1e-3) / 1e9
        out[f"c1_640x480_to_320x240_u8_{name}"] = {
            "frames": n1, "launches": launches, "ms": round(ms, 4), "us_per_launch": round(ms * 1e3 / launches, 3),
            "gpx_s": round(n1 * 240 * 320 / (ms * 1e-3) / 1e9, 2), "alg_bytes": n1 * per_frame, "GB_s": round(gbs, 1),
            "frac_of_measured_hbm": round(gbs / peak, 3),
            "frac_of_measured_hbm_sector": round(n1 * per_frame_sec / (ms * 1e-3) / 1e9 / peak, 3)}
    del src, dst
    # c3
    src3 = torch.from_numpy(inputs.uniform_batch(1002, 16, 2160, 3840)).to(dev)
    dst3 = torch.empty((16, 3, 224, 224), dtype=torch.float32, device=dev)
    s3, d3 = kr.image(src3), kr.image(dst3, "chw")
    pn = kr.post(mean=MEAN, std=STD)
    t3 = extra["c3_resize_norm_f32_chw_3840x2160_to_224x224"]
    ob = 224 * 224 * 3 * 4
    for _ in range(3):
        assert lib.kr_resize_bilinear(ctypes.byref(s3), ctypes.byref(d3), ctypes.byref(pn), st) == 0
    times = []
    for _ in range(reps):
        l2_flush(torch, dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        assert lib.kr_resize_bilinear(ctypes.byref(s3), ctypes.byref(d3), ctypes.byref(pn), st) == 0
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b))
    ms = statistics.median(times)
    alg, alg_sec = 16 * (ob + t3["touched_bytes"]), 16 * (ob + t3["touched_sector_bytes"])
    out["c3_16x3840x2160_to_224x224_norm_f32_chw"] = {
        "images": 16, "launches": 1, "ms": round(ms, 4), "gpx_s": round(16 * 224 * 224 / (ms * 1e-3) / 1e9, 3),
        "alg_bytes": alg, "alg_sector_bytes": alg_sec, "GB_s": round(alg / (ms * 1e-3) / 1e9, 1),
        "frac_of_measured_hbm": round(alg / (ms * 1e-3) / 1e9 / peak, 3),
        "frac_of_measured_hbm_sector": round(alg_sec / (ms * 1e-3) / 1e9 / peak, 3),
        "l2": "flushed (256 MB write) before every timed launch"}
    return out


def cpu_baseline_sample(budget_s=12.0):
    """The oracle (single-threaded C) on a bounded sample of the step: whole frames, all eight
    operations, until the time budget is spent."""
    import oracle
    imgs_n = inputs.BENCH_IMAGES
    Ms = inputs.bench_matrices(imgs_n)
    H, W = inputs.BENCH_H, inputs.BENCH_W
    px_per_img = sum(p for _, p, _ in op_table())
    done, t_total = 0, 0.0
    for i in range(imgs_n):
        img = inputs.noise_gradient_image(2000 + i, H, W)
        t0 = time.perf_counter()
        oracle.resize_u8(img, RS_H, RS_W)
        oracle.resize_u8(img, RS_H, RS_W, gray=True)
        oracle.resize_f64(img, RS_H, RS_W)
        oracle.resize_f64(img, RS_H, RS_W, mean=MEAN, std=STD)
        oracle.warp_u8(img, Ms[i], H, W)
        oracle.warp_u8(img, Ms[i], H, W, gray=True)
        oracle.warp_f64(img, Ms[i], H, W)
        oracle.rgb_to_gray_u8(img)
        t_total += time.perf_counter() - t0
        done += 1
        if t_total >= budget_s:
            break
    return {"value": round(done * px_per_img / t_total / 1e9, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} of {imgs_n} frames, all 8 operations, single-threaded C oracle "
                      f"({t_total:.1f} s)"}


def cpu_baseline_all_cores(budget_s=3.0):
    """The same oracle code on every host core: whole frames spread over one thread per core (the
    oracle's C calls release the interpreter lock), passes over the 32 frames until the time
    budget is spent. A secondary baseline beside the single-threaded one."""
    import concurrent.futures as cf
    import oracle
    imgs_n = inputs.BENCH_IMAGES
    Ms = inputs.bench_matrices(imgs_n)
    H, W = inputs.BENCH_H, inputs.BENCH_W
    imgs = [inputs.noise_gradient_image(2000 + i, H, W) for i in range(imgs_n)]
    px_per_img = sum(p for _, p, _ in op_table())
    cores = os.cpu_count() or 1

    def frame(i):
        img = imgs[i]
        oracle.resize_u8(img, RS_H, RS_W)
        oracle.resize_u8(img, RS_H, RS_W, gray=True)
        oracle.resize_f64(img, RS_H, RS_W)
        oracle.resize_f64(img, RS_H, RS_W, mean=MEAN, std=STD)
        oracle.warp_u8(img, Ms[i], H, W)
        oracle.warp_u8(img, Ms[i], H, W, gray=True)
        oracle.warp_f64(img, Ms[i], H, W)
        oracle.rgb_to_gray_u8(img)

    done, passes = 0, 0
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        t0 = time.perf_counter()
        while True:
            list(ex.map(frame, range(imgs_n)))
            done += imgs_n
            passes += 1
            if time.perf_counter() - t0 >= budget_s:
                break
        dt = time.perf_counter() - t0
    return {"value": round(done * px_per_img / dt / 1e9, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{passes} pass(es) over {imgs_n} frames, all 8 operations, one thread per core ({dt:.1f} s)"}


def run_gpu(args):
    import torch
    import torch.distributed as dist
    import __graft_entry__ as ge
    from paper_2505_12425_gb300 import binding as kr

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world == 1:
        ge.build()
    if world > 1:
        dist.barrier()
    kr.load()

    n = args.images
    imgs = inputs.bench_images(n)
    Ms = inputs.bench_matrices(n)
    imgs_dev = torch.from_numpy(imgs).to(dev)
    step = Step(torch, kr, dev, imgs_dev, Ms)
    stream = torch.cuda.current_stream()
    sh = ctypes.c_void_p(stream.cuda_stream)
    ops = op_table()

    side = [torch.cuda.Stream() for _ in range(args.streams - 1)] if args.streams > 1 else None
    for _ in range(args.warmup):
        step.run(sh) if side is None else step.run_split(stream, side)
    torch.cuda.synchronize()

    K = args.steps
    events = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in ops]
              for _ in range(K)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local, args.clocks_dir) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t_start.record()
        for k in range(K):
            if side is None:
                step.run(sh, events[k])
            else:
                step.run_split(stream, side)
        t_end.record()
        torch.cuda.synchronize()
        if side is not None:
            # second timed phase: the same number of steps with the calls one after another, each
            # call bracketed by CUDA events on its stream (every kernel timed while it runs alone)
            for k in range(K):
                step.run(sh, events[k])
            torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    ms_total = max_over_ranks(t_start.elapsed_time(t_end), dist if world > 1 else None, dev)
    ms_step = ms_total / K
    px_step = n * sum(p for _, p, _ in ops)
    value = world * px_step / (ms_step * 1e-3) / 1e9

    # per-operation kernel times (each call is one launch for this batch size)
    per_op = {}
    for i, (name, px, ob) in enumerate(ops):
        d = [events[k][i][0].elapsed_time(events[k][i][1]) for k in range(K)]
        per_op[name] = statistics.mean(d)
    touched = json.load(open(os.path.join(ROOT, "tests", "golden", "bench_touched.json")))["per_op"]
    dominant = max(per_op, key=per_op.get)
    peak, peak_kind = load_peaks()
    breakdown = {}
    for name, px, ob in ops:
        alg = n * ob + sum(touched[name]["touched_bytes"][:n])
        # the attainable floor: touched source bytes rounded out to whole 32-byte sectors
        alg_sec = n * ob + sum(touched[name]["touched_sector_bytes"][:n])
        gbs = alg / (per_op[name] * 1e-3) / 1e9
        breakdown[name] = {"ms": round(per_op[name], 4), "alg_bytes": alg, "GB_s": round(gbs, 1),
                           "frac_of_measured_hbm": round(gbs / peak, 3),
                           "frac_of_nominal_hbm": round(gbs / NOMINAL_HBM_GBS, 3), "alg_sector_bytes": alg_sec,
                           "frac_of_measured_hbm_sector": round(alg_sec / (per_op[name] * 1e-3) / 1e9 / peak, 3),
                           "share": round(per_op[name] / sum(per_op.values()), 3)}
    dom = breakdown[dominant]
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": dom["GB_s"], "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": dom["frac_of_measured_hbm"],
                "frac_of_nominal_8tbs": dom["frac_of_nominal_hbm"],
                "traffic": load_traffic(dominant), "alg_bytes_per_launch": dom["alg_bytes"]}

    # end to end through the public API: every step copies its inputs in from pinned host
    # memory, runs the eight calls and copies every output back to pinned host memory. Steps
    # are pipelined over two sets of device buffers on three streams (copy in, compute, copy
    # out), so that one step's copies overlap its neighbours' work; the host link (about
    # 0.2 TB/s each way on this machine, shared by both directions) bounds the rate.
    host_in = torch.from_numpy(imgs).pin_memory()
    steps2 = [step, Step(torch, kr, dev, torch.empty_like(imgs_dev), Ms)]
    host_out = [{k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in st.outs.items()}
                for st in steps2]
    h2d = host_in.numel()
    d2h = sum(v.numel() * v.element_size() for v in host_out[0].values())
    K_e2e = max(3, min(K, 20))
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    for b in range(2):   # every event starts in the completed state
        ev_done[b].record(stream)
        ev_out[b].record(stream)

    def e2e_step(i):
        b = i % 2
        st = steps2[b]
        with torch.cuda.stream(s_in):
            s_in.wait_event(ev_done[b])          # compute of step i - 2 has read this input set
            st.src.copy_(host_in, non_blocking=True)
            ev_in[b].record(s_in)
        stream.wait_event(ev_in[b])
        stream.wait_event(ev_out[b])             # step i - 2's outputs have left this set
        st.run(sh)
        ev_done[b].record(stream)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_done[b])
            for k, v in st.outs.items():
                host_out[b][k].copy_(v, non_blocking=True)
            ev_out[b].record(s_out)

    for i in range(2):
        e2e_step(i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s_in.wait_event(e0)
    s_out.wait_event(e0)
    for i in range(K_e2e):
        e2e_step(i)
    stream.wait_event(ev_out[(K_e2e - 1) % 2])
    stream.wait_event(ev_out[K_e2e % 2])
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1) / K_e2e, dist if world > 1 else None, dev)
    e2e = {"value": round(world * px_step / (ms_e2e * 1e-3) / 1e9, 3), "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(ms_e2e, 3),
           "steps": K_e2e}

    widening = next_rows(torch, kr, dev, imgs_dev, peak, reps=args.next_reps) \
        if args.extras in ("all", "next-rows") else None
    ragged = ragged_compare(torch, kr, dev, peak) if args.extras == "all" else \
        ragged_compare(torch, kr, dev, peak, autotune=False) if args.extras == "ragged" else None
    per_config = small_and_strong_downscale(torch, kr, dev, peak) if args.extras in ("all", "configs") else None
    serving = serving_compare(torch, kr, dev, seconds=args.serve_seconds, grid=args.serve_grid) \
        if args.extras == "all" else None
    cpu = cpu_baseline_sample() if (rank == 0 and args.extras == "all") else None
    cpu_all = cpu_baseline_all_cores() if (rank == 0 and args.extras == "all") else None

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8 (int32 fixed-point) + f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if n == inputs.BENCH_IMAGES else WORKLOAD.replace("32 x", f"{n} x"),
                       "images_per_step": n, "out_px_per_step": px_step,
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "streams": args.streams,
                       "l2": "no flush: 199 MB of distinct source frames per step > 129 MB L2"},
            "roofline": roofline, "per_op": breakdown, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all, "e2e": e2e,
            "gpu_launches": K * len(ops), "next_rows": widening, "per_config": per_config, "ragged": ragged,
            "serving": serving,
            "clocks": clk.summary(),
        }
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_reference(args):
    """The oracle as the reference arm: each step is a bounded sample of the workload (one frame,
    all eight operations) on the host cores."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    Ms = inputs.bench_matrices(inputs.BENCH_IMAGES)
    H, W = inputs.BENCH_H, inputs.BENCH_W
    px = sum(p for _, p, _ in op_table())
    frames = [inputs.noise_gradient_image(2000 + i, H, W) for i in range(min(4, inputs.BENCH_IMAGES))]

    def one(i):
        img, M = frames[i % len(frames)], Ms[i % len(frames)]
        oracle.resize_u8(img, RS_H, RS_W)
        oracle.resize_u8(img, RS_H, RS_W, gray=True)
        oracle.resize_f64(img, RS_H, RS_W)
        oracle.resize_f64(img, RS_H, RS_W, mean=MEAN, std=STD)
        oracle.warp_u8(img, M, H, W)
        oracle.warp_u8(img, M, H, W, gray=True)
        oracle.warp_f64(img, M, H, W)
        oracle.rgb_to_gray_u8(img)

    for i in range(args.warmup):
        one(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        one(i)
    dt = time.perf_counter() - t0
    value = args.steps * px / dt / 1e9
    sample = f"each step: 1 of {inputs.BENCH_IMAGES} frames, all 8 operations, single-threaded C oracle"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64 fixed-point + f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "images_per_step": 1},
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--no-extras", action="store_true", help="skip the next rows, the ragged and serving comparisons and the CPU baseline")
    ap.add_argument("--extras", choices=["all", "next-rows", "ragged", "configs", "none"], default="all",
                    help="which extra measurements follow the step: all, only the next rows, only the ragged "
                         "batch (tile configuration 0, no autotuning), only the 640x480 and 16 x 4K resize "
                         "configurations, or none")
    ap.add_argument("--streams", type=int, choices=[1, 2, 3, 4], default=2,
                    help="streams of the timed step: 1 = the eight calls one after another, 2 = the u8 kinds "
                         "and the f32 kinds + rgb_to_gray on two streams, 3-4 = finer splits (Step.SPLITS; "
                         "per-operation times are always taken one call after another)")
    ap.add_argument("--next-reps", type=int, default=50, help="timed launches per next row")
    ap.add_argument("--clocks-dir", default=None,
                    help="directory for the raw nvidia-smi clock samples (default: a temporary one)")
    ap.add_argument("--serve-seconds", type=float, default=1.0, help="seconds of requests per serving rate")
    ap.add_argument("--serve-grid", action="store_true",
                    help="also sweep the serving loop's streams and batch size around saturation")
    ap.add_argument("--images", type=int, default=inputs.BENCH_IMAGES,
                    help="frames per step (the full workload is 32; fewer only for small profiling cases)")
    args = ap.parse_args()
    if args.no_extras:
        args.extras = "none"
    if args.next_reps < 1:
        ap.error("--next-reps must be >= 1")
    if not 1 <= args.images <= inputs.BENCH_IMAGES:
        ap.error(f"--images must be in 1..{inputs.BENCH_IMAGES}")
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
