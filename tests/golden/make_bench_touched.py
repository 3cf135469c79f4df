"""Write bench_touched.json: the unique source bytes that the benchmark's
1920x1080 workload reads, per operation, counted by the oracle's touched-pixel
bitmaps (a source pixel counts when some output sample reads it with a
nonzero weight). Pixel-granular bytes and 32-byte-sector-granular bytes. Also
("extra") the same counts for the other timed workloads: 640x480 -> 320x240,
3840x2160 -> 224x224 and the 256-item ragged batch of warps.

Calls only the oracle and the shared input generators. Run from the repo root:
    python tests/golden/make_bench_touched.py
"""
from __future__ import annotations

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2505_12425_gb300 import inputs  # noqa: E402


def main():
    n, H, W = inputs.BENCH_IMAGES, inputs.BENCH_H, inputs.BENCH_W
    imgs = inputs.bench_images(n)
    Ms = inputs.bench_matrices(n)
    Ps = inputs.bench_homographies(n)
    pitch = W * 3
    acc = {}

    def add(op, bitmap):
        px = oracle.touched_bytes(bitmap, 3)
        sec = oracle.touched_bytes(bitmap, 3, row_bytes=pitch, sector=32)
        a = acc.setdefault(op, [[], []])
        a[0].append(px)
        a[1].append(sec)

    for i in range(n):
        _, t8 = oracle.resize_u8(imgs[i], 720, 1280, touched=True)
        _, tf = oracle.resize_f64(imgs[i], 720, 1280, touched=True)
        for op in ("resize_u8", "resize_gray_u8"):
            add(op, t8)
        for op in ("resize_f32", "resize_norm_f32_chw"):
            add(op, tf)
        _, w8 = oracle.warp_u8(imgs[i], Ms[i], H, W, touched=True)
        _, wf = oracle.warp_f64(imgs[i], Ms[i], H, W, touched=True)
        for op in ("warp_u8", "warp_gray_u8"):
            add(op, w8)
        add("warp_f32", wf)
        add("rgb_to_gray", np.ones((H, W), np.uint8))
        _, p8 = oracle.warp_persp_u8(imgs[i], Ps[i], H, W, touched=True)
        add("warp_persp_u8", p8)
        _, r8 = oracle.warp_u8(imgs[i], Ms[i], H, W, touched=True, border="replicate")
        add("warp_u8_replicate", r8)
    # the other timed workloads: the bytes depend only on the sizes (and maps), not on the pixels
    extra = {}
    z = np.zeros((480, 640, 3), np.uint8)
    _, t = oracle.resize_u8(z, 240, 320, touched=True)
    extra["c1_resize_u8_640x480_to_320x240"] = {
        "per": "one image", "touched_bytes": oracle.touched_bytes(t, 3),
        "touched_sector_bytes": oracle.touched_bytes(t, 3, row_bytes=640 * 3, sector=32)}
    z = np.zeros((2160, 3840, 3), np.uint8)
    _, t = oracle.resize_f64(z, 224, 224, touched=True)
    extra["c3_resize_norm_f32_chw_3840x2160_to_224x224"] = {
        "per": "one image", "touched_bytes": oracle.touched_bytes(t, 3),
        "touched_sector_bytes": oracle.touched_bytes(t, 3, row_bytes=3840 * 3, sector=32)}
    rb, rs, ro = [], [], []
    for it in inputs.ragged_batch(1003, 256):
        _, t = oracle.warp_u8(np.zeros((it.H, it.W, 3), np.uint8), it.M, it.h, it.w, touched=True)
        pitch = (it.W * 3 + 63) // 64 * 64   # the 64-byte pitched layout the benchmark stores sources in
        rb.append(oracle.touched_bytes(t, 3))
        rs.append(oracle.touched_bytes(t, 3, row_bytes=pitch, sector=32))
        ro.append(it.h * it.w * 3)
    extra["ragged_256_warps_u8"] = {
        "per": "item of inputs.ragged_batch(1003, 256), sources in 64-byte pitched rows",
        "touched_bytes": rb, "touched_sector_bytes": rs, "out_bytes": ro}
    out = {
        "workload": f"{n} x {W}x{H}x3 u8 noise+gradient frames (inputs.bench_images / bench_matrices / bench_homographies)",
        "images": n,
        "per_image": "lists hold one value per frame, frame i = bench_images()[i]",
        "per_op": {k: {"touched_bytes": v[0], "touched_sector_bytes": v[1]} for k, v in sorted(acc.items())},
        "extra": extra,
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bench_touched.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print({k: (sum(v['touched_bytes']), sum(v['touched_sector_bytes'])) for k, v in out['per_op'].items()})
    print({k: (v['touched_bytes'] if isinstance(v['touched_bytes'], int) else sum(v['touched_bytes'])) for k, v in extra.items()})


if __name__ == "__main__":
    main()
