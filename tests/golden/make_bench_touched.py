"""Write bench_touched.json: the unique source bytes that the benchmark's
1920x1080 workload reads, per operation, counted by the oracle's touched-pixel
bitmaps (a source pixel counts when some output sample reads it with a
nonzero weight). Pixel-granular bytes and 32-byte-sector-granular bytes.

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
    out = {
        "workload": f"{n} x {W}x{H}x3 u8 noise+gradient frames (inputs.bench_images / bench_matrices / bench_homographies)",
        "images": n,
        "per_image": "lists hold one value per frame, frame i = bench_images()[i]",
        "per_op": {k: {"touched_bytes": v[0], "touched_sector_bytes": v[1]} for k, v in sorted(acc.items())},
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bench_touched.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print({k: (sum(v['touched_bytes']), sum(v['touched_sector_bytes'])) for k, v in out['per_op'].items()})


if __name__ == "__main__":
    main()
