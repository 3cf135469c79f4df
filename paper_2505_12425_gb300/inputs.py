"""Seeded synthetic inputs for the resampling path.

This module only draws random inputs: images, inverse affine matrices, ragged
batch descriptions and request streams. It holds none of the resampling
arithmetic, imports neither the CUDA library nor the oracle, and is the one
module that both sides (the CUDA path's tests/benchmarks and the oracle's
tests) share.

Recipes (numpy ``default_rng(seed)``, PCG64, identical on x86-64 and aarch64):

* uniform images: i.i.d. uniform integers 0..255 per channel;
* noise + gradient images: ``(noise + round(255 * g_c) + 1) // 2`` (the mean
  of uniform noise and a smooth gradient, rounded half up), where
  ``g(x, y) = (x / (W - 1) + y / (H - 1)) / 2`` and channel c is shifted by
  c/3 modulo 1;
* affine maps: rotation U(-30 deg, 30 deg), scale U(0.8, 1.2), translation
  U(-100, 100) px on each axis, about the image centre. The forward map
  A = T(c_dst + t) R(theta) S(s) T(-c_src) is built and inverted in float64,
  then rounded to float32 (the kernels take the destination -> source map);
* ragged batches: H and W each ``round(exp(U(ln 64, ln 2048)))``, output scale
  k ~ U(0.25, 2) (output ``max(1, round(k * H)) x max(1, round(k * W))``),
  affine map as above with scale s * k;
* request streams: Poisson arrivals, width log-uniform 320..3840 and height
  log-uniform 240..2160 (independent), op uniform over
  {resize (k ~ U(0.25, 2)), warp (same size), gray}.
"""
from __future__ import annotations

import functools
import math
from dataclasses import dataclass

import numpy as np

# ImageNet per-channel statistics of p/255, used for the normalised f32 workloads.
IMAGENET_MEAN = (0.485, 0.456, 0.406)
IMAGENET_STD = (0.229, 0.224, 0.225)

OP_RESIZE = 0
OP_WARP = 1
OP_GRAY = 2


def uniform_image(seed: int, H: int, W: int, C: int = 3) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, size=(H, W, C), dtype=np.uint8)


def uniform_batch(seed: int, n: int, H: int, W: int, C: int = 3) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, size=(n, H, W, C), dtype=np.uint8)


@functools.lru_cache(maxsize=4)
def _gradient(H: int, W: int, C: int) -> np.ndarray:
    gx = np.arange(W, dtype=np.float64) / max(W - 1, 1)
    gy = np.arange(H, dtype=np.float64) / max(H - 1, 1)
    g = (gx[None, :] + gy[:, None]) / 2.0
    return np.stack([np.rint(np.mod(g + c / 3.0, 1.0) * 255.0) for c in range(C)], axis=-1).astype(np.uint16)


def noise_gradient_image(seed: int, H: int, W: int, C: int = 3) -> np.ndarray:
    rng = np.random.default_rng(seed)
    noise = rng.integers(0, 256, size=(H, W, C), dtype=np.uint8).astype(np.uint16)
    return ((noise + _gradient(H, W, C) + 1) >> 1).astype(np.uint8)


def _forward_affine(theta, s, tx, ty, c_src, c_dst):
    ct, st = math.cos(theta), math.sin(theta)
    T1 = np.array([[1, 0, -c_src[0]], [0, 1, -c_src[1]], [0, 0, 1]], dtype=np.float64)
    S = np.diag([s, s, 1.0])
    R = np.array([[ct, -st, 0], [st, ct, 0], [0, 0, 1]], dtype=np.float64)
    T2 = np.array([[1, 0, c_dst[0] + tx], [0, 1, c_dst[1] + ty], [0, 0, 1]], dtype=np.float64)
    return T2 @ R @ S @ T1


def random_inverse_affine(rng, H: int, W: int, h: int | None = None, w: int | None = None,
                          k: float = 1.0) -> np.ndarray:
    """A float32 2x3 destination->source map (rotation +-30 deg, scale 0.8-1.2 times k,
    translation +-100 px), about the source centre and the destination centre."""
    h = H if h is None else h
    w = W if w is None else w
    theta = math.radians(rng.uniform(-30.0, 30.0))
    s = rng.uniform(0.8, 1.2) * k
    tx, ty = rng.uniform(-100.0, 100.0, size=2)
    A = _forward_affine(theta, s, tx, ty, (W / 2.0, H / 2.0), (w / 2.0, h / 2.0))
    Minv = np.linalg.inv(A)
    return Minv[:2, :].astype(np.float32)


def random_inverse_homography(rng, H: int, W: int, h: int | None = None, w: int | None = None,
                              tilt: float = 0.25) -> np.ndarray:
    """A float32 3x3 destination->source map: the affine of random_inverse_affine followed by
    a keystone tilt (the projective row (px, py, 1) with |px| W, |py| H up to `tilt`, applied
    about the destination centre), inverted in float64 and scaled so that m22 = 1."""
    h = H if h is None else h
    w = W if w is None else w
    theta = math.radians(rng.uniform(-30.0, 30.0))
    s = rng.uniform(0.8, 1.2)
    tx, ty = rng.uniform(-100.0, 100.0, size=2)
    A = _forward_affine(theta, s, tx, ty, (W / 2.0, H / 2.0), (w / 2.0, h / 2.0))
    px = rng.uniform(-tilt, tilt) / max(w, 1)
    py = rng.uniform(-tilt, tilt) / max(h, 1)
    C1 = np.array([[1, 0, -w / 2.0], [0, 1, -h / 2.0], [0, 0, 1]], dtype=np.float64)
    P = np.array([[1, 0, 0], [0, 1, 0], [px, py, 1]], dtype=np.float64)
    C2 = np.array([[1, 0, w / 2.0], [0, 1, h / 2.0], [0, 0, 1]], dtype=np.float64)
    F = C2 @ P @ C1 @ A
    Minv = np.linalg.inv(F)
    return (Minv / Minv[2, 2]).astype(np.float32)


def homographies(seed: int, n: int, H: int, W: int, tilt: float = 0.25) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.stack([random_inverse_homography(rng, H, W, tilt=tilt) for _ in range(n)])


def warp_matrix(seed: int, H: int, W: int) -> np.ndarray:
    return random_inverse_affine(np.random.default_rng(seed), H, W)


def warp_matrices(seed: int, n: int, H: int, W: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.stack([random_inverse_affine(rng, H, W) for _ in range(n)])


# The 1920x1080 video-frame workload of the benchmark: BENCH_IMAGES noise +
# gradient frames (seeds 2000 + i), each with its own inverse affine map
# (seeds 3000 + i: rotation +-30 deg, scale 0.8-1.2, translation +-100 px).
BENCH_IMAGES = 32
BENCH_H, BENCH_W = 1080, 1920


def bench_images(n: int = BENCH_IMAGES) -> np.ndarray:
    return np.stack([noise_gradient_image(2000 + i, BENCH_H, BENCH_W) for i in range(n)])


def bench_matrices(n: int = BENCH_IMAGES) -> np.ndarray:
    return np.stack([warp_matrix(3000 + i, BENCH_H, BENCH_W) for i in range(n)])


def bench_homographies(n: int = BENCH_IMAGES, tilt: float = 0.25) -> np.ndarray:
    """Per-frame 3x3 inverse maps of the perspective row (seeds 3500 + i)."""
    return np.stack([random_inverse_homography(np.random.default_rng(3500 + i), BENCH_H, BENCH_W, tilt=tilt)
                     for i in range(n)])


@dataclass
class RaggedItem:
    op: int
    H: int
    W: int
    h: int
    w: int
    M: np.ndarray      # float32 (2, 3), destination -> source
    seed: int          # seed of this item's pixels


def ragged_batch(seed: int, n: int = 256, lo: int = 64, hi: int = 2048, ops=(OP_WARP,)) -> list:
    """n ragged items: sizes log-uniform in lo..hi per axis, output scale k ~ U(0.25, 2),
    own affine map. `ops` is cycled through (default: all warps)."""
    rng = np.random.default_rng(seed)
    items = []
    for i in range(n):
        H = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        W = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        k = rng.uniform(0.25, 2.0)
        h = max(1, int(round(k * H)))
        w = max(1, int(round(k * W)))
        op = ops[i % len(ops)]
        if op == OP_GRAY:
            h, w = H, W
        M = random_inverse_affine(rng, H, W, h, w, k)
        items.append(RaggedItem(op, H, W, h, w, M, seed * 100003 + i))
    return items


@dataclass
class Request:
    t_arrival: float   # seconds from stream start
    op: int
    H: int
    W: int
    h: int
    w: int
    M: np.ndarray
    src_index: int     # index into a pool of pre-generated source images


def request_stream(seed: int, rate: float, duration: float, pool: int = 64) -> list:
    """Poisson arrivals at `rate` req/s for `duration` s. Each request names a source image
    of the pool by index; the pool's sizes come from `pool_sizes(seed, pool)`."""
    rng = np.random.default_rng(seed)
    sizes = pool_sizes(seed, pool)
    t = 0.0
    out = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        j = int(rng.integers(0, pool))
        H, W = sizes[j]
        op = int(rng.integers(0, 3))
        if op == OP_RESIZE:
            k = rng.uniform(0.25, 2.0)
            h, w = max(1, int(round(k * H))), max(1, int(round(k * W)))
            M = np.zeros((2, 3), dtype=np.float32)
        elif op == OP_WARP:
            h, w = H, W
            M = random_inverse_affine(rng, H, W)
        else:
            h, w = H, W
            M = np.zeros((2, 3), dtype=np.float32)
        out.append(Request(t, op, H, W, h, w, M, j))
    return out


def pool_sizes(seed: int, pool: int = 64) -> list:
    """(H, W) of the serving source pool: W log-uniform 320..3840, H log-uniform 240..2160."""
    rng = np.random.default_rng(seed + 7919)
    out = []
    for _ in range(pool):
        W = int(round(math.exp(rng.uniform(math.log(320), math.log(3840)))))
        H = int(round(math.exp(rng.uniform(math.log(240), math.log(2160)))))
        out.append((H, W))
    return out
