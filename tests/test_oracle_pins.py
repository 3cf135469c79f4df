"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself:
  * hand-worked cases (tests/golden/hand_cases.txt, each with its citation);
  * closed forms (2x downscale = 2x2 box mean rounded half up, 1.5x weights,
    same-size identity, constant images, integer shifts, flips, rot90);
  * an exact-rational brute force of the definitions (Fractions, with its own
    binary32 rounding to emulate the fp32 coordinate sequence);
  * library routines that compute the same special case: torch's bilinear
    ``interpolate`` (align_corners=False) and ``grid_sample`` (zeros padding)
    in float64, and the real-valued BT.601 formula;
  * error bounds derived from the fixed-point arithmetic (u8 vs exact).
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
from helpers import load_hand_cases, round_f32, fmaf_exact, sub_f32, f32
from paper_2505_12425_gb300 import inputs

# Fixed-point error bound of the u8 path: each 11-bit weight is within 1/4096
# of the exact fraction, so each of the two blends moves the value by at most
# 255/4096; the final half-up rounding adds 1/2.
U8_BOUND = 0.5 + 2 * 255.0 / 4096.0


# ---------------------------------------------------------------------------
# Hand-worked golden cases
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("case", load_hand_cases(), ids=lambda c: c["name"])
def test_hand_cases(case):
    src = case["in"]
    h, w, c = case["out"].shape
    if case["op"] == "resize_u8":
        got = oracle.resize_u8(src, h, w)
    elif case["op"] == "warp_u8":
        got = oracle.warp_u8(src, case["M"], h, w)
    elif case["op"] == "gray_u8":
        got = oracle.rgb_to_gray_u8(src)
    else:
        raise AssertionError(case["op"])
    np.testing.assert_array_equal(got, case["out"], err_msg=case["cite"])


# ---------------------------------------------------------------------------
# Closed forms and invariants
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("H,W,C", [(8, 6, 1), (10, 14, 3), (2, 2, 3)])
def test_resize_down2x_is_box_mean(H, W, C):
    img = inputs.uniform_image(11 + H, H, W, C)
    got = oracle.resize_u8(img, H // 2, W // 2).astype(np.int64)
    s = (img[0::2, 0::2].astype(np.int64) + img[0::2, 1::2] + img[1::2, 0::2] + img[1::2, 1::2])
    np.testing.assert_array_equal(got, (s + 2) >> 2)


def test_resize_1p5x_weights_alternate():
    for i in range(40):
        i0, i1, q, fr = oracle.resize_point(i, 60, 40)
        assert i0 == (3 * i) // 2 and i1 == i0 + 1
        assert q == (512 if i % 2 == 0 else 1536)
        assert fr == (0.25 if i % 2 == 0 else 0.75)


@pytest.mark.parametrize("H,W,C", [(1, 1, 1), (7, 5, 3), (33, 17, 3)])
def test_resize_same_size_is_identity(H, W, C):
    img = inputs.uniform_image(5, H, W, C)
    np.testing.assert_array_equal(oracle.resize_u8(img, H, W), img)
    np.testing.assert_allclose(oracle.resize_f64(img, H, W), img / 255.0, rtol=0, atol=1e-15)


@pytest.mark.parametrize("val", [0, 1, 127, 254, 255])
def test_constant_image_stays_constant(val):
    img = np.full((9, 13, 3), val, np.uint8)
    for h, w in [(4, 5), (18, 26), (9, 13), (1, 1), (31, 7)]:
        np.testing.assert_array_equal(oracle.resize_u8(img, h, w), np.full((h, w, 3), val))
        np.testing.assert_allclose(oracle.resize_f64(img, h, w), val / 255.0, atol=1e-14)
    M = inputs.warp_matrix(3, 9, 13)
    out = oracle.warp_u8(img, M, 9, 13).astype(int)
    # Wherever all four taps are inside, the value is exactly the constant.
    for y in range(9):
        for x in range(13):
            ok, sx, sy, x0, qx, y0, qy = oracle.warp_point(M, x, y)
            if ok and 0 <= x0 and x0 + 1 < 13 and 0 <= y0 and y0 + 1 < 9:
                assert out[y, x, 0] == val


def test_warp_identity_and_shift_and_flip_and_rot90():
    img = inputs.uniform_image(9, 12, 12, 3)
    ident = np.array([[1, 0, 0], [0, 1, 0]], np.float32)
    np.testing.assert_array_equal(oracle.warp_u8(img, ident, 12, 12), img)
    np.testing.assert_allclose(oracle.warp_f64(img, ident, 12, 12), img / 255.0, atol=1e-15)
    # integer translation: dst(x, y) = src(x + 3, y - 2), zero outside
    sh = np.array([[1, 0, 3], [0, 1, -2]], np.float32)
    exp = np.zeros_like(img)
    exp[2:, :9] = img[:10, 3:]
    np.testing.assert_array_equal(oracle.warp_u8(img, sh, 12, 12), exp)
    # horizontal flip
    fl = np.array([[-1, 0, 12], [0, 1, 0]], np.float32)
    np.testing.assert_array_equal(oracle.warp_u8(img, fl, 12, 12), img[:, ::-1])
    # rot90 about the centre: dst(x, y) = src(N - 1 - x, y) read as (row, col) = (N-1-x, y)
    r90 = np.array([[0, 1, 0], [-1, 0, 12]], np.float32)
    np.testing.assert_array_equal(oracle.warp_u8(img, r90, 12, 12), np.rot90(img, -1))
    # An integer-centre convention would be off by a half pixel and blend neighbours:
    assert not np.array_equal(oracle.warp_u8(img, np.array([[-1, 0, 11.5], [0, 1, 0]], np.float32),
                                             12, 12), img[:, ::-1])


def test_warp_nonfinite_and_huge_give_zero():
    img = np.full((4, 4, 3), 200, np.uint8)
    for M in ([[0, 0, np.nan], [0, 1, 0]], [[1, 0, 5e6], [0, 1, 0]], [[1, 0, 0], [0, 1, -5e6]],
              [[np.inf, 0, 0], [0, 1, 0]]):
        M = np.array(M, np.float32)
        np.testing.assert_array_equal(oracle.warp_u8(img, M, 4, 4), 0)
        np.testing.assert_array_equal(oracle.warp_f64(img, M, 4, 4), 0.0)
        assert not oracle.warp_point(M, 1, 1)[0]
    # The range limit is |s| < 2^22 on each axis separately.
    assert oracle.warp_point(np.array([[0, 0, 4194303.5], [0, 0, 0.5]], np.float32), 0, 0)[0]
    assert not oracle.warp_point(np.array([[0, 0, 0.5], [0, 0, 4194304.5]], np.float32), 0, 0)[0]
    assert not oracle.warp_point(np.array([[0, 0, 0.5], [0, 0, -4194303.5]], np.float32), 0, 0)[0]


def test_gray_all_rgb_within_bound():
    # Every one of the 2^24 colours: |gray_u8 - exact BT.601| <= 1/2 + weight rounding.
    v = np.arange(1 << 24, dtype=np.uint32)
    img = np.stack([(v >> 16) & 255, (v >> 8) & 255, v & 255], -1).astype(np.uint8).reshape(4096, 4096, 3)
    got = oracle.rgb_to_gray_u8(img)[..., 0].astype(np.float64)
    exact = img[..., 0] * 0.299 + img[..., 1] * 0.587 + img[..., 2] * 0.114
    wbound = 255 * (abs(4899 / 16384 - 0.299) + abs(9617 / 16384 - 0.587) + abs(1868 / 16384 - 0.114))
    assert np.max(np.abs(got - exact)) <= 0.5 + wbound + 1e-9
    # and the weights are BT.601 rounded to 14 bits
    assert [round(c * 16384) for c in (0.299, 0.587, 0.114)] == [4899, 9617, 1868]


# ---------------------------------------------------------------------------
# Library routines: torch bilinear interpolate / grid_sample in float64
# ---------------------------------------------------------------------------
def _torch_resize(img, h, w):
    t = torch.from_numpy(img.astype(np.float64) / 255.0).permute(2, 0, 1)[None]
    out = F.interpolate(t, size=(h, w), mode="bilinear", align_corners=False, antialias=False)
    return out[0].permute(1, 2, 0).numpy()


@pytest.mark.parametrize("H,W,h,w", [(17, 23, 9, 40), (30, 20, 7, 7), (5, 64, 13, 3),
                                     (48, 64, 32, 43), (3, 3, 10, 10), (1, 9, 4, 2)])
def test_resize_vs_torch_interpolate(H, W, h, w):
    img = inputs.uniform_image(H * 1000 + W, H, W, 3)
    ref = _torch_resize(img, h, w)
    got = oracle.resize_f64(img, h, w)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)
    got8 = oracle.resize_u8(img, h, w).astype(np.float64)
    assert np.max(np.abs(got8 - 255.0 * ref)) <= U8_BOUND + 1e-9


def _torch_warp(img, M, h, w):
    """grid_sample (bilinear, zeros, align_corners=False) at float64 coordinates
    sx = m00 (x+1/2) + m01 (y+1/2) + m02 - 1/2."""
    H, W, _ = img.shape
    M = M.astype(np.float64)
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    sx = M[0, 0] * (xs + 0.5) + M[0, 1] * (ys + 0.5) + M[0, 2] - 0.5
    sy = M[1, 0] * (xs + 0.5) + M[1, 1] * (ys + 0.5) + M[1, 2] - 0.5
    gx = (2 * sx + 1) / W - 1
    gy = (2 * sy + 1) / H - 1
    grid = torch.from_numpy(np.stack([gx, gy], -1))[None]
    t = torch.from_numpy(img.astype(np.float64) / 255.0).permute(2, 0, 1)[None]
    out = F.grid_sample(t, grid, mode="bilinear", padding_mode="zeros", align_corners=False)
    return out[0].permute(1, 2, 0).numpy()


@pytest.mark.parametrize("seed", range(6))
def test_warp_vs_torch_grid_sample(seed):
    H, W = 24 + seed, 31 - seed
    img = inputs.noise_gradient_image(seed, H, W, 3)
    rng = np.random.default_rng(seed)
    M = inputs.random_inverse_affine(rng, H, W)
    ref = _torch_warp(img, M, H, W)
    got = oracle.warp_f64(img, M, H, W)
    # Only the fp32 rounding of the coordinate separates the two (|s| < 64 here,
    # so the coordinate differs by < 2^-17 and the value by < 2 * 2^-17).
    np.testing.assert_allclose(got, ref, rtol=0, atol=2e-5)
    got8 = oracle.warp_u8(img, M, H, W).astype(np.float64)
    assert np.max(np.abs(got8 - 255.0 * ref)) <= U8_BOUND + 255 * 2e-5


def test_normalise_and_gray_are_affine_in_the_interpolant():
    img = inputs.uniform_image(77, 20, 30, 3)
    mean, std = inputs.IMAGENET_MEAN, inputs.IMAGENET_STD
    plain = oracle.resize_f64(img, 11, 17)
    norm = oracle.resize_f64(img, 11, 17, mean=mean, std=std)
    np.testing.assert_allclose(norm, (plain - np.array(mean)) / np.array(std), atol=1e-13)
    g = oracle.resize_f64(img, 11, 17, gray=True, mean=mean, std=std)
    gp = plain @ np.array([0.299, 0.587, 0.114])
    np.testing.assert_allclose(g[..., 0], (gp - mean[0]) / std[0], atol=1e-13)
    M = inputs.warp_matrix(4, 20, 30)
    wp = oracle.warp_f64(img, M, 20, 30)
    wg = oracle.warp_f64(img, M, 20, 30, gray=True)
    np.testing.assert_allclose(wg[..., 0], wp @ np.array([0.299, 0.587, 0.114]), atol=1e-13)


def test_fused_gray_u8_equals_composition():
    img = inputs.uniform_image(8, 21, 19, 3)
    r = oracle.resize_u8(img, 10, 33)
    np.testing.assert_array_equal(oracle.resize_u8(img, 10, 33, gray=True), oracle.rgb_to_gray_u8(r))
    M = inputs.warp_matrix(8, 21, 19)
    wv = oracle.warp_u8(img, M, 21, 19)
    np.testing.assert_array_equal(oracle.warp_u8(img, M, 21, 19, gray=True), oracle.rgb_to_gray_u8(wv))


# ---------------------------------------------------------------------------
# Exact-rational brute force
# ---------------------------------------------------------------------------
def _brute_resize_axis(i, n_in, n_out):
    s = (Fraction(i) + Fraction(1, 2)) * Fraction(n_in, n_out) - Fraction(1, 2)
    if s <= 0:
        i0, fr = 0, Fraction(0)
    elif s >= n_in - 1:
        i0, fr = n_in - 1, Fraction(0)
    else:
        i0 = math.floor(s)
        fr = s - i0
    q = math.floor(2048 * fr + Fraction(1, 2))
    return i0, min(i0 + 1, n_in - 1), q, fr


def _brute_resize_u8(img, h, w):
    H, W, C = img.shape
    out = np.zeros((h, w, C), np.uint8)
    for y in range(h):
        y0, y1, qy, _ = _brute_resize_axis(y, H, h)
        for x in range(w):
            x0, x1, qx, _ = _brute_resize_axis(x, W, w)
            for c in range(C):
                v = (Fraction(int(img[y0, x0, c]) * (2048 - qx) * (2048 - qy))
                     + int(img[y0, x1, c]) * qx * (2048 - qy)
                     + int(img[y1, x0, c]) * (2048 - qx) * qy
                     + int(img[y1, x1, c]) * qx * qy) / 2 ** 22
                out[y, x, c] = math.floor(v + Fraction(1, 2))
    return out


def test_resize_brute_force_all_small_sizes():
    rng = np.random.default_rng(2024)
    for W in range(1, 9):
        for w in range(1, 9):
            for H, h in [(1, 1), (2, 5), (3, 2), (5, 3), (4, 8)]:
                img = rng.integers(0, 256, (H, W, 1), dtype=np.uint8)
                np.testing.assert_array_equal(oracle.resize_u8(img, h, w), _brute_resize_u8(img, h, w),
                                              err_msg=f"{H}x{W}->{h}x{w}")
                for x in range(w):
                    i0, i1, q, fr = oracle.resize_point(x, W, w)
                    b = _brute_resize_axis(x, W, w)
                    assert (i0, i1, q) == b[:3] and fr == float(b[3])


def _brute_warp_point(M, x, y):
    m = [f32(v) for v in np.asarray(M, np.float32).reshape(6)]
    xc = round_f32(Fraction(x) + Fraction(1, 2))
    yc = round_f32(Fraction(y) + Fraction(1, 2))
    sx = sub_f32(fmaf_exact(m[0], xc, fmaf_exact(m[1], yc, m[2])), Fraction(1, 2))
    sy = sub_f32(fmaf_exact(m[3], xc, fmaf_exact(m[4], yc, m[5])), Fraction(1, 2))
    if not (abs(sx) < 2 ** 22 and abs(sy) < 2 ** 22):
        return False, sx, sy, None, None, None, None

    def weight(s):
        k0 = math.floor(s)
        f = sub_f32(s, k0)
        t = f * 2048                      # exact: scaling by 2^11
        k = math.floor(t)
        return k0, k + (1 if t - k >= Fraction(1, 2) else 0)

    x0, qx = weight(sx)
    y0, qy = weight(sy)
    return True, sx, sy, x0, qx, y0, qy


def test_round_f32_matches_numpy_on_doubles():
    rng = np.random.default_rng(1)
    for v in np.concatenate([rng.normal(0, 1e3, 2000), rng.normal(0, 1e-3, 500), [0.1, 1 / 3, 2049.5]]):
        assert round_f32(Fraction(float(v))) == Fraction(float(np.float32(v)))


def _matrices():
    rng = np.random.default_rng(77)
    mats = [np.array([[1, 0, 0], [0, 1, 0]], np.float32),
            np.array([[0.5, 0.25, 1.75], [-0.25, 1.5, -2.0]], np.float32),   # dyadic
            np.array([[-1, 0, 8], [0, -1, 8]], np.float32),
            np.array([[1, 0, -0.3], [0, 1, -0.7]], np.float32)]             # negative fractions
    for _ in range(12):
        mats.append(inputs.random_inverse_affine(rng, 8, 8))
    return mats


@pytest.mark.parametrize("k", range(16))
def test_warp_brute_force_point_and_image(k):
    M = _matrices()[k]
    img = inputs.uniform_image(k, 8, 8, 3)
    exp = np.zeros((8, 8, 3), np.uint8)
    for y in range(8):
        for x in range(8):
            ok, sx, sy, x0, qx, y0, qy = _brute_warp_point(M, x, y)
            got = oracle.warp_point(M, x, y)
            assert got[0] == ok
            assert Fraction(got[1]) == sx and Fraction(got[2]) == sy
            if not ok:
                continue
            assert got[3:] == (x0, qx, y0, qy)
            for c in range(3):
                def tap(yy, xx):
                    return int(img[yy, xx, c]) if 0 <= xx < 8 and 0 <= yy < 8 else 0
                v = Fraction(tap(y0, x0) * (2048 - qx) * (2048 - qy) + tap(y0, x0 + 1) * qx * (2048 - qy)
                             + tap(y0 + 1, x0) * (2048 - qx) * qy + tap(y0 + 1, x0 + 1) * qx * qy, 2 ** 22)
                exp[y, x, c] = math.floor(v + Fraction(1, 2))
    np.testing.assert_array_equal(oracle.warp_u8(img, M, 8, 8), exp)


# ---------------------------------------------------------------------------
# Touched-byte counter (the benchmark's algorithmic input bytes)
# ---------------------------------------------------------------------------
def test_touched_dense_resize_reads_every_pixel():
    img = inputs.uniform_image(1, 60, 90, 3)
    _, t = oracle.resize_u8(img, 40, 60, touched=True)          # 1.5x
    assert t.all() and oracle.touched_bytes(t, 3) == 60 * 90 * 3
    _, t = oracle.resize_u8(img, 30, 45, touched=True)          # 2x: weights 1024 each
    assert t.all()


def test_touched_integer_shift_reads_the_shifted_window():
    img = inputs.uniform_image(1, 10, 12, 3)
    sh = np.array([[1, 0, 3], [0, 1, -2]], np.float32)
    _, t = oracle.warp_u8(img, sh, 10, 12, touched=True)
    exp = np.zeros((10, 12), np.uint8)
    exp[:8, 3:] = 1                       # rows 0..7 and columns 3..11 are read
    np.testing.assert_array_equal(t, exp)


def test_touched_sparse_downscale_counts_rows_and_columns():
    img = inputs.uniform_image(2, 216, 384, 3)
    _, t = oracle.resize_f64(img, 22, 22, touched=True)
    rows = {oracle.resize_point(y, 216, 22)[0] for y in range(22)} | \
           {oracle.resize_point(y, 216, 22)[1] for y in range(22)}
    cols = {oracle.resize_point(x, 384, 22)[0] for x in range(22)} | \
           {oracle.resize_point(x, 384, 22)[1] for x in range(22)}
    assert oracle.touched_bytes(t, 3) == len(rows) * len(cols) * 3
    # sector-granular count is at least the pixel count and at most 2 sectors per pixel
    sec = oracle.touched_bytes(t, 3, sector=32)
    assert len(rows) * len(cols) * 3 <= sec <= len(rows) * len(cols) * 2 * 32


# ---------------------------------------------------------------------------
# Nearest-neighbour resize and horizontal flip
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("C", [1, 3])
def test_nearest_same_size_is_identity(C):
    img = inputs.uniform_image(70, 23, 41, C)
    np.testing.assert_array_equal(oracle.resize_nearest_u8(img, 23, 41), img)


@pytest.mark.parametrize("ky,kx", [(2, 2), (3, 1), (1, 4), (5, 3)])
def test_nearest_integer_upscale_repeats_each_pixel(ky, kx):
    img = inputs.uniform_image(71, 9, 13, 3)
    ref = np.repeat(np.repeat(img, ky, axis=0), kx, axis=1)
    np.testing.assert_array_equal(oracle.resize_nearest_u8(img, 9 * ky, 13 * kx), ref)


@pytest.mark.parametrize("k", [2, 3, 4, 7])
def test_nearest_integer_downscale_takes_the_centre_pixel_of_each_block(k):
    # each k x k block's centre lies in pixel k // 2 of the block
    img = inputs.uniform_image(72, 5 * k, 6 * k, 3)
    ref = img[k // 2::k, k // 2::k]
    np.testing.assert_array_equal(oracle.resize_nearest_u8(img, 5, 6), ref)


def test_nearest_brute_force_exact_rationals():
    rng = np.random.default_rng(73)
    for _ in range(12):
        H, W, h, w = (int(v) for v in rng.integers(1, 40, 4))
        img = inputs.uniform_image(int(rng.integers(1 << 30)), H, W, 3)
        got = oracle.resize_nearest_u8(img, h, w)
        ys = [math.floor((Fraction(y) + Fraction(1, 2)) * H / h) for y in range(h)]
        xs = [math.floor((Fraction(x) + Fraction(1, 2)) * W / w) for x in range(w)]
        np.testing.assert_array_equal(got, img[np.ix_(ys, xs)])


@pytest.mark.parametrize("C", [1, 3])
def test_flip_reverses_columns_and_is_an_involution(C):
    img = inputs.uniform_image(74, 17, 29, C)
    f = oracle.flip_h_u8(img)
    np.testing.assert_array_equal(f, img[:, ::-1])
    np.testing.assert_array_equal(oracle.flip_h_u8(f), img)


def test_flip_equals_the_warp_with_the_mirror_map():
    # the inverse map x_src = W - 1 - x has zero fraction: the bilinear warp copies pixels
    H, W = 19, 31
    img = inputs.uniform_image(75, H, W, 3)
    M = np.array([[-1, 0, W], [0, 1, 0]], np.float32)
    np.testing.assert_array_equal(oracle.flip_h_u8(img), oracle.warp_u8(img, M, H, W))


# ---------------------------------------------------------------------------
# Perspective warp
# ---------------------------------------------------------------------------
def _brute_persp_point(M, x, y):
    m = [f32(v) for v in np.asarray(M, np.float32).reshape(9)]
    xc = round_f32(Fraction(x) + Fraction(1, 2))
    yc = round_f32(Fraction(y) + Fraction(1, 2))
    X = fmaf_exact(m[0], xc, fmaf_exact(m[1], yc, m[2]))
    Y = fmaf_exact(m[3], xc, fmaf_exact(m[4], yc, m[5]))
    Z = fmaf_exact(m[6], xc, fmaf_exact(m[7], yc, m[8]))
    if not Z > 0:
        return False, None, None, None, None, None, None
    q = round_f32(1 / Z)
    sx = sub_f32(round_f32(X * q), Fraction(1, 2))
    sy = sub_f32(round_f32(Y * q), Fraction(1, 2))
    if not (abs(sx) < 2 ** 22 and abs(sy) < 2 ** 22):
        return False, sx, sy, None, None, None, None

    def weight(s):
        k0 = math.floor(s)
        f = sub_f32(s, k0)
        t = f * 2048
        k = math.floor(t)
        return k0, k + (1 if t - k >= Fraction(1, 2) else 0)

    x0, qx = weight(sx)
    y0, qy = weight(sy)
    return True, sx, sy, x0, qx, y0, qy


def _homographies():
    rng = np.random.default_rng(78)
    mats = [np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float32),
            np.array([[1, 0, 0], [0, 1, 0], [0.05, 0, 1]], np.float32),          # keystone in x
            np.array([[1, 0, 0], [0, 1, 0], [-0.3, 0.2, 1]], np.float32)]        # a horizon inside
    for _ in range(9):
        mats.append(inputs.random_inverse_homography(rng, 8, 8, tilt=0.8))
    return mats


@pytest.mark.parametrize("k", range(12))
def test_persp_brute_force_point_and_image(k):
    M = _homographies()[k]
    img = inputs.uniform_image(100 + k, 8, 8, 3)
    exp = np.zeros((8, 8, 3), np.uint8)
    for y in range(8):
        for x in range(8):
            ok, sx, sy, x0, qx, y0, qy = _brute_persp_point(M, x, y)
            got = oracle.persp_point(M, x, y)
            assert got[0] == ok
            if sx is not None:
                assert Fraction(got[1]) == sx and Fraction(got[2]) == sy
            if not ok:
                continue
            assert got[3:] == (x0, qx, y0, qy)
            for c in range(3):
                def tap(yy, xx):
                    return int(img[yy, xx, c]) if 0 <= xx < 8 and 0 <= yy < 8 else 0
                v = Fraction(tap(y0, x0) * (2048 - qx) * (2048 - qy) + tap(y0, x0 + 1) * qx * (2048 - qy)
                             + tap(y0 + 1, x0) * (2048 - qx) * qy + tap(y0 + 1, x0 + 1) * qx * qy, 2 ** 22)
                exp[y, x, c] = math.floor(v + Fraction(1, 2))
    np.testing.assert_array_equal(oracle.warp_persp_u8(img, M, 8, 8), exp)


@pytest.mark.parametrize("k", range(6))
def test_persp_with_affine_last_row_is_the_affine_warp(k):
    A = _matrices()[4 + k]
    M = np.vstack([A, [0, 0, 1]]).astype(np.float32)
    img = inputs.noise_gradient_image(110 + k, 40, 56)
    np.testing.assert_array_equal(oracle.warp_persp_u8(img, M, 33, 61), oracle.warp_u8(img, A, 33, 61))
    np.testing.assert_array_equal(oracle.warp_persp_f64(img, M, 33, 61), oracle.warp_f64(img, A, 33, 61))


def test_persp_is_invariant_to_power_of_two_scaling():
    # X, Y, Z all scale exactly, q = 1/Z scales exactly, X*q does not change
    img = inputs.noise_gradient_image(120, 50, 70)
    M = inputs.random_inverse_homography(np.random.default_rng(121), 50, 70, tilt=0.6)
    ref = oracle.warp_persp_u8(img, M, 50, 70)
    for s in (0.25, 2.0, 8.0):
        np.testing.assert_array_equal(oracle.warp_persp_u8(img, (M * s).astype(np.float32), 50, 70), ref)
    # a negative scale puts every point behind the camera: all zeros
    assert not oracle.warp_persp_u8(img, -M, 50, 70).any()


def test_persp_f64_is_within_the_fixed_point_bound_of_u8():
    img = inputs.noise_gradient_image(122, 60, 80)
    M = inputs.random_inverse_homography(np.random.default_rng(123), 60, 80, tilt=0.5)
    u8 = oracle.warp_persp_u8(img, M, 60, 80).astype(np.float64)
    f = oracle.warp_persp_f64(img, M, 60, 80) * 255.0
    assert np.abs(u8 - f).max() <= U8_BOUND


# ---------------------------------------------------------------------------
# Sobel 3x3
# ---------------------------------------------------------------------------
def test_sobel_of_a_constant_image_is_zero():
    f, u = oracle.sobel(np.full((9, 11, 3), 77, np.uint8))
    assert not f.any() and not u.any()


def test_sobel_of_a_ramp():
    # I = 3x: interior gx = (1 + 2 + 1) * (I(x+1) - I(x-1)) = 4 * 6 = 24 -> 24 / 8 = 3;
    # at the replicated edges the difference is one step: 4 * 3 / 8 = 1.5
    W = 12
    img = np.tile((3 * np.arange(W, dtype=np.uint8))[None, :, None], (7, 1, 1))
    f, u = oracle.sobel(img)
    np.testing.assert_array_equal(f[:, 1:-1, 0], 3.0)
    np.testing.assert_array_equal(f[:, [0, -1], 0], 1.5)
    np.testing.assert_array_equal(u[:, [0, -1], 0], 2)          # floor(1.5 + 0.5)


def test_sobel_matches_scipy_with_nearest_mode():
    ndimage = pytest.importorskip("scipy.ndimage")
    img = inputs.uniform_image(130, 31, 47, 1)
    f, u = oracle.sobel(img)
    g = img[..., 0].astype(np.float64)
    sx = ndimage.sobel(g, axis=1, mode="nearest")
    sy = ndimage.sobel(g, axis=0, mode="nearest")
    ref = np.hypot(sx, sy) / 8.0
    np.testing.assert_allclose(f[..., 0], ref, rtol=1e-6, atol=1e-6)
    away = np.abs(ref - np.floor(ref) - 0.5) > 1e-3                  # not at a rounding tie
    np.testing.assert_array_equal(u[..., 0][away], np.floor(ref + 0.5)[away])


def test_sobel_commutes_with_transpose_and_fuses_gray():
    img = inputs.noise_gradient_image(131, 23, 29)
    f, u = oracle.sobel(img)
    g = oracle.rgb_to_gray_u8(img)
    fg, ug = oracle.sobel(g)
    np.testing.assert_array_equal(f, fg)
    ft, _ = oracle.sobel(np.ascontiguousarray(g.transpose(1, 0, 2)))
    np.testing.assert_array_equal(ft, f.transpose(1, 0, 2))


# ---------------------------------------------------------------------------
# Replicate border (both warps)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dx,dy", [(3, -2), (-5, 4), (0, 7), (40, -30)])
def test_replicate_integer_shift_is_the_edge_padded_window(dx, dy):
    H, W = 21, 27
    img = inputs.uniform_image(140, H, W, 3)
    M = np.array([[1, 0, dx], [0, 1, dy]], np.float32)        # out(x, y) = in(x + dx, y + dy)
    ys = np.clip(np.arange(H) + dy, 0, H - 1)
    xs = np.clip(np.arange(W) + dx, 0, W - 1)
    ref = img[np.ix_(ys, xs)]
    np.testing.assert_array_equal(oracle.warp_u8(img, M, H, W, border="replicate"), ref)
    P = np.vstack([M, [0, 0, 1]]).astype(np.float32)
    np.testing.assert_array_equal(oracle.warp_persp_u8(img, P, H, W, border="replicate"), ref)


def test_replicate_matches_torch_grid_sample_border_mode():
    H, W = 17, 23
    img = inputs.uniform_image(141, H, W, 3)
    M = inputs.random_inverse_affine(np.random.default_rng(142), H, W, k=1.3)
    got = oracle.warp_f64(img, M, H, W, border="replicate")
    gx, gy = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    Md = M.astype(np.float64)
    sx = Md[0, 0] * gx + Md[0, 1] * gy + Md[0, 2]              # continuous source position
    sy = Md[1, 0] * gx + Md[1, 1] * gy + Md[1, 2]
    grid = torch.from_numpy(np.stack([2 * sx / W - 1, 2 * sy / H - 1], -1)[None])
    t = torch.from_numpy(img.transpose(2, 0, 1)[None].astype(np.float64) / 255.0)
    ref = F.grid_sample(t, grid, mode="bilinear", padding_mode="border", align_corners=False)[0]
    ref = ref.numpy().transpose(1, 2, 0)
    assert np.abs(got - ref).max() < 1e-5                        # fp32 vs fp64 coordinates


def test_replicate_equals_zero_border_inside_and_fills_outside():
    H, W = 30, 40
    img = inputs.noise_gradient_image(143, H, W)
    M = inputs.random_inverse_affine(np.random.default_rng(144), H, W)
    z = oracle.warp_u8(img, M, H, W)
    r = oracle.warp_u8(img, M, H, W, border="replicate")
    inside = np.zeros((H, W), bool)
    for y in range(H):
        for x in range(W):
            ok, sx, sy, *_ = oracle.warp_point(M, x, y)
            inside[y, x] = ok and 0 <= sx <= W - 1 and 0 <= sy <= H - 1 and math.floor(sx) + 1 < W \
                and math.floor(sy) + 1 < H
    np.testing.assert_array_equal(r[inside], z[inside])
    assert r[~inside].any() and (r[~inside] != z[~inside]).any()


# ---------------------------------------------------------------------------
# Area (antialiased) downscale
# ---------------------------------------------------------------------------
def test_area_same_size_is_identity():
    img = inputs.uniform_image(150, 13, 17, 3)
    np.testing.assert_array_equal(oracle.resize_area_u8(img, 13, 17), img)


@pytest.mark.parametrize("ky,kx", [(2, 2), (3, 5), (4, 1), (17, 17)])
def test_area_integer_factor_is_the_block_mean_rounded_half_up(ky, kx):
    h, w = 5, 4
    img = inputs.uniform_image(151, h * ky, w * kx, 3)
    blocks = img.reshape(h, ky, w, kx, 3).astype(np.int64).sum(axis=(1, 3))
    n = ky * kx
    ref = (2 * blocks + n) // (2 * n)
    np.testing.assert_array_equal(oracle.resize_area_u8(img, h, w), ref)
    t = torch.from_numpy(img.transpose(2, 0, 1)[None].astype(np.float64) / 255.0)
    pooled = F.avg_pool2d(t, (ky, kx))[0].numpy().transpose(1, 2, 0)
    np.testing.assert_allclose(oracle.resize_area_f64(img, h, w), pooled, atol=1e-12)


def test_area_brute_force_exact_overlaps():
    rng = np.random.default_rng(152)
    for _ in range(10):
        H, W = (int(v) for v in rng.integers(2, 24, 2))
        h, w = int(rng.integers(1, H + 1)), int(rng.integers(1, W + 1))
        img = inputs.uniform_image(int(rng.integers(1 << 30)), H, W, 1)
        got = oracle.resize_area_u8(img, h, w)
        gotf = oracle.resize_area_f64(img, h, w)
        for y in range(h):
            for x in range(w):
                fx0, fx1 = Fraction(x * W, w), Fraction((x + 1) * W, w)
                fy0, fy1 = Fraction(y * H, h), Fraction((y + 1) * H, h)
                acc = Fraction(0)
                for j in range(H):
                    oy = min(fy1, j + 1) - max(fy0, j)
                    if oy <= 0:
                        continue
                    for i in range(W):
                        ox = min(fx1, i + 1) - max(fx0, i)
                        if ox > 0:
                            acc += ox * oy * int(img[j, i, 0])
                mean = acc / ((fx1 - fx0) * (fy1 - fy0))
                assert got[y, x, 0] == math.floor(mean + Fraction(1, 2))
                assert abs(gotf[y, x, 0] - float(mean) / 255.0) < 1e-12


def test_area_of_a_constant_image_is_the_constant_and_preserves_the_mean():
    np.testing.assert_array_equal(oracle.resize_area_u8(np.full((37, 53, 3), 201, np.uint8), 11, 7), 201)
    img = inputs.uniform_image(153, 60, 90, 3)
    f = oracle.resize_area_f64(img, 7, 13)                # the footprints tile the source exactly
    np.testing.assert_allclose(f.mean(axis=(0, 1)), img.reshape(-1, 3).mean(0) / 255.0, rtol=1e-12)
