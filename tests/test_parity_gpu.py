"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

u8 results are compared bit for bit; f32 results within 1e-5 absolute (the
tolerance of the f32 path). Sizes span several tiles with ragged tails, and
include the full-size workloads (640x480 -> 320x240; 1920x1080 resize and
warp; 16 x 3840x2160 -> 224x224 normalised NCHW). Destinations carry guard
bands of canary bytes that must survive every call.
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
CANARY_U8 = 0xA5
CANARY_F32 = -12345.0
MEAN, STD = inputs.IMAGENET_MEAN, inputs.IMAGENET_STD


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()
    kr.load()


def dev():
    return torch.device("cuda:0")


class Guarded:
    """A destination tensor inside a canary-filled buffer (guard bands before and after)."""

    def __init__(self, shape, dtype, guard=256):
        n = int(np.prod(shape))
        fill = CANARY_U8 if dtype == torch.uint8 else CANARY_F32
        self.buf = torch.full((guard + n + guard,), fill, dtype=dtype, device=dev())
        self.t = self.buf[guard:guard + n].view(*shape)
        self.guard, self.n, self.fill = guard, n, fill

    def check(self):
        b = self.buf.cpu().numpy()
        assert np.all(b[:self.guard] == self.fill), "write before the destination"
        assert np.all(b[self.guard + self.n:] == self.fill), "write after the destination"

    def np(self):
        return self.t.cpu().numpy()


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


# ---------------------------------------------------------------------------
# Resize
# ---------------------------------------------------------------------------
RESIZE_CASES = [
    (480, 640, 240, 320, 3),      # 640x480 -> 320x240 (full size)
    (1080, 1920, 720, 1280, 3),   # 1920x1080 -> 1280x720 (full size)
    (37, 53, 91, 17, 3), (100, 100, 33, 47, 1), (1, 1, 5, 7, 3), (1, 200, 1, 64, 3),
    (200, 1, 64, 1, 1), (64, 64, 64, 64, 3), (33, 65, 130, 258, 3), (500, 700, 50, 70, 3),
    (70, 90, 140, 181, 1), (257, 129, 65, 97, 3),
]


@pytest.mark.parametrize("H,W,h,w,C", RESIZE_CASES)
def test_resize_u8(H, W, h, w, C):
    img = inputs.uniform_image(H * 7 + W, H, W, C)
    out = Guarded((h, w, C), torch.uint8)
    kr.kr_resize_bilinear(to_dev(img), out.t)
    torch.cuda.synchronize()
    out.check()
    np.testing.assert_array_equal(out.np(), oracle.resize_u8(img, h, w))


@pytest.mark.parametrize("H,W,h,w", [(1080, 1920, 720, 1280), (45, 77, 100, 31), (300, 200, 37, 301)])
def test_resize_u8_gray(H, W, h, w):
    img = inputs.noise_gradient_image(3, H, W)
    out = Guarded((h, w, 1), torch.uint8)
    kr.kr_resize_bilinear(to_dev(img), out.t, gray=True)
    torch.cuda.synchronize()
    out.check()
    np.testing.assert_array_equal(out.np(), oracle.resize_u8(img, h, w, gray=True))


@pytest.mark.parametrize("layout", ["hwc", "chw"])
@pytest.mark.parametrize("H,W,h,w,C", [(1080, 1920, 720, 1280, 3), (50, 61, 129, 33, 3), (90, 70, 45, 140, 1)])
def test_resize_f32(H, W, h, w, C, layout):
    img = inputs.noise_gradient_image(5, H, W, C)
    shape = (h, w, C) if layout == "hwc" else (C, h, w)
    out = Guarded(shape, torch.float32)
    kr.kr_resize_bilinear(to_dev(img), out.t, mean=MEAN[:C], std=STD[:C], dst_layout=layout)
    torch.cuda.synchronize()
    out.check()
    got = out.np() if layout == "hwc" else out.np().transpose(1, 2, 0)
    ref = oracle.resize_f64(img, h, w, mean=MEAN[:C], std=STD[:C])
    assert np.abs(got - ref).max() <= F32_TOL


def test_resize_f32_plain_and_gray():
    img = inputs.uniform_image(8, 123, 211, 3)
    out = Guarded((77, 300, 3), torch.float32)
    kr.kr_resize_bilinear(to_dev(img), out.t)      # no normalisation: p / 255
    g = Guarded((77, 300, 1), torch.float32)
    kr.kr_resize_bilinear(to_dev(img), g.t, gray=True, mean=MEAN, std=STD)
    torch.cuda.synchronize()
    out.check()
    g.check()
    assert np.abs(out.np() - oracle.resize_f64(img, 77, 300)).max() <= F32_TOL
    assert np.abs(g.np() - oracle.resize_f64(img, 77, 300, gray=True, mean=MEAN, std=STD)).max() <= F32_TOL


def test_resize_16x4k_to_224_normalised_nchw():
    """16 uniform 3840x2160 images -> 224x224 f32 NCHW with per-channel mean/std, one launch."""
    n, H, W = 16, 2160, 3840
    imgs = inputs.uniform_batch(1002, n, H, W, 3)
    src = to_dev(imgs)
    out = Guarded((n, 3, 224, 224), torch.float32)
    kr.kr_resize_bilinear(src, out.t, mean=MEAN, std=STD, dst_layout="chw")
    torch.cuda.synchronize()
    out.check()
    got = out.np()
    for i in range(n):
        ref = oracle.resize_f64(imgs[i], 224, 224, mean=MEAN, std=STD)
        assert np.abs(got[i].transpose(1, 2, 0) - ref).max() <= F32_TOL, i


# ---------------------------------------------------------------------------
# Warp
# ---------------------------------------------------------------------------
WARP_CASES = [(1080, 1920, 3, 11), (77, 131, 3, 1), (64, 64, 1, 2), (300, 41, 3, 3), (5, 9, 3, 4), (129, 257, 1, 5)]


@pytest.mark.parametrize("H,W,C,seed", WARP_CASES)
def test_warp_u8(H, W, C, seed):
    img = inputs.noise_gradient_image(seed, H, W, C)
    M = inputs.warp_matrix(seed, H, W)
    out = Guarded((H, W, C), torch.uint8)
    kr.kr_warp_affine(to_dev(img), out.t, M)
    torch.cuda.synchronize()
    out.check()
    np.testing.assert_array_equal(out.np(), oracle.warp_u8(img, M, H, W))


@pytest.mark.parametrize("H,W,seed", [(1080, 1920, 12), (99, 160, 3)])
def test_warp_u8_gray(H, W, seed):
    img = inputs.noise_gradient_image(seed, H, W)
    M = inputs.warp_matrix(seed, H, W)
    out = Guarded((H, W, 1), torch.uint8)
    kr.kr_warp_affine(to_dev(img), out.t, M, gray=True)
    torch.cuda.synchronize()
    out.check()
    np.testing.assert_array_equal(out.np(), oracle.warp_u8(img, M, H, W, gray=True))


@pytest.mark.parametrize("layout", ["hwc", "chw"])
@pytest.mark.parametrize("H,W,seed", [(1080, 1920, 13), (71, 90, 4)])
def test_warp_f32(H, W, seed, layout):
    img = inputs.noise_gradient_image(seed, H, W)
    M = inputs.warp_matrix(seed, H, W)
    shape = (H, W, 3) if layout == "hwc" else (3, H, W)
    out = Guarded(shape, torch.float32)
    kr.kr_warp_affine(to_dev(img), out.t, M, mean=MEAN, std=STD, dst_layout=layout)
    g = Guarded((H, W, 1), torch.float32)
    kr.kr_warp_affine(to_dev(img), g.t, M, gray=True)
    torch.cuda.synchronize()
    out.check()
    g.check()
    got = out.np() if layout == "hwc" else out.np().transpose(1, 2, 0)
    assert np.abs(got - oracle.warp_f64(img, M, H, W, mean=MEAN, std=STD)).max() <= F32_TOL
    assert np.abs(g.np() - oracle.warp_f64(img, M, H, W, gray=True)).max() <= F32_TOL


def _special_matrices(H, W):
    return {
        "identity": [[1, 0, 0], [0, 1, 0]],
        "hflip": [[-1, 0, W], [0, 1, 0]],
        "shift": [[1, 0, 3], [0, 1, -2]],
        "half_shift": [[1, 0, 0.5], [0, 1, -0.25]],
        "far_away": [[1, 0, 1e5], [0, 1, 0]],
        "huge": [[1, 0, 5e6], [0, 1, 5e6]],
        "zoom_in_x8": [[0.125, 0, 3.3], [0, 0.125, 2.1]],
        "zoom_out_x9": [[9.1, 0.3, -40], [-0.2, 8.7, -33]],
        "shear": [[1, 0.7, -20], [0.1, 1, 0]],
        "degenerate_row": [[0, 0, 10.5], [0, 0, 5.25]],
        "negative_frac": [[1, 0, -0.3], [0, 1, -0.7]],
    }


@pytest.mark.parametrize("H,W", [(67, 93), (64, 96)])     # 96 * 3 bytes per row: TMA staging
@pytest.mark.parametrize("name", list(_special_matrices(1, 1)))
def test_warp_special_matrices(name, H, W):
    img = inputs.uniform_image(21, H, W, 3)
    M = np.array(_special_matrices(H, W)[name], np.float32)
    out = Guarded((H, W, 3), torch.uint8)
    kr.kr_warp_affine(to_dev(img), out.t, M)
    f = Guarded((H, W, 3), torch.float32)
    kr.kr_warp_affine(to_dev(img), f.t, M)
    torch.cuda.synchronize()
    out.check()
    f.check()
    np.testing.assert_array_equal(out.np(), oracle.warp_u8(img, M, H, W))
    assert np.abs(f.np() - oracle.warp_f64(img, M, H, W)).max() <= F32_TOL
    if name == "identity":
        np.testing.assert_array_equal(out.np(), img)
    if name == "hflip":
        np.testing.assert_array_equal(out.np(), img[:, ::-1])


def test_warp_output_size_differs_from_source():
    img = inputs.uniform_image(2, 150, 260, 3)
    rng = np.random.default_rng(9)
    M = inputs.random_inverse_affine(rng, 150, 260, 333, 95, k=1.7)
    out = Guarded((333, 95, 3), torch.uint8)
    kr.kr_warp_affine(to_dev(img), out.t, M)
    torch.cuda.synchronize()
    out.check()
    np.testing.assert_array_equal(out.np(), oracle.warp_u8(img, M, 333, 95))


# ---------------------------------------------------------------------------
# Views, pitches and batches
# ---------------------------------------------------------------------------
def test_views_with_odd_pitch_and_offset():
    H, W = 83, 129
    img = inputs.uniform_image(31, H, W, 3)
    big = torch.full((H + 5, W + 3, 3), 7, dtype=torch.uint8, device=dev())
    big[2:2 + H, 1:1 + W] = to_dev(img)
    src = big[2:2 + H, 1:1 + W]                          # pitch (W+3)*3 = 396, offset 2*396 + 3
    dbig = torch.full((60, 77, 3), CANARY_U8, dtype=torch.uint8, device=dev())
    dst = dbig[3:3 + 51, 5:5 + 70]                       # odd offset, pitch 231
    kr.kr_resize_bilinear(src, dst)
    M = inputs.warp_matrix(31, H, W)
    wbig = torch.full((H + 2, W + 1, 3), CANARY_U8, dtype=torch.uint8, device=dev())
    wdst = wbig[1:1 + H, 1:1 + W]
    kr.kr_warp_affine(src, wdst, M)
    gbig = torch.full((H + 3, W + 5), CANARY_U8, dtype=torch.uint8, device=dev())
    gdst = gbig[1:1 + H, 3:3 + W]
    kr.kr_rgb_to_gray(src, gdst)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(dst.cpu().numpy(), oracle.resize_u8(img, 51, 70))
    np.testing.assert_array_equal(wdst.cpu().numpy(), oracle.warp_u8(img, M, H, W))
    np.testing.assert_array_equal(gdst.cpu().numpy()[..., None], oracle.rgb_to_gray_u8(img))
    for b, sl in ((dbig, (slice(3, 54), slice(5, 75))), (wbig, (slice(1, 1 + H), slice(1, 1 + W))),
                  (gbig, (slice(1, 1 + H), slice(3, 3 + W)))):
        m = torch.ones(b.shape[:2], dtype=torch.bool, device=dev())
        m[sl] = False
        assert bool((b[m] == CANARY_U8).all()), "write outside the destination view"


@pytest.mark.parametrize("W", [100, 101])
def test_tma_staging_of_padded_views(W):
    # Rows of W pixels inside rows of 112 (336 bytes, a multiple of 16) that start 16-byte
    # aligned. W = 100 (300 bytes, a whole number of words): the source is staged by TMA;
    # W = 101 (303 bytes): by bulk row copies. The row padding (set to 200 here) must never
    # be read: right of each row the staged box holds zeros, the zero border of warp boxes.
    n, H, Wp = 3, 150, 112
    imgs = np.stack([inputs.noise_gradient_image(60 + i, H, W) for i in range(n)])
    big = torch.full((n, H, Wp, 3), 200, dtype=torch.uint8, device=dev())
    big[:, :, :W] = to_dev(imgs)
    src = big[:, :, :W]
    Ms = inputs.warp_matrices(60, n, H, W)
    wu = Guarded((n, H, W, 3), torch.uint8)
    kr.kr_warp_affine(src, wu.t, Ms)
    wf = Guarded((n, 3, H, W), torch.float32)
    kr.kr_warp_affine(src, wf.t, Ms, mean=MEAN, std=STD, dst_layout="chw")
    wg = Guarded((n, H, W, 1), torch.uint8)
    kr.kr_warp_affine(src, wg.t, Ms, gray=True)
    r = Guarded((n, 77, 190, 3), torch.uint8)
    kr.kr_resize_bilinear(src, r.t)
    torch.cuda.synchronize()
    for g in (wu, wf, wg, r):
        g.check()
    for i in range(n):
        np.testing.assert_array_equal(wu.np()[i], oracle.warp_u8(imgs[i], Ms[i], H, W))
        np.testing.assert_array_equal(wg.np()[i], oracle.warp_u8(imgs[i], Ms[i], H, W, gray=True))
        ref = oracle.warp_f64(imgs[i], Ms[i], H, W, mean=MEAN, std=STD)
        assert np.abs(wf.np()[i].transpose(1, 2, 0) - ref).max() <= F32_TOL
        np.testing.assert_array_equal(r.np()[i], oracle.resize_u8(imgs[i], 77, 190))


def test_batch_dimension_one_call():
    n, H, W, h, w = 5, 61, 97, 40, 130
    imgs = np.stack([inputs.noise_gradient_image(40 + i, H, W) for i in range(n)])
    Ms = inputs.warp_matrices(40, n, H, W)
    src = to_dev(imgs)
    r = Guarded((n, h, w, 3), torch.uint8)
    kr.kr_resize_bilinear(src, r.t)
    wu = Guarded((n, H, W, 3), torch.uint8)
    kr.kr_warp_affine(src, wu.t, Ms)
    wf = Guarded((n, 3, H, W), torch.float32)
    kr.kr_warp_affine(src, wf.t, Ms, mean=MEAN, std=STD, dst_layout="chw")
    torch.cuda.synchronize()
    for g in (r, wu, wf):
        g.check()
    for i in range(n):
        np.testing.assert_array_equal(r.np()[i], oracle.resize_u8(imgs[i], h, w))
        np.testing.assert_array_equal(wu.np()[i], oracle.warp_u8(imgs[i], Ms[i], H, W))
        ref = oracle.warp_f64(imgs[i], Ms[i], H, W, mean=MEAN, std=STD)
        assert np.abs(wf.np()[i].transpose(1, 2, 0) - ref).max() <= F32_TOL


def test_warp_batch_over_one_launch_limit():
    # more images than one launch carries matrices for: the library splits launches
    n, H, W = 130, 20, 24
    imgs = inputs.uniform_batch(5, n, H, W, 3)
    Ms = inputs.warp_matrices(5, n, H, W)
    out = Guarded((n, H, W, 3), torch.uint8)
    kr.kr_warp_affine(to_dev(imgs), out.t, Ms)
    torch.cuda.synchronize()
    out.check()
    got = out.np()
    for i in (0, 1, 127, 128, 129):
        np.testing.assert_array_equal(got[i], oracle.warp_u8(imgs[i], Ms[i], H, W))


@pytest.mark.parametrize("H,W", [(1080, 1920), (7, 13), (33, 16), (5, 47)])
def test_rgb_to_gray(H, W):
    img = inputs.uniform_image(H + W, H, W, 3)
    out = Guarded((H, W, 1), torch.uint8)
    kr.kr_rgb_to_gray(to_dev(img), out.t)
    torch.cuda.synchronize()
    out.check()
    np.testing.assert_array_equal(out.np(), oracle.rgb_to_gray_u8(img))


def test_errors_do_not_enqueue():
    src = torch.zeros((10, 10, 3), dtype=torch.uint8, device=dev())
    dst = torch.zeros((5, 5, 1), dtype=torch.uint8, device=dev())
    with pytest.raises(kr.KrError) as e:
        kr.kr_resize_bilinear(src, dst)           # channel mismatch without gray
    assert e.value.status == 1
    with pytest.raises(kr.KrError) as e:
        kr.kr_resize_bilinear(src, src[:5, :5])   # overlapping destination
    assert e.value.status == 3
    with pytest.raises(kr.KrError):
        kr.kr_warp_affine(src, src.clone(), [np.nan, 0, 0, 0, 1, 0])


# ---------------------------------------------------------------------------
# Nearest-neighbour resize and horizontal flip (pixel gathers)
# ---------------------------------------------------------------------------
NEAREST_CASES = [
    (480, 640, 240, 320, 3), (1080, 1920, 720, 1280, 3), (37, 53, 91, 17, 3), (100, 100, 33, 47, 1),
    (1, 1, 5, 7, 3), (1, 300, 1, 257, 3), (300, 1, 257, 1, 1), (64, 64, 64, 64, 3), (2160, 3840, 224, 224, 3),
    (33, 65, 130, 258, 1), (257, 129, 65, 97, 3),
    # source rows above 48 KB take the byte-gather kernel; the others are staged whole
    (3, 16400, 4, 301, 3), (2, 16371, 3, 20000, 3), (2, 16372, 3, 9, 3),
    # (2x + 1) W above 2^32: the first division of a row chunk needs 64 bits
    (2, 48000, 2, 65000, 1),
]


@pytest.mark.parametrize("H,W,h,w,C", NEAREST_CASES)
def test_resize_nearest(H, W, h, w, C):
    img = inputs.uniform_image(H * 7 + W, H, W, C)
    out = Guarded((h, w, C), torch.uint8)
    kr.kr_resize_nearest(to_dev(img), out.t)
    torch.cuda.synchronize()
    out.check()
    np.testing.assert_array_equal(out.np(), oracle.resize_nearest_u8(img, h, w))


@pytest.mark.parametrize("H,W,C", [(1080, 1920, 3), (17, 29, 3), (1, 1, 3), (5, 301, 1), (300, 2, 3),
                                   (3, 16371, 3), (3, 16372, 3), (2, 49114, 1), (2, 49115, 1), (2, 60001, 1)])
def test_flip_horizontal(H, W, C):
    img = inputs.uniform_image(H + 3 * W, H, W, C)
    out = Guarded((H, W, C), torch.uint8)
    kr.kr_flip_horizontal(to_dev(img), out.t)
    torch.cuda.synchronize()
    out.check()
    np.testing.assert_array_equal(out.np(), oracle.flip_h_u8(img))
    back = torch.empty_like(out.t)
    kr.kr_flip_horizontal(out.t, back)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(back.cpu().numpy(), img)


def test_gathers_on_views_and_batches():
    n, H, W = 3, 41, 77
    imgs = np.stack([inputs.uniform_image(80 + i, H, W, 3) for i in range(n)])
    big = torch.full((n, H + 4, W + 5, 3), 9, dtype=torch.uint8, device=dev())
    big[:, 2:2 + H, 3:3 + W] = to_dev(imgs)
    src = big[:, 2:2 + H, 3:3 + W]                                   # odd pitch and offset
    dbig = torch.full((n, 60, 90, 3), CANARY_U8, dtype=torch.uint8, device=dev())
    nd = dbig[:, 1:1 + 50, 2:2 + 63]
    fd = torch.full((n, H, W, 3), CANARY_U8, dtype=torch.uint8, device=dev())
    kr.kr_resize_nearest(src, nd)
    kr.kr_flip_horizontal(src, fd)
    torch.cuda.synchronize()
    m = torch.ones(dbig.shape[:3], dtype=torch.bool, device=dev())
    m[:, 1:51, 2:65] = False
    assert bool((dbig[m] == CANARY_U8).all()), "write outside the destination view"
    for i in range(n):
        np.testing.assert_array_equal(nd[i].cpu().numpy(), oracle.resize_nearest_u8(imgs[i], 50, 63))
        np.testing.assert_array_equal(fd[i].cpu().numpy(), oracle.flip_h_u8(imgs[i]))


@pytest.mark.parametrize("sx0,dx0", [(1, 0), (0, 3), (5, 2), (7, 7)])
def test_gathers_on_views_with_16_byte_pitches(sx0, dx0):
    # pitches and batch strides multiples of 16 with the first pixel at a byte phase: every row
    # and image shares the phase, the 3-channel path with one chunk per thread runs
    n, H, W = 3, 37, 101
    imgs = np.stack([inputs.uniform_image(90 + i, H, W, 3) for i in range(n)])
    big = torch.full((n, H, 112, 3), 7, dtype=torch.uint8, device=dev())
    big[:, :, sx0:sx0 + W] = to_dev(imgs)
    src = big[:, :, sx0:sx0 + W]
    for name, w in (("nearest", 70), ("nearest", 150), ("flip", W)):
        dbig = torch.full((n, 24 if name == "nearest" else H, 176, 3), CANARY_U8, dtype=torch.uint8, device=dev())
        h = dbig.shape[1]
        out = dbig[:, :, dx0:dx0 + w]
        if name == "nearest":
            kr.kr_resize_nearest(src, out)
        else:
            kr.kr_flip_horizontal(src, out)
        torch.cuda.synchronize()
        m = torch.ones(dbig.shape[:3], dtype=torch.bool, device=dev())
        m[:, :, dx0:dx0 + w] = False
        assert bool((dbig[m] == CANARY_U8).all()), "write outside the destination view"
        for i in range(n):
            want = oracle.resize_nearest_u8(imgs[i], h, w) if name == "nearest" else oracle.flip_h_u8(imgs[i])
            np.testing.assert_array_equal(out[i].cpu().numpy(), want)


def test_flip_equals_warp_with_the_mirror_map():
    H, W = 90, 131
    img = inputs.noise_gradient_image(81, H, W)
    M = np.array([[-1, 0, W], [0, 1, 0]], np.float32)
    f = torch.empty((H, W, 3), dtype=torch.uint8, device=dev())
    w = torch.empty_like(f)
    kr.kr_flip_horizontal(to_dev(img), f)
    kr.kr_warp_affine(to_dev(img), w, M)
    torch.cuda.synchronize()
    assert torch.equal(f, w)


# ---------------------------------------------------------------------------
# Perspective warp
# ---------------------------------------------------------------------------
PERSP_CASES = [(1080, 1920, 3, 0.25, 30), (99, 160, 3, 0.8, 31), (71, 90, 1, 0.5, 32), (64, 96, 3, 1.5, 33),
               (257, 129, 3, 2.5, 34)]   # the last ones put a horizon inside the output


@pytest.mark.parametrize("H,W,C,tilt,seed", PERSP_CASES)
def test_warp_perspective_u8(H, W, C, tilt, seed):
    img = inputs.noise_gradient_image(seed, H, W, C)
    M = inputs.random_inverse_homography(np.random.default_rng(seed), H, W, tilt=tilt)
    out = Guarded((H, W, C), torch.uint8)
    kr.kr_warp_perspective(to_dev(img), out.t, M)
    torch.cuda.synchronize()
    out.check()
    np.testing.assert_array_equal(out.np(), oracle.warp_persp_u8(img, M, H, W))


@pytest.mark.parametrize("layout", ["hwc", "chw"])
@pytest.mark.parametrize("H,W,tilt,seed", [(1080, 1920, 0.25, 40), (83, 121, 1.2, 41)])
def test_warp_perspective_f32(H, W, tilt, seed, layout):
    img = inputs.noise_gradient_image(seed, H, W)
    M = inputs.random_inverse_homography(np.random.default_rng(seed), H, W, tilt=tilt)
    shape = (H, W, 3) if layout == "hwc" else (3, H, W)
    out = Guarded(shape, torch.float32)
    kr.kr_warp_perspective(to_dev(img), out.t, M, mean=MEAN, std=STD, dst_layout=layout)
    g = Guarded((H, W, 1), torch.uint8)
    kr.kr_warp_perspective(to_dev(img), g.t, M, gray=True)
    torch.cuda.synchronize()
    out.check()
    g.check()
    got = out.np() if layout == "hwc" else out.np().transpose(1, 2, 0)
    assert np.abs(got - oracle.warp_persp_f64(img, M, H, W, mean=MEAN, std=STD)).max() <= F32_TOL
    np.testing.assert_array_equal(g.np(), oracle.warp_persp_u8(img, M, H, W, gray=True))


def test_perspective_with_affine_last_row_equals_affine_warp():
    n, H, W = 4, 1080, 1920
    imgs = inputs.bench_images(n)
    A = inputs.bench_matrices(n)
    P = np.concatenate([A.reshape(n, 2, 3), np.tile(np.array([[[0, 0, 1]]], np.float32), (n, 1, 1))], axis=1)
    src = to_dev(imgs)
    a = torch.empty((n, H, W, 3), dtype=torch.uint8, device=dev())
    p = torch.empty_like(a)
    kr.kr_warp_affine(src, a, A)
    kr.kr_warp_perspective(src, p, P)
    af = torch.empty((n, H, W, 3), dtype=torch.float32, device=dev())
    pf = torch.empty_like(af)
    kr.kr_warp_affine(src, af, A)
    kr.kr_warp_perspective(src, pf, P)
    torch.cuda.synchronize()
    assert torch.equal(a, p)
    assert torch.equal(af, pf)


def test_perspective_behind_the_camera_is_the_zero_sample():
    H, W = 50, 70
    img = inputs.uniform_image(44, H, W, 3)
    M = -np.eye(3, dtype=np.float32)                   # Z = -1 everywhere
    u = Guarded((H, W, 3), torch.uint8)
    f = Guarded((H, W, 3), torch.float32)
    kr.kr_warp_perspective(to_dev(img), u.t, M)
    kr.kr_warp_perspective(to_dev(img), f.t, M, mean=MEAN, std=STD)
    torch.cuda.synchronize()
    assert not u.np().any()
    np.testing.assert_allclose(f.np(), np.broadcast_to(-np.array(MEAN) / np.array(STD), (H, W, 3)), atol=1e-6)


# ---------------------------------------------------------------------------
# Sobel 3x3
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("H,W,C", [(1080, 1920, 3), (1, 1, 3), (2, 3, 1), (7, 13, 3), (33, 65, 1), (100, 129, 3)])
def test_sobel(H, W, C):
    img = inputs.noise_gradient_image(H + W, H, W, C) if C == 3 else inputs.uniform_image(H + W, H, W, 1)
    f = Guarded((H, W, 1), torch.float32)
    u = Guarded((H, W, 1), torch.uint8)
    kr.kr_sobel(to_dev(img), f.t)
    kr.kr_sobel(to_dev(img), u.t)
    torch.cuda.synchronize()
    f.check()
    u.check()
    rf, ru = oracle.sobel(img)
    np.testing.assert_array_equal(f.np(), rf)          # the same fp32 operations: bit for bit
    np.testing.assert_array_equal(u.np(), ru)


def test_sobel_on_views_and_batches():
    n, H, W = 3, 45, 70
    imgs = np.stack([inputs.noise_gradient_image(90 + i, H, W) for i in range(n)])
    big = torch.full((n, H + 3, W + 4, 3), 250, dtype=torch.uint8, device=dev())
    big[:, 1:1 + H, 2:2 + W] = to_dev(imgs)
    src = big[:, 1:1 + H, 2:2 + W]
    dbig = torch.full((n, H + 2, W + 6, 1), -3.0, dtype=torch.float32, device=dev())
    dst = dbig[:, 1:1 + H, 3:3 + W]
    kr.kr_sobel(src, dst)
    torch.cuda.synchronize()
    m = torch.ones(dbig.shape[:3], dtype=torch.bool, device=dev())
    m[:, 1:1 + H, 3:3 + W] = False
    assert bool((dbig[m] == -3.0).all()), "write outside the destination view"
    for i in range(n):
        np.testing.assert_array_equal(dst[i].cpu().numpy(), oracle.sobel(imgs[i])[0])


# ---------------------------------------------------------------------------
# Replicated border (affine and perspective warps, single images and ragged batches)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("H,W,C,seed", [(1080, 1920, 3, 50), (99, 160, 3, 51), (71, 90, 1, 52)])
def test_warp_replicate_border(H, W, C, seed):
    img = inputs.noise_gradient_image(seed, H, W, C)
    rng = np.random.default_rng(seed)
    A = inputs.random_inverse_affine(rng, H, W, k=1.4)
    P = inputs.random_inverse_homography(rng, H, W, tilt=0.6)
    a = Guarded((H, W, C), torch.uint8)
    p = Guarded((H, W, C), torch.uint8)
    kr.kr_warp_affine(to_dev(img), a.t, A, border="replicate")
    kr.kr_warp_perspective(to_dev(img), p.t, P, border="replicate")
    torch.cuda.synchronize()
    a.check()
    p.check()
    np.testing.assert_array_equal(a.np(), oracle.warp_u8(img, A, H, W, border="replicate"))
    np.testing.assert_array_equal(p.np(), oracle.warp_persp_u8(img, P, H, W, border="replicate"))
    if C == 3:
        f = Guarded((3, H, W), torch.float32)
        kr.kr_warp_affine(to_dev(img), f.t, A, mean=MEAN, std=STD, dst_layout="chw", border="replicate")
        torch.cuda.synchronize()
        f.check()
        ref = oracle.warp_f64(img, A, H, W, mean=MEAN, std=STD, border="replicate")
        assert np.abs(f.np().transpose(1, 2, 0) - ref).max() <= F32_TOL


def test_ragged_batch_with_replicate_border():
    items = []
    rng = np.random.default_rng(53)
    srcs, dsts, work = [], [], []
    for i in range(12):
        H, W = (int(v) for v in rng.integers(20, 300, 2))
        img = inputs.uniform_image(530 + i, H, W, 3)
        M = inputs.random_inverse_affine(rng, H, W, k=1.5)
        s = to_dev(img)
        d = torch.empty((H, W, 3), dtype=torch.uint8, device=dev())
        srcs.append(s)
        dsts.append(d)
        items.append((img, M, H, W))
        work.append(kr.work_item(kr.KR_OP_WARP, s, d, M=M, border="replicate" if i % 2 else "zero"))
    ws = torch.empty(kr.kr_batch_workspace_size(len(work)), dtype=torch.uint8, device=dev())
    kr.kr_batch_submit(kr.work_array(work), ws)
    torch.cuda.synchronize()
    for i, ((img, M, H, W), d) in enumerate(zip(items, dsts)):
        ref = oracle.warp_u8(img, M, H, W, border="replicate" if i % 2 else "zero")
        np.testing.assert_array_equal(d.cpu().numpy(), ref)


# ---------------------------------------------------------------------------
# Area (antialiased) downscale
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("H,W,h,w,C", [(1080, 1920, 720, 1280, 3), (1080, 1920, 540, 960, 3), (37, 53, 11, 17, 3),
                                       (100, 100, 33, 47, 1), (64, 64, 64, 64, 3), (1, 300, 1, 7, 3),
                                       (300, 2, 5, 1, 1), (257, 129, 65, 97, 3),
                                       # strips of fewer than 256 columns (a footprint row of 6667 pixels)
                                       (2, 20000, 2, 3, 3),
                                       # 64-bit sums: 255 W H >= 2^32
                                       (4100, 4100, 3, 5, 1)])
def test_resize_area(H, W, h, w, C):
    img = inputs.uniform_image(H * 3 + W, H, W, C)
    u = Guarded((h, w, C), torch.uint8)
    f = Guarded((h, w, C), torch.float32)
    kr.kr_resize_area(to_dev(img), u.t)
    kr.kr_resize_area(to_dev(img), f.t)
    torch.cuda.synchronize()
    u.check()
    f.check()
    np.testing.assert_array_equal(u.np(), oracle.resize_area_u8(img, h, w))
    assert np.abs(f.np() - oracle.resize_area_f64(img, h, w)).max() <= F32_TOL


def test_resize_area_on_views_and_batches():
    # odd pitch and offset (every staged row has its own 16-byte phase), several strips and bands
    n, H, W, h, w = 3, 91, 700, 40, 300
    imgs = np.stack([inputs.uniform_image(60 + i, H, W, 3) for i in range(n)])
    big = torch.full((n, H + 2, W + 5, 3), 9, dtype=torch.uint8, device=dev())
    big[:, 1:1 + H, 3:3 + W] = to_dev(imgs)
    src = big[:, 1:1 + H, 3:3 + W]
    dbig = torch.full((n, h + 2, w + 3, 3), CANARY_U8, dtype=torch.uint8, device=dev())
    out = dbig[:, 1:1 + h, 2:2 + w]
    kr.kr_resize_area(src, out)
    torch.cuda.synchronize()
    m = torch.ones(dbig.shape[:3], dtype=torch.bool, device=dev())
    m[:, 1:1 + h, 2:2 + w] = False
    assert bool((dbig[m] == CANARY_U8).all()), "write outside the destination view"
    for i in range(n):
        np.testing.assert_array_equal(out[i].cpu().numpy(), oracle.resize_area_u8(imgs[i], h, w))


def test_resize_area_16x4k_to_224_normalised_nchw():
    n, H, W = 16, 2160, 3840
    imgs = np.stack([inputs.uniform_image(700 + i, H, W, 3) for i in range(n)])
    out = Guarded((n, 3, 224, 224), torch.float32)
    kr.kr_resize_area(to_dev(imgs), out.t, mean=MEAN, std=STD, dst_layout="chw")
    u = torch.empty((n, 224, 224, 3), dtype=torch.uint8, device=dev())
    kr.kr_resize_area(to_dev(imgs), u)
    torch.cuda.synchronize()
    out.check()
    for i in (0, 7, 15):
        ref = oracle.resize_area_f64(imgs[i], 224, 224, mean=MEAN, std=STD)
        assert np.abs(out.np()[i].transpose(1, 2, 0) - ref).max() <= F32_TOL
        np.testing.assert_array_equal(u[i].cpu().numpy(), oracle.resize_area_u8(imgs[i], 224, 224))
