/*
 * Reference oracle for the image-resampling path of Kornia-rs (arXiv 2505.12425).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or load
 * this file: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it. It shares no code, header or table with the CUDA library.
 *
 * What it computes (one output pixel at a time, single-threaded, no tables,
 * no tiling):
 *   - bilinear resize of an HWC u8 image (Sec. III of the paper names
 *     "oversizing" and "downsizing"), u8 fixed-point and f64 forms;
 *   - affine warp with a 2x3 inverse map (Sec. II-A: "geometric transforms"
 *     of kornia-imgproc), u8 fixed-point and f64 forms;
 *   - RGB -> gray (Sec. III "RGB to grayscale"; Sec. IV-B gray_from_rgb),
 *     standalone and fused after either resampler;
 *   - u8 -> float normalisation (value/255 - mean)/std, fused;
 *   - nearest-neighbour resize (Sec. IV-A, the Python bindings' "nearest-
 *     neighbor resizing") and horizontal flip (Sec. IV-A, Rust benchmark);
 *   - perspective warp with a 3x3 inverse map (the projective generalisation
 *     of the affine warp; Sec. II-A "geometric transforms"), same taps,
 *     weights and border as the affine warp;
 *   - a replicate-border variant of both warps (taps outside the image read the
 *     nearest edge pixel instead of zero);
 *   - area (antialiased) downscale: each output pixel the exact overlap-
 *     weighted mean of the source pixels its footprint covers;
 *   - Sobel 3x3 gradient magnitude (Sec. V: the robotics example's
 *     imgproc::filter::sobel(&img, &mut out, 3), RGB8 in, Gray8 out).
 *
 * The paper prints none of the arithmetic. The conventions used here are:
 *   half-pixel centres; resize clamps to the edge; warp reads zero outside the
 *   image, tap by tap; 11-bit weights rounded half up; final rounding
 *   (v + 2^21) >> 22; BT.601 gray with 14-bit weights 4899/9617/1868;
 *   the warp coordinate is the fp32 sequence
 *       sx = fmaf(m00, x + 0.5, fmaf(m01, y + 0.5, m02)) - 0.5
 *   with round-to-nearest-even, and a coordinate whose magnitude is not below
 *   2^22 (or NaN) yields a zero sample.
 *
 * Build: gcc -O2 -ffp-contract=off -shared -fPIC (no FMA contraction, so the
 * fp32 sequence is the same on x86-64 and aarch64).
 *
 * The f32 forms interpolate in double and return double; the u8 forms are
 * pure integer arithmetic apart from the warp coordinate, which is fp32 by
 * definition.
 *
 * Optional "touched" bitmaps (H*W bytes, may be NULL) mark every source pixel
 * that some output sample reads with a nonzero weight; the benchmark's
 * algorithmic byte count is derived from them.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

#define ORACLE_OK 0
#define ORACLE_BAD 1

/* ------------------------------------------------------------------------ */
/* Resize coordinate along one axis (half-pixel centres, clamp to edge).     */
/*   sx = (i + 1/2) * n_in / n_out - 1/2 = num / den, exactly, with          */
/*   num = (2i + 1) * n_in - n_out and den = 2 * n_out.                      */
/* Outputs: i0, i1 = the two taps; q = 11-bit weight of i1 (round half up   */
/* of 2048 * frac); frac = exact fraction as a double (f32 form).            */
/* ------------------------------------------------------------------------ */
static void resize_axis(long i, long n_in, long n_out,
                        long *i0, long *i1, long *q, double *frac)
{
    long long num = (2LL * i + 1LL) * (long long)n_in - (long long)n_out;
    long long den = 2LL * (long long)n_out;
    if (num <= 0) {                 /* sx <= 0: clamp to the first sample  */
        *i0 = 0;
        *q = 0;
        *frac = 0.0;
    } else {
        long long k = num / den;
        long long r = num % den;
        if (k >= n_in - 1) {        /* sx >= n_in - 1: clamp to the last   */
            *i0 = n_in - 1;
            *q = 0;
            *frac = 0.0;
        } else {
            *i0 = (long)k;
            /* round half up of 2048 * r / den */
            *q = (long)((4096LL * r + den) / (2LL * den));
            *frac = (double)r / (double)den;
        }
    }
    *i1 = (*i0 + 1 < n_in) ? *i0 + 1 : n_in - 1;
}

/* 4-tap blend of u8 samples with 11-bit weights, rounded half up. */
static long blend_u8(long p00, long p01, long p10, long p11, long qx, long qy)
{
    long top = p00 * (2048 - qx) + p01 * qx;
    long bot = p10 * (2048 - qx) + p11 * qx;
    long v = top * (2048 - qy) + bot * qy;
    return (v + (1L << 21)) >> 22;
}

/* BT.601 luma with 14-bit integer weights (they sum to 16384). */
static long gray_u8(long r, long g, long b)
{
    return (4899 * r + 9617 * g + 1868 * b + 8192) >> 14;
}

static double gray_f64(double r, double g, double b)
{
    return 0.299 * r + 0.587 * g + 0.114 * b;
}

static void mark(uint8_t *touched, long W, long y, long x)
{
    if (touched) touched[y * W + x] = 1;
}

/* ======================================================================== */
/* Bilinear resize, u8 out.                                                 */
/* src: H x W x C contiguous (C = 1 or 3). dst: h x w x dC contiguous,      */
/* dC = C, or dC = 1 with gray = 1 (C must be 3): gray of the rounded RGB.  */
/* ======================================================================== */
int oracle_resize_u8(const uint8_t *src, long H, long W, long C,
                     uint8_t *dst, long h, long w, int gray, uint8_t *touched)
{
    if (H < 1 || W < 1 || h < 1 || w < 1 || (C != 1 && C != 3)) return ORACLE_BAD;
    if (gray && C != 3) return ORACLE_BAD;
    long dC = gray ? 1 : C;
    for (long y = 0; y < h; ++y) {
        long y0, y1, qy;
        double fy;
        resize_axis(y, H, h, &y0, &y1, &qy, &fy);
        for (long x = 0; x < w; ++x) {
            long x0, x1, qx;
            double fx;
            resize_axis(x, W, w, &x0, &x1, &qx, &fx);
            long out[3];
            for (long c = 0; c < C; ++c) {
                long p00 = src[(y0 * W + x0) * C + c];
                long p01 = src[(y0 * W + x1) * C + c];
                long p10 = src[(y1 * W + x0) * C + c];
                long p11 = src[(y1 * W + x1) * C + c];
                out[c] = blend_u8(p00, p01, p10, p11, qx, qy);
            }
            if (qx < 2048 && qy < 2048) mark(touched, W, y0, x0);
            if (qx > 0 && qy < 2048) mark(touched, W, y0, x1);
            if (qx < 2048 && qy > 0) mark(touched, W, y1, x0);
            if (qx > 0 && qy > 0) mark(touched, W, y1, x1);
            if (gray) {
                dst[y * w + x] = (uint8_t)gray_u8(out[0], out[1], out[2]);
            } else {
                for (long c = 0; c < C; ++c) dst[(y * w + x) * dC + c] = (uint8_t)out[c];
            }
        }
    }
    return ORACLE_OK;
}

/* ======================================================================== */
/* Bilinear resize, f32 form (computed in double).                          */
/* Samples are p/255; out = (v - mean[c]) / std[c]. gray = 1: one channel   */
/* 0.299R + 0.587G + 0.114B of the interpolants, normalised with mean[0],   */
/* std[0]. dst: h x w x dC doubles, HWC.                                    */
/* ======================================================================== */
int oracle_resize_f64(const uint8_t *src, long H, long W, long C,
                      double *dst, long h, long w, int gray,
                      const double *mean, const double *stdv, uint8_t *touched)
{
    if (H < 1 || W < 1 || h < 1 || w < 1 || (C != 1 && C != 3)) return ORACLE_BAD;
    if (gray && C != 3) return ORACLE_BAD;
    long dC = gray ? 1 : C;
    for (long y = 0; y < h; ++y) {
        long y0, y1, qy;
        double fy;
        resize_axis(y, H, h, &y0, &y1, &qy, &fy);
        for (long x = 0; x < w; ++x) {
            long x0, x1, qx;
            double fx;
            resize_axis(x, W, w, &x0, &x1, &qx, &fx);
            double v[3];
            for (long c = 0; c < C; ++c) {
                double a = src[(y0 * W + x0) * C + c] / 255.0;
                double b = src[(y0 * W + x1) * C + c] / 255.0;
                double d0 = src[(y1 * W + x0) * C + c] / 255.0;
                double d1 = src[(y1 * W + x1) * C + c] / 255.0;
                v[c] = (1.0 - fy) * ((1.0 - fx) * a + fx * b)
                     + fy * ((1.0 - fx) * d0 + fx * d1);
            }
            if (fx < 1.0 && fy < 1.0) mark(touched, W, y0, x0);
            if (fx > 0.0 && fy < 1.0) mark(touched, W, y0, x1);
            if (fx < 1.0 && fy > 0.0) mark(touched, W, y1, x0);
            if (fx > 0.0 && fy > 0.0) mark(touched, W, y1, x1);
            if (gray) {
                dst[y * w + x] = (gray_f64(v[0], v[1], v[2]) - mean[0]) / stdv[0];
            } else {
                for (long c = 0; c < C; ++c)
                    dst[(y * w + x) * dC + c] = (v[c] - mean[c]) / stdv[c];
            }
        }
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Warp coordinate: M maps destination -> source (inverse map).             */
/* Returns 0 when the sample lies beyond |s| < 2^22 (or is NaN).            */
/* ------------------------------------------------------------------------ */
static int warp_coord(const float *M, long x, long y, float *sx, float *sy)
{
    float xc = (float)x + 0.5f;
    float yc = (float)y + 0.5f;
    *sx = fmaf(M[0], xc, fmaf(M[1], yc, M[2])) - 0.5f;
    *sy = fmaf(M[3], xc, fmaf(M[4], yc, M[5])) - 0.5f;
    return (fabsf(*sx) < 4194304.0f) && (fabsf(*sy) < 4194304.0f);
}

/* Perspective coordinate: M (3x3, row-major) maps destination -> source in */
/* homogeneous coordinates. fp32, round to nearest, exactly as written:      */
/*   X, Y, Z = fmaf(m_r0, xc, fmaf(m_r1, yc, m_r2)) for rows r = 0, 1, 2;    */
/*   q = 1 / Z; sx = X * q - 0.5; sy = Y * q - 0.5.                          */
/* A point with Z <= 0 (or NaN) has no source: zero sample, as is a sample  */
/* beyond |s| < 2^22. With the last row (0, 0, 1), q = 1 and X * q = X, so  */
/* the affine warp is the special case bit for bit.                         */
static int persp_coord(const float *M, long x, long y, float *sx, float *sy)
{
    float xc = (float)x + 0.5f;
    float yc = (float)y + 0.5f;
    float X = fmaf(M[0], xc, fmaf(M[1], yc, M[2]));
    float Y = fmaf(M[3], xc, fmaf(M[4], yc, M[5]));
    float Z = fmaf(M[6], xc, fmaf(M[7], yc, M[8]));
    if (!(Z > 0.0f)) return 0;
    float q = 1.0f / Z;
    *sx = X * q - 0.5f;
    *sy = Y * q - 0.5f;
    return (fabsf(*sx) < 4194304.0f) && (fabsf(*sy) < 4194304.0f);
}

static int coord_of(const float *M, int persp, long x, long y, float *sx, float *sy)
{
    return persp ? persp_coord(M, x, y, sx, sy) : warp_coord(M, x, y, sx, sy);
}

/* 11-bit weight of a coordinate: floor and round-half-up of 2048 * frac,   */
/* all in fp32 exactly as written.                                          */
static void warp_weight(float s, long *i0, long *q)
{
    long k0 = (long)floorf(s);
    float f = s - (float)k0;
    float t = f * 2048.0f;
    long k = (long)floorf(t);
    *i0 = k0;
    *q = k + ((t - (float)k) >= 0.5f ? 1 : 0);
}

/* Border modes of the warps: zero outside the image, or the nearest edge pixel. */
#define BORDER_ZERO 0
#define BORDER_REPLICATE 1

static long clamp_index(long v, long n) { return v < 0 ? 0 : (v >= n ? n - 1 : v); }

static long tap_u8(const uint8_t *src, long H, long W, long C, long y, long x, long c, int border)
{
    if (border == BORDER_REPLICATE) {
        x = clamp_index(x, W);
        y = clamp_index(y, H);
    }
    if (x < 0 || x >= W || y < 0 || y >= H) return 0;
    return src[(y * W + x) * C + c];
}

static void mark_in(uint8_t *touched, long H, long W, long y, long x, int border)
{
    if (border == BORDER_REPLICATE) {
        x = clamp_index(x, W);
        y = clamp_index(y, H);
    }
    if (x >= 0 && x < W && y >= 0 && y < H) mark(touched, W, y, x);
}

/* ======================================================================== */
/* Affine (persp = 0; M: 6 floats, row-major 2x3) or perspective (persp = 1; */
/* M: 9 floats, row-major 3x3) warp, u8 out (zero border per tap).          */
/* ======================================================================== */
static int warp_u8_impl(const uint8_t *src, long H, long W, long C, const float *M, int persp, int border,
                        uint8_t *dst, long h, long w, int gray, uint8_t *touched)
{
    if (H < 1 || W < 1 || h < 1 || w < 1 || (C != 1 && C != 3)) return ORACLE_BAD;
    if (gray && C != 3) return ORACLE_BAD;
    long dC = gray ? 1 : C;
    for (long y = 0; y < h; ++y) {
        for (long x = 0; x < w; ++x) {
            float sx, sy;
            long out[3] = {0, 0, 0};
            if (coord_of(M, persp, x, y, &sx, &sy)) {
                long x0, qx, y0, qy;
                warp_weight(sx, &x0, &qx);
                warp_weight(sy, &y0, &qy);
                for (long c = 0; c < C; ++c) {
                    long p00 = tap_u8(src, H, W, C, y0, x0, c, border);
                    long p01 = tap_u8(src, H, W, C, y0, x0 + 1, c, border);
                    long p10 = tap_u8(src, H, W, C, y0 + 1, x0, c, border);
                    long p11 = tap_u8(src, H, W, C, y0 + 1, x0 + 1, c, border);
                    out[c] = blend_u8(p00, p01, p10, p11, qx, qy);
                }
                if (qx < 2048 && qy < 2048) mark_in(touched, H, W, y0, x0, border);
                if (qx > 0 && qy < 2048) mark_in(touched, H, W, y0, x0 + 1, border);
                if (qx < 2048 && qy > 0) mark_in(touched, H, W, y0 + 1, x0, border);
                if (qx > 0 && qy > 0) mark_in(touched, H, W, y0 + 1, x0 + 1, border);
            }
            if (gray) {
                dst[y * w + x] = (uint8_t)gray_u8(out[0], out[1], out[2]);
            } else {
                for (long c = 0; c < C; ++c) dst[(y * w + x) * dC + c] = (uint8_t)out[c];
            }
        }
    }
    return ORACLE_OK;
}

int oracle_warp_u8(const uint8_t *src, long H, long W, long C, const float *M,
                   uint8_t *dst, long h, long w, int gray, uint8_t *touched)
{
    return warp_u8_impl(src, H, W, C, M, 0, BORDER_ZERO, dst, h, w, gray, touched);
}

int oracle_warp_persp_u8(const uint8_t *src, long H, long W, long C, const float *M,
                         uint8_t *dst, long h, long w, int gray, uint8_t *touched)
{
    return warp_u8_impl(src, H, W, C, M, 1, BORDER_ZERO, dst, h, w, gray, touched);
}

static double tap_f64(const uint8_t *src, long H, long W, long C, long y, long x, long c, int border)
{
    if (border == BORDER_REPLICATE) {
        x = clamp_index(x, W);
        y = clamp_index(y, H);
    }
    if (x < 0 || x >= W || y < 0 || y >= H) return 0.0;
    return src[(y * W + x) * C + c] / 255.0;
}

/* ======================================================================== */
/* Affine or perspective warp, f32 form in double. The coordinate is the    */
/* fp32 value from warp_coord / persp_coord; the fraction s - floor(s) is    */
/* taken exactly in double and not quantised.                               */
/* ======================================================================== */
static int warp_f64_impl(const uint8_t *src, long H, long W, long C, const float *M, int persp, int border,
                         double *dst, long h, long w, int gray,
                         const double *mean, const double *stdv, uint8_t *touched)
{
    if (H < 1 || W < 1 || h < 1 || w < 1 || (C != 1 && C != 3)) return ORACLE_BAD;
    if (gray && C != 3) return ORACLE_BAD;
    long dC = gray ? 1 : C;
    for (long y = 0; y < h; ++y) {
        for (long x = 0; x < w; ++x) {
            float sx, sy;
            double v[3] = {0.0, 0.0, 0.0};
            if (coord_of(M, persp, x, y, &sx, &sy)) {
                double dsx = (double)sx, dsy = (double)sy;
                double fx0 = floor(dsx), fy0 = floor(dsy);
                double fx = dsx - fx0, fy = dsy - fy0;
                long x0 = (long)fx0, y0 = (long)fy0;
                for (long c = 0; c < C; ++c) {
                    double a = tap_f64(src, H, W, C, y0, x0, c, border);
                    double b = tap_f64(src, H, W, C, y0, x0 + 1, c, border);
                    double d0 = tap_f64(src, H, W, C, y0 + 1, x0, c, border);
                    double d1 = tap_f64(src, H, W, C, y0 + 1, x0 + 1, c, border);
                    v[c] = (1.0 - fy) * ((1.0 - fx) * a + fx * b)
                         + fy * ((1.0 - fx) * d0 + fx * d1);
                }
                if (fx < 1.0 && fy < 1.0) mark_in(touched, H, W, y0, x0, border);
                if (fx > 0.0 && fy < 1.0) mark_in(touched, H, W, y0, x0 + 1, border);
                if (fx < 1.0 && fy > 0.0) mark_in(touched, H, W, y0 + 1, x0, border);
                if (fx > 0.0 && fy > 0.0) mark_in(touched, H, W, y0 + 1, x0 + 1, border);
            }
            if (gray) {
                dst[y * w + x] = (gray_f64(v[0], v[1], v[2]) - mean[0]) / stdv[0];
            } else {
                for (long c = 0; c < C; ++c)
                    dst[(y * w + x) * dC + c] = (v[c] - mean[c]) / stdv[c];
            }
        }
    }
    return ORACLE_OK;
}

int oracle_warp_f64(const uint8_t *src, long H, long W, long C, const float *M,
                    double *dst, long h, long w, int gray,
                    const double *mean, const double *stdv, uint8_t *touched)
{
    return warp_f64_impl(src, H, W, C, M, 0, BORDER_ZERO, dst, h, w, gray, mean, stdv, touched);
}

int oracle_warp_persp_f64(const uint8_t *src, long H, long W, long C, const float *M,
                          double *dst, long h, long w, int gray,
                          const double *mean, const double *stdv, uint8_t *touched)
{
    return warp_f64_impl(src, H, W, C, M, 1, BORDER_ZERO, dst, h, w, gray, mean, stdv, touched);
}

/* Either warp (persp = 0: M 2x3, 1: M 3x3) with either border (0 zero, 1 replicate). */
int oracle_warp_ex_u8(const uint8_t *src, long H, long W, long C, const float *M, int persp, int border,
                      uint8_t *dst, long h, long w, int gray, uint8_t *touched)
{
    if (border != BORDER_ZERO && border != BORDER_REPLICATE) return ORACLE_BAD;
    return warp_u8_impl(src, H, W, C, M, persp != 0, border, dst, h, w, gray, touched);
}

int oracle_warp_ex_f64(const uint8_t *src, long H, long W, long C, const float *M, int persp, int border,
                       double *dst, long h, long w, int gray,
                       const double *mean, const double *stdv, uint8_t *touched)
{
    if (border != BORDER_ZERO && border != BORDER_REPLICATE) return ORACLE_BAD;
    return warp_f64_impl(src, H, W, C, M, persp != 0, border, dst, h, w, gray, mean, stdv, touched);
}

/* ======================================================================== */
/* Standalone RGB -> gray, u8 (Sec. IV-B gray_from_rgb: Image<u8,3> in,     */
/* Image<u8,1> out of the same size).                                       */
/* ======================================================================== */
int oracle_rgb_to_gray_u8(const uint8_t *src, long H, long W, uint8_t *dst)
{
    if (H < 1 || W < 1) return ORACLE_BAD;
    for (long y = 0; y < H; ++y)
        for (long x = 0; x < W; ++x) {
            const uint8_t *p = src + (y * W + x) * 3;
            dst[y * W + x] = (uint8_t)gray_u8(p[0], p[1], p[2]);
        }
    return ORACLE_OK;
}

/* The warp coordinate and weights of one output pixel, exposed so the     */
/* tests can pin the fp32 sequence against an exact-rational computation.  */
int oracle_warp_point(const float *M, long x, long y, float *sx, float *sy,
                      long *x0, long *qx, long *y0, long *qy)
{
    int ok = warp_coord(M, x, y, sx, sy);
    if (ok) {
        warp_weight(*sx, x0, qx);
        warp_weight(*sy, y0, qy);
    }
    return ok;
}

/* The same for the perspective coordinate. */
int oracle_persp_point(const float *M, long x, long y, float *sx, float *sy,
                       long *x0, long *qx, long *y0, long *qy)
{
    int ok = persp_coord(M, x, y, sx, sy);
    if (ok) {
        warp_weight(*sx, x0, qx);
        warp_weight(*sy, y0, qy);
    }
    return ok;
}

/* The resize taps and weights along one axis, exposed for the same reason. */
int oracle_resize_point(long i, long n_in, long n_out, long *i0, long *i1,
                        long *q, double *frac)
{
    if (n_in < 1 || n_out < 1 || i < 0 || i >= n_out) return ORACLE_BAD;
    resize_axis(i, n_in, n_out, i0, i1, q, frac);
    return ORACLE_OK;
}

/* ======================================================================== */
/* Nearest-neighbour resize, u8, C = 1 or 3 (Sec. IV-A names the operation, */
/* not its convention). With half-pixel centres the output pixel (x, y) has */
/* its centre at source position ((x + 1/2) W / w, (y + 1/2) H / h) in      */
/* continuous coordinates where source pixel i covers [i, i + 1); it copies */
/* the source pixel covering that point:                                    */
/*     sx = floor((x + 1/2) W / w) = ((2x + 1) W) div (2w),  likewise sy,   */
/* exact integer arithmetic, never outside [0, W - 1] x [0, H - 1].         */
/* ======================================================================== */
int oracle_resize_nearest_u8(const uint8_t *src, long H, long W, long C, uint8_t *dst, long h, long w)
{
    if (H < 1 || W < 1 || h < 1 || w < 1 || (C != 1 && C != 3)) return ORACLE_BAD;
    for (long y = 0; y < h; ++y) {
        const long sy = (long)(((2LL * y + 1LL) * (long long)H) / (2LL * (long long)h));
        for (long x = 0; x < w; ++x) {
            const long sx = (long)(((2LL * x + 1LL) * (long long)W) / (2LL * (long long)w));
            for (long c = 0; c < C; ++c)
                dst[(y * w + x) * C + c] = src[(sy * W + sx) * C + c];
        }
    }
    return ORACLE_OK;
}

/* ======================================================================== */
/* Horizontal flip, u8, C = 1 or 3 (Sec. IV-A): out(y, x) = in(y, W - 1 - x) */
/* ======================================================================== */
int oracle_flip_h_u8(const uint8_t *src, long H, long W, long C, uint8_t *dst)
{
    if (H < 1 || W < 1 || (C != 1 && C != 3)) return ORACLE_BAD;
    for (long y = 0; y < H; ++y)
        for (long x = 0; x < W; ++x)
            for (long c = 0; c < C; ++c)
                dst[(y * W + x) * C + c] = src[(y * W + (W - 1 - x)) * C + c];
    return ORACLE_OK;
}

/* ======================================================================== */
/* Sobel 3x3 gradient magnitude (Sec. V example: kernel size 3, an RGB8     */
/* image in and a Gray8 image out; the paper gives no formula). Readings:   */
/* a 3-channel source is first the u8 BT.601 gray above; the border         */
/* replicates the edge pixel; with                                          */
/*   gx = sum_{dy,dx} (dx (2 - |dy|)) I(y + dy, x + dx),                    */
/*   gy = sum_{dy,dx} (dy (2 - |dx|)) I(y + dy, x + dx),                    */
/* (the Sobel kernels [-1 0 1; -2 0 2; -1 0 1] and their transpose, both    */
/* integers) the f32 output is the magnitude of the normalised kernels      */
/*   m = sqrtf((float)(gx*gx + gy*gy)) / 8     (exact up to the one sqrt     */
/*                                              rounding: gx^2 + gy^2 < 2^24) */
/* and the u8 output is floorf(m + 0.5f) (at most 181).                     */
/* Either output pointer may be NULL.                                       */
/* ======================================================================== */
static long clampl(long v, long lo, long hi) { return v < lo ? lo : (v > hi ? hi : v); }

int oracle_sobel(const uint8_t *src, long H, long W, long C, float *out_f32, uint8_t *out_u8)
{
    if (H < 1 || W < 1 || (C != 1 && C != 3)) return ORACLE_BAD;
    for (long y = 0; y < H; ++y) {
        for (long x = 0; x < W; ++x) {
            long gx = 0, gy = 0;
            for (long dy = -1; dy <= 1; ++dy) {
                for (long dx = -1; dx <= 1; ++dx) {
                    const long yy = clampl(y + dy, 0, H - 1), xx = clampl(x + dx, 0, W - 1);
                    const uint8_t *p = src + (yy * W + xx) * C;
                    const long v = C == 3 ? gray_u8(p[0], p[1], p[2]) : p[0];
                    gx += dx * (2 - (dy < 0 ? -dy : dy)) * v;
                    gy += dy * (2 - (dx < 0 ? -dx : dx)) * v;
                }
            }
            const float m = sqrtf((float)(gx * gx + gy * gy)) / 8.0f;
            if (out_f32) out_f32[y * W + x] = m;
            if (out_u8) out_u8[y * W + x] = (uint8_t)floorf(m + 0.5f);
        }
    }
    return ORACLE_OK;
}

/* ======================================================================== */
/* Area (antialiased) downscale, u8 source, C = 1 or 3, w <= W, h <= H.      */
/* Output pixel (x, y) covers the source rectangle [x W/w, (x+1) W/w) x      */
/* [y H/h, (y+1) H/h) (source pixel i covers [i, i+1)); its value is the    */
/* mean of the source over it, each pixel weighted by its overlap area.    */
/* In units of 1/w (1/h) of a pixel the overlaps are integers:              */
/*   ax(i) = max(0, min((x+1) W, (i+1) w) - max(x W, i w)),  sum_i ax = W,  */
/* likewise ay(j) (sum = H), and                                            */
/*   S = sum_j ay(j) sum_i ax(i) p(j, i)        (exact, 64-bit)             */
/*   u8  = floor((2 S + W H) / (2 W H))         (mean rounded half up)      */
/*   f64 = (S / (W H) / 255 - mean) / std.                                  */
/* ======================================================================== */
static long long area_sum(const uint8_t *src, long H, long W, long C, long h, long w, long x, long y, long c)
{
    const long long xa = (long long)x * W, xb = (long long)(x + 1) * W;
    const long long ya = (long long)y * H, yb = (long long)(y + 1) * H;
    long long S = 0;
    for (long j = (long)(ya / h); j < H && (long long)j * h < yb; ++j) {
        long long ay = (yb < (long long)(j + 1) * h ? yb : (long long)(j + 1) * h) -
                       (ya > (long long)j * h ? ya : (long long)j * h);
        if (ay <= 0) continue;
        long long row = 0;
        for (long i = (long)(xa / w); i < W && (long long)i * w < xb; ++i) {
            long long ax = (xb < (long long)(i + 1) * w ? xb : (long long)(i + 1) * w) -
                           (xa > (long long)i * w ? xa : (long long)i * w);
            if (ax > 0) row += ax * src[(j * W + i) * C + c];
        }
        S += ay * row;
    }
    return S;
}

int oracle_resize_area_u8(const uint8_t *src, long H, long W, long C, uint8_t *dst, long h, long w)
{
    if (H < 1 || W < 1 || h < 1 || w < 1 || h > H || w > W || (C != 1 && C != 3)) return ORACLE_BAD;
    const long long WH = (long long)W * H;
    for (long y = 0; y < h; ++y)
        for (long x = 0; x < w; ++x)
            for (long c = 0; c < C; ++c) {
                const long long S = area_sum(src, H, W, C, h, w, x, y, c);
                dst[(y * w + x) * C + c] = (uint8_t)((2 * S + WH) / (2 * WH));
            }
    return ORACLE_OK;
}

int oracle_resize_area_f64(const uint8_t *src, long H, long W, long C, double *dst, long h, long w,
                           const double *mean, const double *stdv)
{
    if (H < 1 || W < 1 || h < 1 || w < 1 || h > H || w > W || (C != 1 && C != 3)) return ORACLE_BAD;
    const double WH = (double)W * (double)H;
    for (long y = 0; y < h; ++y)
        for (long x = 0; x < w; ++x)
            for (long c = 0; c < C; ++c) {
                const long long S = area_sum(src, H, W, C, h, w, x, y, c);
                dst[(y * w + x) * C + c] = ((double)S / WH / 255.0 - mean[c]) / stdv[c];
            }
    return ORACLE_OK;
}
