// extern "C" entry points of the single-image operators: argument validation
// (everything is checked on the host before anything is enqueued), mapping of
// the public descriptors to the internal launch descriptors, status text.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "kr_device.cuh"
#include "kr_internal.h"

namespace kr {

static thread_local char g_last_error[256];

void set_last_error(const char *what, cudaError_t e)
{
    std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s)", what, cudaGetErrorName(e),
                  cudaGetErrorString(e));
}

// Largest accepted image side.
constexpr int kMaxSide = 65535;

static int esize_of(int dtype) { return dtype == KR_F32 ? 4 : 1; }

// Bytes from `data` to one past the last byte of one image.
static int64_t image_extent(const kr_image_t &im)
{
    const int es = esize_of(im.dtype);
    if (im.layout == KR_CHW)
        return (int64_t)(im.channels - 1) * im.plane_stride + (int64_t)(im.height - 1) * im.pitch +
               (int64_t)im.width * es;
    return (int64_t)(im.height - 1) * im.pitch + (int64_t)im.width * im.channels * es;
}

// [lo, hi) of all bytes an image (batch) may touch.
static void image_range(const kr_image_t &im, uintptr_t &lo, uintptr_t &hi)
{
    lo = (uintptr_t)im.data;
    hi = lo + (uintptr_t)image_extent(im) + (uintptr_t)(im.batch - 1) * (uintptr_t)im.batch_stride;
}

// Structural checks shared by sources and destinations.
static kr_status check_image(const kr_image_t *im, bool is_dst)
{
    if (!im || !im->data) return KR_ERR_INVALID_ARG;
    if (im->height < 1 || im->width < 1 || im->height > kMaxSide || im->width > kMaxSide)
        return KR_ERR_INVALID_ARG;
    if (im->channels != 1 && im->channels != 3) return KR_ERR_INVALID_ARG;
    if (im->dtype != KR_U8 && im->dtype != KR_F32) return KR_ERR_INVALID_ARG;
    if (im->layout != KR_HWC && im->layout != KR_CHW) return KR_ERR_INVALID_ARG;
    if (im->batch < 1 || im->batch > kMaxSide) return KR_ERR_INVALID_ARG;   // batches index the grid's z
    const int es = esize_of(im->dtype);
    if (im->dtype == KR_F32) {
        if (((uintptr_t)im->data | (uintptr_t)im->pitch) & 3) return KR_ERR_INVALID_ARG;
        if (im->layout == KR_CHW && (im->plane_stride & 3)) return KR_ERR_INVALID_ARG;
        if (im->batch > 1 && (im->batch_stride & 3)) return KR_ERR_INVALID_ARG;
    }
    if (im->layout == KR_CHW) {
        if (im->dtype != KR_F32 || !is_dst) return KR_ERR_UNSUPPORTED;
        if (im->pitch < (int64_t)im->width * 4) return KR_ERR_INVALID_ARG;
        if (im->channels > 1 && im->plane_stride < (int64_t)(im->height - 1) * im->pitch + im->width * 4)
            return KR_ERR_INVALID_ARG;
    } else {
        if (im->pitch < (int64_t)im->width * im->channels * es) return KR_ERR_INVALID_ARG;
    }
    if (im->batch > 1) {
        if (im->batch_stride < 0) return KR_ERR_INVALID_ARG;
        // destinations may not overlap between images; sources may (e.g. stride 0)
        if (is_dst && im->batch_stride < image_extent(*im)) return KR_ERR_INVALID_ARG;
    }
    return KR_OK;
}

static kr_status check_alias(const kr_image_t &a, const kr_image_t &b)
{
    uintptr_t alo, ahi, blo, bhi;
    image_range(a, alo, ahi);
    image_range(b, blo, bhi);
    return (alo < bhi && blo < ahi) ? KR_ERR_ALIAS : KR_OK;
}

// Validate the common part of resize/warp and fill the internal descriptor.
kr_status build_resample(int op, const kr_image_t *src, const kr_image_t *dst, const kr_post_t *post,
                         OpDesc &d)
{
    kr_status st;
    if ((st = check_image(src, false)) != KR_OK) return st;
    if ((st = check_image(dst, true)) != KR_OK) return st;
    if (src->dtype != KR_U8) return KR_ERR_UNSUPPORTED;
    if (src->batch != dst->batch) return KR_ERR_INVALID_ARG;
    const uint32_t flags = post ? post->flags : 0u;
    if (flags & ~(KR_GRAY | KR_NORMALIZE | KR_BORDER_REPLICATE)) return KR_ERR_INVALID_ARG;
    if ((flags & KR_BORDER_REPLICATE) && op == OP_RESIZE) return KR_ERR_INVALID_ARG;
    const bool gray = flags & KR_GRAY, norm = flags & KR_NORMALIZE;
    if (gray) {
        if (src->channels != 3 || dst->channels != 1) return KR_ERR_INVALID_ARG;
    } else if (dst->channels != src->channels) {
        return KR_ERR_INVALID_ARG;
    }
    if (norm && dst->dtype != KR_F32) return KR_ERR_INVALID_ARG;
    if (dst->dtype == KR_U8 && dst->layout != KR_HWC) return KR_ERR_INVALID_ARG;
    if ((st = check_alias(*src, *dst)) != KR_OK) return st;

    std::memset(&d, 0, sizeof(d));
    d.op = op;
    d.cin = src->channels;
    d.outk = dst->dtype == KR_U8 ? (gray ? OUT_U8_GRAY : OUT_U8) : (gray ? OUT_F32_GRAY : OUT_F32);
    d.src = (const uint8_t *)src->data;
    d.spitch = src->pitch;
    d.sbatch = src->batch > 1 ? src->batch_stride : 0;
    d.H = src->height;
    d.W = src->width;
    d.dst = (uint8_t *)dst->data;
    d.dpitch = dst->pitch;
    d.dplane = dst->layout == KR_CHW ? dst->plane_stride : 0;
    d.dbatch = dst->batch > 1 ? dst->batch_stride : 0;
    d.h = dst->height;
    d.w = dst->width;
    d.chw = dst->layout == KR_CHW && dst->channels == 3;
    d.replicate = (flags & KR_BORDER_REPLICATE) ? 1 : 0;
    d.batch = src->batch;
    for (int c = 0; c < 3; ++c) {
        double mean = 0.0, stdv = 1.0;
        if (norm) {
            mean = post->mean[c];
            stdv = post->std[c];
            if (!std::isfinite(mean) || !std::isfinite(stdv) || stdv == 0.0) return KR_ERR_INVALID_ARG;
        }
        d.scale[c] = (float)(1.0 / (255.0 * stdv));
        d.bias[c] = (float)(-mean / stdv);
    }
    return KR_OK;
}

kr_status build_gray(const kr_image_t *src, const kr_image_t *dst, GrayDesc &d)
{
    kr_status st;
    if ((st = check_image(src, false)) != KR_OK) return st;
    if ((st = check_image(dst, true)) != KR_OK) return st;
    if (src->dtype != KR_U8 || dst->dtype != KR_U8 || dst->layout != KR_HWC) return KR_ERR_UNSUPPORTED;
    if (src->channels != 3 || dst->channels != 1) return KR_ERR_INVALID_ARG;
    if (src->height != dst->height || src->width != dst->width || src->batch != dst->batch)
        return KR_ERR_INVALID_ARG;
    if ((st = check_alias(*src, *dst)) != KR_OK) return st;
    d.src = (const uint8_t *)src->data;
    d.spitch = src->pitch;
    d.sbatch = src->batch > 1 ? src->batch_stride : 0;
    d.dst = (uint8_t *)dst->data;
    d.dpitch = dst->pitch;
    d.dbatch = dst->batch > 1 ? dst->batch_stride : 0;
    d.H = src->height;
    d.W = src->width;
    d.batch = src->batch;
    return KR_OK;
}

// Validate a pixel gather (u8 HWC in and out, same channels and batch; the flip keeps
// the size) and fill its descriptor.
static kr_status build_gather(const kr_image_t *src, const kr_image_t *dst, bool same_size, GatherDesc &d)
{
    kr_status st;
    if ((st = check_image(src, false)) != KR_OK) return st;
    if ((st = check_image(dst, true)) != KR_OK) return st;
    if (src->dtype != KR_U8 || dst->dtype != KR_U8 || src->layout != KR_HWC || dst->layout != KR_HWC)
        return KR_ERR_UNSUPPORTED;
    if (src->channels != dst->channels || src->batch != dst->batch) return KR_ERR_INVALID_ARG;
    if (same_size && (src->height != dst->height || src->width != dst->width)) return KR_ERR_INVALID_ARG;
    if ((st = check_alias(*src, *dst)) != KR_OK) return st;
    d.src = (const uint8_t *)src->data;
    d.spitch = src->pitch;
    d.sbatch = src->batch > 1 ? src->batch_stride : 0;
    d.H = src->height;
    d.W = src->width;
    d.dst = (uint8_t *)dst->data;
    d.dpitch = dst->pitch;
    d.dbatch = dst->batch > 1 ? dst->batch_stride : 0;
    d.h = dst->height;
    d.w = dst->width;
    d.C = src->channels;
    d.batch = src->batch;
    return KR_OK;
}

}  // namespace kr

using namespace kr;

extern "C" {

kr_status kr_resize_nearest(const kr_image_t *src, const kr_image_t *dst, kr_stream_t stream)
{
    GatherDesc d;
    kr_status st = build_gather(src, dst, false, d);
    if (st != KR_OK) return st;
    cudaError_t e = launch_resize_nearest(d, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_last_error("kr_resize_nearest", e);
        return KR_ERR_CUDA;
    }
    return KR_OK;
}

kr_status kr_resize_area(const kr_image_t *src, const kr_image_t *dst, const kr_post_t *post, kr_stream_t stream)
{
    OpDesc o;
    kr_status st = build_resample(OP_RESIZE, src, dst, post, o);
    if (st != KR_OK) return st;
    if (o.outk == OUT_U8_GRAY || o.outk == OUT_F32_GRAY) return KR_ERR_UNSUPPORTED;
    if (o.h > o.H || o.w > o.W) return KR_ERR_INVALID_ARG;   // a downscale (or the same size)
    AreaDesc d;
    d.src = o.src;
    d.spitch = o.spitch;
    d.sbatch = o.sbatch;
    d.H = o.H;
    d.W = o.W;
    d.dst = o.dst;
    d.dpitch = o.dpitch;
    d.dplane = o.dplane;
    d.dbatch = o.dbatch;
    d.h = o.h;
    d.w = o.w;
    d.C = o.cin;
    d.f32 = o.outk == OUT_F32;
    d.chw = o.chw;
    d.batch = o.batch;
    for (int k = 0; k < 3; ++k) {
        d.scale[k] = o.scale[k];
        d.bias[k] = o.bias[k];
    }
    bool too_large = false;
    cudaError_t e = launch_area(d, (cudaStream_t)stream, too_large);
    if (e != cudaSuccess) {
        set_last_error("kr_resize_area", e);
        return KR_ERR_CUDA;
    }
    return too_large ? KR_ERR_UNSUPPORTED : KR_OK;
}

kr_status kr_sobel(const kr_image_t *src, const kr_image_t *dst, int32_t ksize, kr_stream_t stream)
{
    kr_status st;
    if ((st = check_image(src, false)) != KR_OK) return st;
    if ((st = check_image(dst, true)) != KR_OK) return st;
    if (ksize != 3) return KR_ERR_UNSUPPORTED;
    if (src->dtype != KR_U8 || src->layout != KR_HWC || dst->layout != KR_HWC) return KR_ERR_UNSUPPORTED;
    if (dst->channels != 1 || src->height != dst->height || src->width != dst->width || src->batch != dst->batch)
        return KR_ERR_INVALID_ARG;
    if ((st = check_alias(*src, *dst)) != KR_OK) return st;
    SobelDesc d;
    d.src = (const uint8_t *)src->data;
    d.spitch = src->pitch;
    d.sbatch = src->batch > 1 ? src->batch_stride : 0;
    d.H = src->height;
    d.W = src->width;
    d.dst = (uint8_t *)dst->data;
    d.dpitch = dst->pitch;
    d.dbatch = dst->batch > 1 ? dst->batch_stride : 0;
    d.C = src->channels;
    d.f32 = dst->dtype == KR_F32;
    d.batch = src->batch;
    cudaError_t e = launch_sobel(d, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_last_error("kr_sobel", e);
        return KR_ERR_CUDA;
    }
    return KR_OK;
}

kr_status kr_flip_horizontal(const kr_image_t *src, const kr_image_t *dst, kr_stream_t stream)
{
    GatherDesc d;
    kr_status st = build_gather(src, dst, true, d);
    if (st != KR_OK) return st;
    cudaError_t e = launch_flip_h(d, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_last_error("kr_flip_horizontal", e);
        return KR_ERR_CUDA;
    }
    return KR_OK;
}

kr_status kr_resize_bilinear(const kr_image_t *src, const kr_image_t *dst, const kr_post_t *post,
                             kr_stream_t stream)
{
    OpDesc d;
    kr_status st = build_resample(OP_RESIZE, src, dst, post, d);
    if (st != KR_OK) return st;
    cudaError_t e = launch_resample(d, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_last_error("kr_resize_bilinear", e);
        return KR_ERR_CUDA;
    }
    return KR_OK;
}

kr_status kr_warp_affine(const kr_image_t *src, const kr_image_t *dst, const float *M,
                         const kr_post_t *post, kr_stream_t stream)
{
    if (!M) return KR_ERR_INVALID_ARG;
    OpDesc d;
    kr_status st = build_resample(OP_WARP, src, dst, post, d);
    if (st != KR_OK) return st;
    for (int64_t i = 0; i < (int64_t)d.batch * 6; ++i)
        if (!std::isfinite(M[i])) return KR_ERR_INVALID_ARG;
    d.M = M;
    cudaError_t e = launch_resample(d, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_last_error("kr_warp_affine", e);
        return KR_ERR_CUDA;
    }
    return KR_OK;
}

kr_status kr_warp_perspective(const kr_image_t *src, const kr_image_t *dst, const float *M,
                              const kr_post_t *post, kr_stream_t stream)
{
    if (!M) return KR_ERR_INVALID_ARG;
    OpDesc d;
    kr_status st = build_resample(OP_PERSP, src, dst, post, d);
    if (st != KR_OK) return st;
    for (int64_t i = 0; i < (int64_t)d.batch * 9; ++i)
        if (!std::isfinite(M[i])) return KR_ERR_INVALID_ARG;
    d.M = M;
    cudaError_t e = launch_resample(d, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_last_error("kr_warp_perspective", e);
        return KR_ERR_CUDA;
    }
    return KR_OK;
}

kr_status kr_rgb_to_gray(const kr_image_t *src, const kr_image_t *dst, kr_stream_t stream)
{
    GrayDesc d;
    kr_status st = build_gray(src, dst, d);
    if (st != KR_OK) return st;
    cudaError_t e = launch_gray(d, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_last_error("kr_rgb_to_gray", e);
        return KR_ERR_CUDA;
    }
    return KR_OK;
}

const char *kr_status_string(kr_status s)
{
    switch (s) {
    case KR_OK: return "ok";
    case KR_ERR_INVALID_ARG: return "invalid argument";
    case KR_ERR_UNSUPPORTED: return "unsupported combination";
    case KR_ERR_ALIAS: return "source and destination overlap";
    case KR_ERR_CUDA: return "CUDA error";
    case KR_ERR_NO_SPACE: return "workspace or memory budget too small";
    case KR_ERR_TIMEOUT: return "bounded wait timed out";
    }
    return "unknown status";
}

const char *kr_last_error(void) { return g_last_error; }

kr_status kr_debug_set_stage_wait_ns(uint64_t ns)
{
    cudaError_t e = set_stage_wait_ns_ops(ns);
    if (e == cudaSuccess) e = set_stage_wait_ns_batch(ns);
    if (e != cudaSuccess) {
        set_last_error("kr_debug_set_stage_wait_ns", e);
        return KR_ERR_CUDA;
    }
    return KR_OK;
}

kr_status kr_device_errors(uint32_t *flags, int32_t clear)
{
    if (!flags) return KR_ERR_INVALID_ARG;
    unsigned v = 0, vb = 0;
    cudaError_t e = device_error_flags(&v, clear != 0);
    if (e == cudaSuccess) e = batch_error_flags(&vb, clear != 0);
    v |= vb;
    if (e != cudaSuccess) {
        set_last_error("kr_device_errors", e);
        return KR_ERR_CUDA;
    }
    *flags = v;
    return KR_OK;
}

}  // extern "C"
