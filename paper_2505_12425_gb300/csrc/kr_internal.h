// Host-side internals shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/kr.h"

namespace kr {

// Largest number of per-image warp matrices carried by one launch's parameters.
constexpr int kMaxMPerLaunch = 128;
// Shared-memory caps: region A (the staged box: one word per pixel for 3-channel
// sources, raw bytes for 1-channel sources) and region B (raw rows of a 3-channel
// box, later the output tile).
constexpr int kFootCap = 40 * 1024;
constexpr int kRegionBCap = 34 * 1024;

// A validated single-image-op request, pointers as device addresses.
struct OpDesc {
    int op;          // OP_RESIZE / OP_WARP / OP_PERSP
    int cin;         // source channels (1 or 3)
    int outk;        // OUT_U8 / OUT_U8_GRAY / OUT_F32 / OUT_F32_GRAY
    const uint8_t *src;
    int64_t spitch, sbatch;
    int H, W;
    uint8_t *dst;
    int64_t dpitch, dplane, dbatch;
    int h, w;
    int chw;
    int batch;
    float scale[3], bias[3];
    const float *M;  // host, 6 * batch floats (warp) or 9 * batch (perspective)
    int replicate;   // warps: replicated border (else zero)
};

// Per-op launch (per-image tiles, blockIdx.z = image). Returns cudaSuccess or the launch error.
cudaError_t launch_resample(const OpDesc &d, cudaStream_t stream);

// Standalone RGB -> gray.
struct GrayDesc {
    const uint8_t *src;
    int64_t spitch, sbatch;
    uint8_t *dst;
    int64_t dpitch, dbatch;
    int H, W, batch;
};
cudaError_t launch_gray(const GrayDesc &d, cudaStream_t stream);

// Pixel gathers (nearest-neighbour resize, horizontal flip): u8 HWC, C = 1 or 3.
struct GatherDesc {
    const uint8_t *src;
    int64_t spitch, sbatch;
    int H, W;
    uint8_t *dst;
    int64_t dpitch, dbatch;
    int h, w;
    int C;
    int batch;
};
cudaError_t launch_resize_nearest(const GatherDesc &d, cudaStream_t stream);

// Sobel 3x3 magnitude: u8 HWC source (C = 1 or 3), single-channel u8 or f32 HWC output.
struct SobelDesc {
    const uint8_t *src;
    int64_t spitch, sbatch;
    int H, W;
    uint8_t *dst;
    int64_t dpitch, dbatch;
    int C;
    int f32;
    int batch;
};
cudaError_t launch_sobel(const SobelDesc &d, cudaStream_t stream);

// Area (antialiased) downscale: u8 HWC source (C = 1 or 3), u8 HWC or f32 HWC/CHW output of
// the same channels, w <= W and h <= H. too_large: two ring slots of one output column's
// source footprint row exceed kAreaSmemCap (nothing launched).
constexpr size_t kAreaSmemCap = 96 * 1024;
struct AreaDesc {
    const uint8_t *src;
    int64_t spitch, sbatch;
    int H, W;
    uint8_t *dst;
    int64_t dpitch, dplane, dbatch;
    int h, w;
    int C;
    int f32, chw;
    int batch;
    float scale[3], bias[3];
};
cudaError_t launch_area(const AreaDesc &d, cudaStream_t stream, bool &too_large);
cudaError_t launch_flip_h(const GatherDesc &d, cudaStream_t stream);

// Shared-memory budget of one tile: region A bytes (0 = no staging) and region B bytes
// (at least out_bytes, the output tile). Multiples of 16.
inline int round128(int x) { return (x + 127) & ~127; }

struct Budget {
    int a = 0;
    int b = 0;
    int cols = 0, rows = 0;   // bound of a tile's source box (pixels), clipped to the image
    bool fits = false;        // a box of that bound fits the staging caps
};
Budget budget_resize(int cin, int H, int W, int h, int w, int tw, int th, int out_bytes);
Budget budget_warp(int cin, int H, int W, const float *M, int tw, int th, int out_bytes);
Budget budget_persp(int cin, int H, int W, const float *M, int h, int w, int tw, int th, int out_bytes);
// Warp maps whose terms |m00| w, |m01| h, |m02| (and the second row) stay below 2^19 keep
// every intermediate of the fp32 coordinate below 2^20, so interior pixels deviate from the
// corner hull by far less than the box margin: such maps may use the fast tile path.
bool warp_allows_fast(const float *M, int h, int w);

// Device error flags of the per-operation kernels (synchronous read, optional clear).
cudaError_t device_error_flags(unsigned *flags, bool clear);
// Bound of the first wait for a staged box (per-operation kernels; ragged kernels).
cudaError_t set_stage_wait_ns_ops(unsigned long long ns);
cudaError_t set_stage_wait_ns_batch(unsigned long long ns);
cudaError_t batch_error_flags(unsigned *flags, bool clear);

// Validation + descriptor construction (kr_abi.cu); nothing is enqueued.
kr_status build_resample(int op, const kr_image_t *src, const kr_image_t *dst, const kr_post_t *post,
                         OpDesc &d);
kr_status build_gray(const kr_image_t *src, const kr_image_t *dst, GrayDesc &d);

// Thread-local last CUDA error text.
void set_last_error(const char *what, cudaError_t e);

}  // namespace kr
