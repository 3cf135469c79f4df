// Pixel gathers: nearest-neighbour resize and horizontal flip (u8, 1 or 3
// channels, HWC, any pitch, batched). Each output pixel copies one source pixel,
// so the kernels move bytes only: lanes of a warp take consecutive output pixels
// of a row (their source pixels are consecutive too, forwards or backwards), so
// every byte load and store of a warp touches a few adjacent 32-byte sectors.
//
//   nearest  output (x, y) <- source (((2x + 1) W) div (2w), ((2y + 1) H) div (2h))
//            (half-pixel centres: the source pixel covering the output centre)
//   flip     output (x, y) <- source (W - 1 - x, y)
//
// A CTA owns 256 columns x kRows rows of one image: the column map is computed
// once per thread and the row map once per row (shared memory), then every
// row is one load + one store per channel and pixel.
#include "kr_internal.h"

namespace kr {
namespace {

constexpr int kGatherThreads = 256;
constexpr int kRows = 16;

struct GatherParams {
    const uint8_t *src;
    int64_t spitch, sbatch;
    int32_t H, W;
    uint8_t *dst;
    int64_t dpitch, dbatch;
    int32_t h, w;
};

template <int C, bool NEAREST>
__global__ void __launch_bounds__(kGatherThreads) gather_kernel(const __grid_constant__ GatherParams p)
{
    __shared__ int s_sy[kRows];
    const int y0 = blockIdx.y * kRows;
    const int x = blockIdx.x * kGatherThreads + threadIdx.x;
    if (threadIdx.x < kRows) {
        const unsigned long long y = (unsigned long long)(y0 + threadIdx.x);
        s_sy[threadIdx.x] = NEAREST ? (int)(((2ull * y + 1ull) * (unsigned long long)p.H) / (2ull * (unsigned)p.h))
                                    : (int)y;
    }
    __syncthreads();
    if (x >= p.w) return;
    const int sx = NEAREST ? (int)(((2ull * (unsigned)x + 1ull) * (unsigned long long)p.W) / (2ull * (unsigned)p.w))
                           : p.W - 1 - x;
    const uint8_t *sb = p.src + (int64_t)blockIdx.z * p.sbatch + (int64_t)sx * C;
    uint8_t *db = p.dst + (int64_t)blockIdx.z * p.dbatch + (int64_t)x * C;
    const int ny = min(kRows, p.h - y0);
    for (int r = 0; r < ny; ++r) {
        const uint8_t *s = sb + (int64_t)s_sy[r] * p.spitch;
        uint8_t *d = db + (int64_t)(y0 + r) * p.dpitch;
#pragma unroll
        for (int c = 0; c < C; ++c) d[c] = __ldg(s + c);
    }
}

template <bool NEAREST>
cudaError_t launch_gather(const GatherDesc &d, cudaStream_t stream)
{
    GatherParams p;
    p.src = d.src;
    p.spitch = d.spitch;
    p.sbatch = d.sbatch;
    p.H = d.H;
    p.W = d.W;
    p.dst = d.dst;
    p.dpitch = d.dpitch;
    p.dbatch = d.dbatch;
    p.h = d.h;
    p.w = d.w;
    const dim3 grid((d.w + kGatherThreads - 1) / kGatherThreads, (d.h + kRows - 1) / kRows, d.batch);
    if (d.C == 3)
        gather_kernel<3, NEAREST><<<grid, kGatherThreads, 0, stream>>>(p);
    else
        gather_kernel<1, NEAREST><<<grid, kGatherThreads, 0, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_resize_nearest(const GatherDesc &d, cudaStream_t stream) { return launch_gather<true>(d, stream); }
cudaError_t launch_flip_h(const GatherDesc &d, cudaStream_t stream) { return launch_gather<false>(d, stream); }

}  // namespace kr
