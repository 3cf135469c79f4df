// Sobel 3x3 gradient magnitude (u8 HWC source, 1 or 3 channels; 3 channels are first the
// u8 BT.601 gray), replicated border, f32 or u8 single-channel output:
//   m = sqrt(gx^2 + gy^2) / 8 (normalised kernels), u8 = floor(m + 1/2).
// One CTA of 256 threads per 64 x 32 output tile: the tile's gray values with a one-pixel
// halo (border replicated) are staged in shared memory; each thread then slides a 3 x 3
// window down 4 rows of 2 columns, keeping per row the horizontal smooth (v0 + 2 v1 + v2)
// and difference (v2 - v0), so each output reads 3 new shared-memory bytes.
#include "kr_device.cuh"
#include "kr_internal.h"

namespace kr {
namespace {

constexpr int kSW = 64, kSH = 32;                     // output tile
constexpr int kHW = kSW + 2, kHH = kSH + 2;           // staged halo box
constexpr int kRowsPerThread = kSH / kWarps;          // 4

struct SobelParams {
    const uint8_t *src;
    int64_t spitch, sbatch;
    int32_t H, W;
    uint8_t *dst;
    int64_t dpitch, dbatch;
};

template <int C, bool F32>
__global__ void __launch_bounds__(kThreads) sobel_kernel(const __grid_constant__ SobelParams p)
{
    __shared__ uint8_t g[kHH][kHW + 2];
    const int tx0 = blockIdx.x * kSW, ty0 = blockIdx.y * kSH;
    const uint8_t *src = p.src + (int64_t)blockIdx.z * p.sbatch;
    // stage the gray halo box, border replicated
    for (int i = threadIdx.x; i < kHH * kHW; i += kThreads) {
        const int hy = i / kHW, hx = i - hy * kHW;
        const int y = min(max(ty0 + hy - 1, 0), p.H - 1), x = min(max(tx0 + hx - 1, 0), p.W - 1);
        const uint8_t *s = src + (int64_t)y * p.spitch + (int64_t)x * C;
        g[hy][hx] = C == 3 ? (uint8_t)gray_u8(__ldg(s), __ldg(s + 1), __ldg(s + 2)) : __ldg(s);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r0 = warp * kRowsPerThread;
    uint8_t *dst = p.dst + (int64_t)blockIdx.z * p.dbatch;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int c = lane + 32 * j;             // output column in the tile; halo column c + 1
        const int x = tx0 + c;
        if (x >= p.W) continue;
        // rows r0 - 1 and r0 of the output are halo rows r0 and r0 + 1
        int d_a, h_a, d_b, h_b;
        {
            const int v0 = g[r0][c], v1 = g[r0][c + 1], v2 = g[r0][c + 2];
            d_a = v2 - v0;
            h_a = v0 + 2 * v1 + v2;
        }
        {
            const int v0 = g[r0 + 1][c], v1 = g[r0 + 1][c + 1], v2 = g[r0 + 1][c + 2];
            d_b = v2 - v0;
            h_b = v0 + 2 * v1 + v2;
        }
#pragma unroll
        for (int k = 0; k < kRowsPerThread; ++k) {
            const int hr = r0 + k + 2;
            const int v0 = g[hr][c], v1 = g[hr][c + 1], v2 = g[hr][c + 2];
            const int d_c = v2 - v0, h_c = v0 + 2 * v1 + v2;
            const int gx = d_a + 2 * d_b + d_c;
            const int gy = h_c - h_a;
            const int y = ty0 + r0 + k;
            if (y < p.H) {
                const float m = __fmul_rn(__fsqrt_rn((float)(gx * gx + gy * gy)), 0.125f);
                uint8_t *row = dst + (int64_t)y * p.dpitch;
                if (F32)
                    reinterpret_cast<float *>(row)[x] = m;
                else
                    row[x] = (uint8_t)floorf(__fadd_rn(m, 0.5f));
            }
            d_a = d_b; h_a = h_b;
            d_b = d_c; h_b = h_c;
        }
    }
}

}  // namespace

cudaError_t launch_sobel(const SobelDesc &d, cudaStream_t stream)
{
    SobelParams p;
    p.src = d.src;
    p.spitch = d.spitch;
    p.sbatch = d.sbatch;
    p.H = d.H;
    p.W = d.W;
    p.dst = d.dst;
    p.dpitch = d.dpitch;
    p.dbatch = d.dbatch;
    const dim3 grid((d.W + kSW - 1) / kSW, (d.H + kSH - 1) / kSH, d.batch);
    if (d.C == 3) {
        if (d.f32) sobel_kernel<3, true><<<grid, kThreads, 0, stream>>>(p);
        else sobel_kernel<3, false><<<grid, kThreads, 0, stream>>>(p);
    } else {
        if (d.f32) sobel_kernel<1, true><<<grid, kThreads, 0, stream>>>(p);
        else sobel_kernel<1, false><<<grid, kThreads, 0, stream>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace kr
