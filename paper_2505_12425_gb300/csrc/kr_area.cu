// Area (antialiased) downscale: each output pixel is the overlap-weighted mean of the
// source over its footprint [x W/w, (x+1) W/w) x [y H/h, (y+1) H/h). In units of 1/w and
// 1/h of a pixel the overlaps are integers, so the weighted sum S is exact (32-bit when
// 255 W H < 2^32, else 64-bit) and u8 = floor((2 S + W H) / (2 W H)); f32 outputs take
// S / (W H) in fp32 and the fused normalisation.
//
// A CTA owns up to 64 output columns of one band of output rows. For each output row it
// stages the footprint box of its columns (rows of u8 pixels, coalesced) and the row
// weights in shared memory, then thread (column, channel) sums its footprint: column by
// column, the column's row-weighted sum, times the column weight.
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "kr_device.cuh"
#include "kr_internal.h"

namespace kr {
namespace {

constexpr int kAreaCols = 64;       // output columns per CTA
constexpr int kAreaRows = 4;        // output rows per CTA (one after another)

struct AreaParams {
    const uint8_t *src;
    int64_t spitch, sbatch;
    int32_t H, W;
    uint8_t *dst;
    int64_t dpitch, dplane, dbatch;
    int32_t h, w;
    int32_t C;
    int32_t f32, chw;
    int32_t box_cols;               // staged columns per row (bound over the CTAs)
    float inv_wh;                   // 1 / (W H)
    float scale[3], bias[3];
};

template <bool WIDE>
__global__ void __launch_bounds__(kThreads) area_kernel(const __grid_constant__ AreaParams p)
{
    using Acc = typename std::conditional<WIDE, unsigned long long, unsigned>::type;
    extern __shared__ __align__(16) uint8_t sm[];
    int *ay = reinterpret_cast<int *>(sm);                       // row weights of the box
    const int maxr = (p.H + p.h - 1) / p.h + 1;                  // rows a footprint can span
    uint8_t *box = sm + ((maxr * 4 + 15) & ~15);
    const int bc = p.box_cols * p.C;                             // bytes per staged row
    const int xs = blockIdx.x * kAreaCols;
    const int nx = min(kAreaCols, p.w - xs);
    const int tx = threadIdx.x % kAreaCols, c = threadIdx.x / kAreaCols;
    const int x = xs + tx;
    const uint8_t *src = p.src + (int64_t)blockIdx.z * p.sbatch;
    // the CTA's source columns: footprints of its nx output columns
    const long long xa0 = (long long)xs * p.W, xb1 = (long long)(xs + nx) * p.W;
    const int i_lo = (int)(xa0 / p.w), i_hi = (int)min((xb1 - 1) / p.w, (long long)p.W - 1);
    const int ncols = i_hi - i_lo + 1;                           // <= box_cols
    for (int r = 0; r < kAreaRows; ++r) {
        const int y = blockIdx.y * kAreaRows + r;
        if (y >= p.h) break;
        const long long ya = (long long)y * p.H, yb = (long long)(y + 1) * p.H;
        const int j_lo = (int)(ya / p.h), j_hi = (int)min((yb - 1) / p.h, (long long)p.H - 1);
        const int nrows = j_hi - j_lo + 1;                       // <= maxr
        if (r > 0) __syncthreads();                              // the previous row's box is read
        for (int k = threadIdx.x; k < nrows; k += kThreads) {
            const long long j = j_lo + k;
            ay[k] = (int)(min(yb, (j + 1) * (long long)p.h) - max(ya, j * (long long)p.h));
        }
        for (int k = threadIdx.x; k < nrows * ncols * p.C; k += kThreads) {
            const int rr = k / (ncols * p.C), b = k - rr * (ncols * p.C);
            box[rr * bc + b] = __ldg(src + (int64_t)(j_lo + rr) * p.spitch + (int64_t)i_lo * p.C + b);
        }
        __syncthreads();
        if (tx < nx && c < p.C) {
            const long long xa = (long long)x * p.W, xb = (long long)(x + 1) * p.W;
            const int i0 = (int)(xa / p.w), i1 = (int)min((xb - 1) / p.w, (long long)p.W - 1);
            Acc S = 0;
            for (int i = i0; i <= i1; ++i) {
                const long long ax = min(xb, (long long)(i + 1) * p.w) - max(xa, (long long)i * p.w);
                const uint8_t *col = box + (i - i_lo) * p.C + c;
                Acc cs = 0;
                for (int rr = 0; rr < nrows; ++rr) cs += (Acc)ay[rr] * col[rr * bc];
                S += (Acc)ax * cs;
            }
            uint8_t *row = p.dst + (int64_t)blockIdx.z * p.dbatch + (int64_t)y * p.dpitch;
            if (!p.f32) {
                const unsigned long long wh = (unsigned long long)p.W * (unsigned)p.H;
                row[x * p.C + c] = (uint8_t)((2ull * (unsigned long long)S + wh) / (2ull * wh));
            } else {
                const float v = __fmul_rn((float)S, p.inv_wh);   // mean in [0, 255]
                const float o = __fmaf_rn(v, p.scale[c], p.bias[c]);
                if (p.chw)
                    reinterpret_cast<float *>(row + (int64_t)c * p.dplane)[x] = o;
                else
                    reinterpret_cast<float *>(row)[x * p.C + c] = o;
            }
        }
    }
}

}  // namespace

// Shared bytes an area launch needs (0: the footprint box of 64 columns is too large).
static size_t area_smem(const AreaDesc &d, int &box_cols)
{
    const int maxr = (d.H + d.h - 1) / d.h + 1;
    box_cols = (int)std::min<long long>(((long long)kAreaCols * d.W + d.w - 1) / d.w + 1, d.W);
    const size_t bytes = (size_t)((maxr * 4 + 15) & ~15) + (size_t)maxr * box_cols * d.C;
    return bytes;
}

cudaError_t launch_area(const AreaDesc &d, cudaStream_t stream, bool &too_large)
{
    AreaParams p;
    std::memset(&p, 0, sizeof(p));
    p.src = d.src;
    p.spitch = d.spitch;
    p.sbatch = d.sbatch;
    p.H = d.H;
    p.W = d.W;
    p.dst = d.dst;
    p.dpitch = d.dpitch;
    p.dplane = d.dplane;
    p.dbatch = d.dbatch;
    p.h = d.h;
    p.w = d.w;
    p.C = d.C;
    p.f32 = d.f32;
    p.chw = d.chw;
    p.inv_wh = (float)(1.0 / ((double)d.W * (double)d.H));
    for (int k = 0; k < 3; ++k) {
        p.scale[k] = d.scale[k];   // applied to the mean in [0, 255], as to the other paths' v255
        p.bias[k] = d.bias[k];
    }
    const size_t smem = area_smem(d, p.box_cols);
    too_large = smem > kAreaSmemCap;
    if (too_large) return cudaSuccess;
    const bool wide = 255.0 * (double)d.W * (double)d.H >= 4294967296.0;
    const void *k = wide ? (const void *)area_kernel<true> : (const void *)area_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAreaSmemCap);
    if (e != cudaSuccess) return e;
    const dim3 grid((d.w + kAreaCols - 1) / kAreaCols, (d.h + kAreaRows - 1) / kAreaRows, d.batch);
    if (wide)
        area_kernel<true><<<grid, kThreads, smem, stream>>>(p);
    else
        area_kernel<false><<<grid, kThreads, smem, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace kr
