// Area (antialiased) downscale: each output pixel is the overlap-weighted mean of the
// source over its footprint [x W/w, (x+1) W/w) x [y H/h, (y+1) H/h). In units of 1/w and
// 1/h of a pixel the overlaps are integers, so the weighted sum S is exact (32-bit when
// 255 W H < 2^32, else 64-bit) and u8 = floor((2 S + W H) / (2 W H)); f32 outputs take
// S / (W H) in fp32 and the fused normalisation.
//
// A CTA owns up to 64 output columns of a band of R output rows (R chosen on the host so
// that the band's footprint box fits in shared memory). It stages the box once (rows of u8
// pixels, coalesced byte loads) with, per output row, the weights of its source rows;
// thread (column, channel) then works out its column footprint once and, row by row of the
// band, sums column by column the row-weighted sum times the column weight.
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "kr_device.cuh"
#include "kr_internal.h"

namespace kr {
namespace {

constexpr int kAreaCols = 64;       // output columns per CTA
constexpr int kAreaMaxRows = 16;    // output rows per CTA at most

struct AreaParams {
    const uint8_t *src;
    int64_t spitch, sbatch;
    int32_t H, W;
    uint8_t *dst;
    int64_t dpitch, dplane, dbatch;
    int32_t h, w;
    int32_t C;
    int32_t f32, chw;
    int32_t rows;                   // output rows per CTA (R)
    int32_t box_cols;               // staged columns per row (bound over the CTAs)
    int32_t box_rows;               // staged rows (bound over the CTAs)
    int32_t fp_rows;                // source rows one output row's footprint can span
    int32_t bc;                     // bytes per staged row (a multiple of 16)
    int32_t rows16;                 // source base and pitch are 16-byte aligned
    float inv_wh;                   // 1 / (W H)
    float inv_2wh;                  // 1 / (2 W H)
    float scale[3], bias[3];
};

// WIDE: 64-bit sums (255 W H >= 2^32). IDX64: 64-bit footprint arithmetic ((w + 1) W or
// (h + 1) H >= 2^32); else every product and quotient of the footprint bounds is 32-bit.
template <bool WIDE, bool IDX64>
__global__ void __launch_bounds__(kThreads) area_kernel(const __grid_constant__ AreaParams p)
{
    using Acc = typename std::conditional<WIDE, unsigned long long, unsigned>::type;
    using Ix = typename std::conditional<IDX64, unsigned long long, unsigned>::type;
    extern __shared__ __align__(16) uint8_t sm[];
    __shared__ int s_j0[kAreaMaxRows], s_nj[kAreaMaxRows];
    int *ayt = reinterpret_cast<int *>(sm);                      // [rows][fp_rows] row weights
    uint8_t *box = sm + ((kAreaMaxRows * p.fp_rows * 4 + 15) & ~15);
    const int bc = p.bc;                                         // bytes per staged row
    const int xs = blockIdx.x * kAreaCols, nx = min(kAreaCols, p.w - xs);
    const int y0 = blockIdx.y * p.rows, ny = min(p.rows, p.h - y0);
    const uint8_t *src = p.src + (int64_t)blockIdx.z * p.sbatch;
    // the band's source box: footprints of its nx columns and ny rows
    const Ix Wd = (Ix)p.W, Hd = (Ix)p.H, wd = (Ix)p.w, hd = (Ix)p.h;
    const int i_lo = (int)(((Ix)xs * Wd) / wd);
    const int i_hi = (int)min(((Ix)(xs + nx) * Wd - 1) / wd, Wd - 1);
    const int j_lo = (int)(((Ix)y0 * Hd) / hd);
    const int j_hi = (int)min(((Ix)(y0 + ny) * Hd - 1) / hd, Hd - 1);
    const int ncols = i_hi - i_lo + 1, nrows = j_hi - j_lo + 1;  // <= box_cols, box_rows
    if (threadIdx.x < ny) {
        // output row r: source rows [j0, j0 + nj) with their overlaps (units of 1/h)
        const int r = threadIdx.x;
        const Ix ya = (Ix)(y0 + r) * Hd, yb = ya + Hd;
        const int j0 = (int)(ya / hd);
        const int j1 = (int)min((yb - 1) / hd, Hd - 1);
        s_j0[r] = j0 - j_lo;
        s_nj[r] = j1 - j0 + 1;
        for (int k = 0; k <= j1 - j0; ++k) {
            const Ix j = (Ix)(j0 + k);
            ayt[r * p.fp_rows + k] = (int)(min(yb, (j + 1) * hd) - max(ya, j * hd));
        }
    }
    const int rowb = ncols * p.C;
    // 16-byte aligned rows: every staged row keeps the phase ph of its first byte and is
    // copied as whole 16-byte chunks, except those cut by the end of the image row (byte by
    // byte: nothing past the row's own W C bytes is read); else byte by byte at phase 0
    const int ph = p.rows16 ? (i_lo * p.C) & 15 : 0;
    if (p.rows16) {
        const int nch = (ph + rowb + 15) >> 4;
        const int lim = p.W * p.C - (i_lo * p.C - ph);           // row bytes from the first chunk
        for (int k = threadIdx.x; k < nrows * nch; k += kThreads) {
            const int rr = k / nch, jc = k - rr * nch;
            const uint8_t *g = src + (int64_t)(j_lo + rr) * p.spitch + (int64_t)(i_lo * p.C - ph) + 16 * jc;
            uint8_t *d = box + rr * bc + 16 * jc;
            if (16 * jc + 16 <= lim) {
                *reinterpret_cast<uint4 *>(d) = __ldg(reinterpret_cast<const uint4 *>(g));
            } else {
                for (int b = 0; b < 16 && 16 * jc + b < lim; ++b) d[b] = __ldg(g + b);
            }
        }
    } else {
        for (int rr = 0; rr < nrows; ++rr) {
            const uint8_t *g = src + (int64_t)(j_lo + rr) * p.spitch + (int64_t)i_lo * p.C;
            uint8_t *d = box + rr * bc;
            for (int b = threadIdx.x; b < rowb; b += kThreads) d[b] = __ldg(g + b);
        }
    }
    __syncthreads();
    const int tx = threadIdx.x % kAreaCols, c = threadIdx.x / kAreaCols;
    if (tx >= nx || c >= p.C) return;
    const int x = xs + tx;
    const Ix xa = (Ix)x * Wd, xb = xa + Wd;
    const int i0 = (int)(xa / wd), i1 = (int)min((xb - 1) / wd, Wd - 1);
    const unsigned long long wh = (unsigned long long)p.W * (unsigned)p.H;
    uint8_t *drow = p.dst + (int64_t)blockIdx.z * p.dbatch + (int64_t)y0 * p.dpitch;
    for (int r = 0; r < ny; ++r) {
        const int nj = s_nj[r];
        const int *ay = ayt + r * p.fp_rows;
        const uint8_t *col0 = box + s_j0[r] * bc + ph + c;
        Acc S = 0;
        for (int i = i0; i <= i1; ++i) {
            const Ix ax = min(xb, (Ix)(i + 1) * wd) - max(xa, (Ix)i * wd);
            const uint8_t *col = col0 + (i - i_lo) * p.C;
            Acc cs = 0;
            for (int k = 0; k < nj; ++k) cs += (Acc)ay[k] * col[k * bc];
            S += (Acc)ax * cs;
        }
        uint8_t *row = drow + (int64_t)r * p.dpitch;
        if (!p.f32) {
            // floor((2 S + W H) / (2 W H)) in [0, 255]: a float estimate is within one of the
            // quotient; one step each way makes it exact
            const unsigned long long num = 2ull * (unsigned long long)S + wh, den = 2ull * wh;
            unsigned q = (unsigned)__fmul_rz((float)num, p.inv_2wh);
            if ((unsigned long long)q * den > num) --q;
            else if ((unsigned long long)(q + 1) * den <= num) ++q;
            row[x * p.C + c] = (uint8_t)q;
        } else {
            const float v = __fmul_rn((float)S, p.inv_wh);       // mean in [0, 255]
            const float o = __fmaf_rn(v, p.scale[c], p.bias[c]);
            if (p.chw)
                reinterpret_cast<float *>(row + (int64_t)c * p.dplane)[x] = o;
            else
                reinterpret_cast<float *>(row)[x * p.C + c] = o;
        }
    }
}

}  // namespace

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
    p.inv_2wh = (float)(0.5 / ((double)d.W * (double)d.H));
    for (int k = 0; k < 3; ++k) {
        p.scale[k] = d.scale[k];   // applied to the mean in [0, 255], as to the other paths' v255
        p.bias[k] = d.bias[k];
    }
    // footprint bounds: one output row spans at most ceil(H/h) + 1 source rows, R rows at most
    // ceil(R H/h) + 1, and 64 columns at most ceil(64 W/w) + 1 source columns
    p.fp_rows = (int)((d.H + d.h - 1) / d.h) + 1;
    p.box_cols = (int)std::min<long long>(((long long)kAreaCols * d.W + d.w - 1) / d.w + 1, d.W);
    p.bc = round16(p.box_cols * d.C + 15);                      // room for the 16-byte phase
    p.rows16 = ((uintptr_t)d.src & 15) == 0 && (d.spitch & 15) == 0 && (d.batch == 1 || (d.sbatch & 15) == 0);
    const size_t head = (size_t)((kAreaMaxRows * p.fp_rows * 4 + 15) & ~15);
    too_large = true;
    for (int R = kAreaMaxRows; R >= 1; --R) {
        const int rows = (int)std::min<long long>(((long long)R * d.H + d.h - 1) / d.h + 1, d.H);
        if (head + (size_t)rows * p.bc <= kAreaSmemCap) {
            p.rows = R;
            p.box_rows = rows;
            too_large = false;
            break;
        }
    }
    if (too_large) return cudaSuccess;
    const size_t smem = head + (size_t)p.box_rows * p.bc;
    const bool wide = 255.0 * (double)d.W * (double)d.H >= 4294967296.0;
    const bool idx64 = ((double)d.w + 1) * d.W >= 4294967296.0 || ((double)d.h + 1) * d.H >= 4294967296.0;
    const void *k = wide ? (idx64 ? (const void *)area_kernel<true, true> : (const void *)area_kernel<true, false>)
                         : (idx64 ? (const void *)area_kernel<false, true> : (const void *)area_kernel<false, false>);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAreaSmemCap);
    if (e != cudaSuccess) return e;
    const dim3 grid((d.w + kAreaCols - 1) / kAreaCols, (d.h + p.rows - 1) / p.rows, d.batch);
    void *args[] = {&p};
    e = cudaLaunchKernel(k, grid, dim3(kThreads), args, smem, stream);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace kr
