// Sobel 3x3 gradient magnitude (the filter of the Sec. V example; u8 HWC source, 1 or 3
// channels; 3 channels are first the u8 BT.601 gray), replicated border, f32 or u8
// single-channel output:
//   m = sqrt(gx^2 + gy^2) / 8 (normalised kernels), u8 = floor(m + 1/2).
// A thread owns 4 output columns x0 .. x0+3 of a run of 16 output rows and walks down the
// run: per source row it forms the gray values of the 6 source pixels x0-1 .. x0+4, their
// horizontal smooths (v0 + 2 v1 + v2) and differences (v2 - v0), and keeps the last three
// rows' in registers. Inside the row (3 channels) the 18 source bytes are read as aligned
// words (their phase is the same for every thread of a row, so one switch picks the byte
// positions) and each gray is one dp2a; at the left and right edges pixels are read one by
// one with the column clamped. No shared memory.
#include "kr_device.cuh"
#include "kr_internal.h"

namespace kr {
namespace {

constexpr int kGroup = 4;   // output columns per thread
constexpr int kRun = 16;    // output rows per thread

struct SobelParams {
    const uint8_t *src;
    int64_t spitch, sbatch;
    int32_t H, W;
    uint8_t *dst;
    int64_t dpitch, dbatch;
};

// gray of the 3-channel pixel in bytes 0..2 of P: (4899 R + 9617 G + 1868 B + 8192) >> 14
__device__ __forceinline__ int gray_word(uint32_t P)
{
    return (int)(__dp2a_lo(4899u | (9617u << 16), P, 8192u + 1868u * ((P >> 16) & 255u)) >> 14);
}

// the six pixels of a row starting at byte SH of the words w[0..5]
template <int SH>
__device__ __forceinline__ void gray6_words(const uint32_t (&w)[6], int (&gv)[6])
{
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const int o = SH + 3 * i;
        gv[i] = gray_word(__funnelshift_r(w[o >> 2], w[(o >> 2) + 1], 8 * (o & 3)));
    }
}

template <int C, bool F32>
__global__ void __launch_bounds__(kThreads) sobel_kernel(const __grid_constant__ SobelParams p)
{
    const int x0 = kGroup * (int)(blockIdx.x * kThreads + threadIdx.x);
    if (x0 >= p.W) return;
    const int y0 = blockIdx.y * kRun, ny = min(kRun, p.H - y0);
    const uint8_t *src = p.src + (int64_t)blockIdx.z * p.sbatch;
    uint8_t *dst = p.dst + (int64_t)blockIdx.z * p.dbatch;
    // word reads stay inside the row: its bytes from 3 (x0 - 2) to 3 (x0 + 6) - 1
    const bool fast = C == 3 && x0 >= 2 && x0 + 5 <= p.W - 1;
    // the fast path loads a row's words one row ahead of its use (load6, then gray6 of them)
    auto load6 = [&](int y, uint32_t (&w)[6], int &sh) {
        const uint8_t *a = src + (int64_t)min(max(y, 0), p.H - 1) * p.spitch + 3 * (x0 - 1);
        sh = (int)((uintptr_t)a & 3);
        const uint32_t *wp = reinterpret_cast<const uint32_t *>(a - sh);
#pragma unroll
        for (int t = 0; t < 6; ++t) w[t] = 4 * t < sh + 18 ? __ldg(wp + t) : 0u;
    };
    uint32_t wq[6];
    int shq = 0;
    auto gray6 = [&](int y, int (&gv)[6]) {
        const uint8_t *row = src + (int64_t)min(max(y, 0), p.H - 1) * p.spitch;
        if (fast) {
            uint32_t w[6];
            int sh = shq;
#pragma unroll
            for (int t = 0; t < 6; ++t) w[t] = wq[t];
            load6(y + 1, wq, shq);   // the next row's words
            switch (sh) {
            case 0: gray6_words<0>(w, gv); break;
            case 1: gray6_words<1>(w, gv); break;
            case 2: gray6_words<2>(w, gv); break;
            default: gray6_words<3>(w, gv); break;
            }
        } else {
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                const uint8_t *s = row + (int64_t)min(max(x0 - 1 + i, 0), p.W - 1) * C;
                gv[i] = C == 3 ? (int)gray_u8(__ldg(s), __ldg(s + 1), __ldg(s + 2)) : (int)__ldg(s);
            }
        }
    };
    int da[4], ha[4], db[4], hb[4];
    if (fast) load6(y0 - 1, wq, shq);
    {
        int gv[6];
        gray6(y0 - 1, gv);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            da[i] = gv[i + 2] - gv[i];
            ha[i] = gv[i] + 2 * gv[i + 1] + gv[i + 2];
        }
        gray6(y0, gv);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            db[i] = gv[i + 2] - gv[i];
            hb[i] = gv[i] + 2 * gv[i + 1] + gv[i + 2];
        }
    }
    const bool full = x0 + 3 < p.W;
#pragma unroll 2
    for (int k = 0; k < ny; ++k) {
        int gv[6];
        gray6(y0 + k + 1, gv);
        float m[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int dc = gv[i + 2] - gv[i], hc = gv[i] + 2 * gv[i + 1] + gv[i + 2];
            const int gx = da[i] + 2 * db[i] + dc, gy = hc - ha[i];
            m[i] = __fmul_rn(__fsqrt_rn((float)(gx * gx + gy * gy)), 0.125f);
            da[i] = db[i];
            ha[i] = hb[i];
            db[i] = dc;
            hb[i] = hc;
        }
        uint8_t *row = dst + (int64_t)(y0 + k) * p.dpitch;
        if (F32) {
            float *o = reinterpret_cast<float *>(row) + x0;
            if (full && ((uintptr_t)o & 15) == 0) {
                *reinterpret_cast<float4 *>(o) = make_float4(m[0], m[1], m[2], m[3]);
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (x0 + i < p.W) o[i] = m[i];
            }
        } else {
            uint8_t *o = row + x0;
            uint8_t v[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) v[i] = (uint8_t)floorf(__fadd_rn(m[i], 0.5f));
            if (full && ((uintptr_t)o & 3) == 0) {
                *reinterpret_cast<uchar4 *>(o) = make_uchar4(v[0], v[1], v[2], v[3]);
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (x0 + i < p.W) o[i] = v[i];
            }
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
    const int groups = (d.W + kGroup - 1) / kGroup;
    const dim3 grid((groups + kThreads - 1) / kThreads, (d.H + kRun - 1) / kRun, d.batch);
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
