// Pixel gathers: nearest-neighbour resize (Sec. IV-A) and horizontal flip (Sec. III,
// Sec. IV-A) of u8 images (1 or 3 channels, HWC, any pitch, batched). Each output pixel
// copies one source pixel, so the kernels move bytes only.
//
//   nearest  output (x, y) <- source (((2x + 1) W) div (2w), ((2y + 1) H) div (2h))
//            (half-pixel centres: the source pixel covering the output centre)
//   flip     output (x, y) <- source (W - 1 - x, y)
//
// Rows whose staged copy fits 48 KB of shared memory: a CTA takes whole output rows. It
// stages each source row in shared memory (16-byte cp.async copies into a ring of two to
// four row buffers: later rows are staged while the current one is written) and writes the
// output row as 16-byte chunks aligned in memory. A 3-channel chunk covers six output
// pixels: each source pixel is read as one funnel-shifted word pair, and the chunk's four
// words are byte permutes of neighbouring pixels; 1-channel chunks are packed byte by byte.
// Longer rows: a CTA owns 256 columns x kRows rows; the column map is computed once per
// thread and the row map once per row (shared memory), then every row is one byte load +
// one byte store per channel and pixel (lanes of a warp take consecutive output pixels, so
// each warp-wide byte access touches a few adjacent 32-byte sectors).
#include <algorithm>

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

constexpr int kRowBufBytes = 48 * 1024;   // one staged source row with its pads and phase
constexpr int kChunkThreadsMax = 1024;

__device__ __forceinline__ void cp_async16(void *sdst, const void *gsrc)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most n of this thread's newest copy groups are still in flight (n < 4)
__device__ __forceinline__ void cp_async_wait(int n)
{
    if (n >= 3)
        asm volatile("cp.async.wait_group 3;\n" ::: "memory");
    else if (n == 2)
        asm volatile("cp.async.wait_group 2;\n" ::: "memory");
    else if (n == 1)
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    else
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ uint32_t lds32(const uint8_t *s) { return *reinterpret_cast<const uint32_t *>(s); }

// Exact quotient num div den for num < 2^34 whose quotient is below 2^17: a float estimate
// (relative error below 2^-22, so off by at most one) corrected with the integer remainder.
__device__ __forceinline__ unsigned div_est(long long num, unsigned den, float inv, unsigned *rem = nullptr)
{
    long long q = (long long)((float)num * inv);
    long long r = num - q * (long long)den;
    if (r < 0) {
        --q;
        r += den;
    } else if (r >= (long long)den) {
        ++q;
        r -= den;
    }
    if (rem) *rem = (unsigned)r;
    return (unsigned)q;
}

// Source column map stepped along a row: sx(x) = ((2x + 1) W) div (2w) for nearest (quotient q
// and remainder r of the division, advanced by 2W per pixel as a whole step plus a carry),
// W - 1 - x for the flip; clamped to the row so that pixels of a chunk outside the output row
// (their bytes are not stored) still read staged bytes; one exact division starts a chunk.
template <bool NEAREST>
struct ColMap {
    unsigned step = 0, rem = 0, w2 = 0;
    float inv = 0.f;
    int W;
    __device__ __forceinline__ ColMap(int W_, int w_) : W(W_)
    {
        if (NEAREST) {
            w2 = 2u * (unsigned)w_;
            const unsigned W2 = 2u * (unsigned)W_;
            step = W2 / w2;
            rem = W2 - step * w2;
            inv = 1.0f / (float)w2;
        }
    }
    struct Cursor {
        unsigned q, r;
        int x;
    };
    __device__ __forceinline__ Cursor at(int x0) const
    {
        Cursor c{0u, 0u, x0};
        if (NEAREST) {
            c.q = div_est((long long)max(x0, 0) * (2LL * W) + W, w2, inv, &c.r);
        }
        return c;
    }
    __device__ __forceinline__ int sx(const Cursor &c) const
    {
        return NEAREST ? min((int)c.q, W - 1) : min(max(W - 1 - c.x, 0), W - 1);
    }
    __device__ __forceinline__ void next(Cursor &c) const
    {
        if (NEAREST && c.x >= 0) {
            c.q += step;
            c.r += rem;
            if (c.r >= w2) {
                c.r -= w2;
                ++c.q;
            }
        }
        ++c.x;
    }
};

// The four output words of a 16-byte chunk whose first byte has pixel phase ph (3 channels):
// word j starts at chunk byte 4j, i.e. pixel (ph + 4j) div 3 of the chunk's six P[0..5], channel
// (ph + 4j) mod 3, and takes its bytes from that pixel and the next one (one byte permute).
__device__ __forceinline__ void words3(const uint32_t (&P)[6], int ph, uint32_t (&w)[4])
{
    constexpr unsigned seq = 0x654210u;   // byte sources: P.c0 P.c1 P.c2 Q.c0 Q.c1 Q.c2
    const unsigned sel0 = (seq >> (4 * ph)) & 0xFFFFu;
    const unsigned sel1 = (seq >> (4 * (ph < 2 ? ph + 1 : 0))) & 0xFFFFu;
    const unsigned sel2 = (seq >> (4 * (ph == 0 ? 2 : ph - 1))) & 0xFFFFu;
    w[0] = __byte_perm(P[0], P[1], sel0);
    w[1] = ph < 2 ? __byte_perm(P[1], P[2], sel1) : __byte_perm(P[2], P[3], sel1);
    w[2] = ph == 0 ? __byte_perm(P[2], P[3], sel2) : __byte_perm(P[3], P[4], sel2);
    w[3] = __byte_perm(P[4], P[5], sel0);
}

template <int C, bool NEAREST>
__global__ void __launch_bounds__(kGatherThreads, 8) row_gather_kernel(const __grid_constant__ GatherParams p, int buf, int nbuf)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const uint8_t *src = p.src + (int64_t)blockIdx.y * p.sbatch;
    uint8_t *dst = p.dst + (int64_t)blockIdx.y * p.dbatch;
    const int sbytes = p.W * C, dbytes = p.w * C;
    const ColMap<NEAREST> cm(p.W, p.w);
    const unsigned h2 = 2u * (unsigned)p.h;
    const float inv_h2 = 1.0f / (float)h2;
    auto row_of = [&](int y) -> const uint8_t * {
        const int sy = NEAREST ? (int)div_est((2LL * y + 1) * p.H, h2, inv_h2) : y;
        return src + (int64_t)sy * p.spitch;
    };
    // stage a source row at its own 16-byte phase: whole aligned chunks by cp.async, the
    // partial head and tail chunks byte by byte (only the row's own bytes are read)
    auto stage = [&](const uint8_t *g, uint8_t *s) {
        const int ph = (int)((uintptr_t)g & 15);
        const uint8_t *g0 = g - ph;
        const int nch = (ph + sbytes + 15) >> 4;
        for (int k = threadIdx.x; k < nch; k += blockDim.x) {
            const int o = 16 * k;
            if (o >= ph && o + 16 <= ph + sbytes) {
                cp_async16(s + o, g0 + o);
            } else {
                for (int b = 0; b < 16; ++b)
                    if (o + b >= ph && o + b < ph + sbytes) s[o + b] = __ldg(g0 + o + b);
            }
        }
    };
    // a ring of nbuf row buffers: rows it+1 .. it+nbuf-1 are in flight while row it is written
    const int G = gridDim.x;
    for (int i = 0; i < nbuf - 1; ++i) {
        const int yi = blockIdx.x + i * G;
        if (yi < p.h) stage(row_of(yi), smem + i * buf);
        cp_async_commit();
    }
    int slot = 0;
    for (int y = blockIdx.x, it = 0; y < p.h; ++it, y += G) {
        uint8_t *s = smem + slot * buf;
        const int ya = y + (nbuf - 1) * G;
        const int sa = slot == 0 ? nbuf - 1 : slot - 1;   // the slot written out one iteration ago
        if (ya < p.h) stage(row_of(ya), smem + sa * buf);
        cp_async_commit();
        cp_async_wait(nbuf - 1);   // this row's copies are done (later rows' may be in flight)
        __syncthreads();
        slot = slot + 1 == nbuf ? 0 : slot + 1;
        const int r0 = (int)((uintptr_t)row_of(y) & 15);   // staged offset of the row's byte 0
        const uint8_t *s0 = s + r0;
        uint8_t *d = dst + (int64_t)y * p.dpitch;
        const int dph = (int)((uintptr_t)d & 15);
        const int nchd = (dph + dbytes + 15) >> 4;
        for (int k = threadIdx.x; k < nchd; k += blockDim.x) {
            const int b0 = 16 * k - dph;   // row byte of the chunk's first byte (>= -15)
            uint32_t w[4];
            if (C == 3) {
                const int xb = (b0 + 15) / 3 - 5;   // floor(b0 / 3)
                const int ph = b0 - 3 * xb;
                auto c = cm.at(xb);
                uint32_t P[6];
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    const int a = r0 + 3 * cm.sx(c);
                    const int sh = a & 3;
                    const uint8_t *qa = s + (a - sh);
                    P[i] = __funnelshift_r(lds32(qa), lds32(qa + 4), 8 * sh);
                    cm.next(c);
                }
                words3(P, ph, w);
            } else {
                auto c = cm.at(b0);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    uint32_t v = 0;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        v |= (uint32_t)s0[cm.sx(c)] << (8 * i);
                        cm.next(c);
                    }
                    w[j] = v;
                }
            }
            uint8_t *dc = d - dph + 16 * k;
            if (b0 >= 0 && b0 + 16 <= dbytes) {
                *reinterpret_cast<uint4 *>(dc) = make_uint4(w[0], w[1], w[2], w[3]);
            } else {
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (b0 + i >= 0 && b0 + i < dbytes) dc[i] = (uint8_t)(w[i >> 2] >> (8 * (i & 3)));
            }
        }
        __syncthreads();   // the buffer is read out before a later row is staged into it
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Nearest-neighbour 3-channel rows whose 16-byte phases are the same in every row and image
// (pitches and batch strides multiples of 16) and whose output row has at most 1024 chunks
// (the kernel also maps the flip, which the launcher sends to the one above): thread k owns output
// chunk k of every row, so its six source offsets (into the staged row) and its byte permutes
// are computed once; a row then costs each thread 12 shared loads, 6 funnel shifts, 4 byte
// permutes and one 16-byte store.
template <bool NEAREST>
__global__ void __launch_bounds__(kChunkThreadsMax, 2) row_gather3_kernel(const __grid_constant__ GatherParams p, int buf,
                                                                           int nbuf)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const uint8_t *src = p.src + (int64_t)blockIdx.y * p.sbatch;
    uint8_t *dst = p.dst + (int64_t)blockIdx.y * p.dbatch;
    const int sbytes = 3 * p.W, dbytes = 3 * p.w;
    const int sph = (int)((uintptr_t)src & 15), dph = (int)((uintptr_t)dst & 15);
    const int nch = (sph + sbytes + 15) >> 4, nchd = (dph + dbytes + 15) >> 4;
    const int k = threadIdx.x;
    const int b0 = 16 * k - dph;                 // row byte of this thread's chunk (>= -15)
    const bool full = b0 >= 0 && b0 + 16 <= dbytes;
    const int xb = (b0 + 15) / 3 - 5, ph = b0 - 3 * xb;   // first pixel of the chunk, its phase
    int off[6];                                  // staged byte offsets of the chunk's six pixels
    {
        const ColMap<NEAREST> cm(p.W, p.w);
        auto c = cm.at(xb);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            off[i] = sph + 3 * cm.sx(c);
            cm.next(c);
        }
    }
    // word j of the chunk: pixel (ph + 4j) div 3 and the next one, from channel (ph + 4j) mod 3
    constexpr unsigned seq = 0x654210u;          // byte sources: P.c0 P.c1 P.c2 Q.c0 Q.c1 Q.c2
    const unsigned sel0 = (seq >> (4 * ph)) & 0xFFFFu;
    const unsigned sel1 = (seq >> (4 * (ph < 2 ? ph + 1 : 0))) & 0xFFFFu;
    const unsigned sel2 = (seq >> (4 * (ph == 0 ? 2 : ph - 1))) & 0xFFFFu;
    const unsigned h2 = 2u * (unsigned)p.h;
    const float inv_h2 = 1.0f / (float)h2;
    auto row_of = [&](int y) -> const uint8_t * {
        const int sy = NEAREST ? (int)div_est((2LL * y + 1) * p.H, h2, inv_h2) : y;
        return src + (int64_t)sy * p.spitch;
    };
    auto stage = [&](const uint8_t *g, uint8_t *s) {
        const uint8_t *g0 = g - sph;
        for (int kk = threadIdx.x; kk < nch; kk += blockDim.x) {
            const int o = 16 * kk;
            if (o >= sph && o + 16 <= sph + sbytes) {
                cp_async16(s + o, g0 + o);
            } else {
                for (int b = 0; b < 16; ++b)
                    if (o + b >= sph && o + b < sph + sbytes) s[o + b] = __ldg(g0 + o + b);
            }
        }
    };
    const int G = gridDim.x;
    for (int i = 0; i < nbuf - 1; ++i) {
        const int yi = blockIdx.x + i * G;
        if (yi < p.h) stage(row_of(yi), smem + i * buf);
        cp_async_commit();
    }
    int slot = 0;
    for (int y = blockIdx.x; y < p.h; y += G) {
        const uint8_t *s = smem + slot * buf;
        const int ya = y + (nbuf - 1) * G;
        const int sa = slot == 0 ? nbuf - 1 : slot - 1;
        if (ya < p.h) stage(row_of(ya), smem + sa * buf);
        cp_async_commit();
        cp_async_wait(nbuf - 1);
        __syncthreads();
        slot = slot + 1 == nbuf ? 0 : slot + 1;
        if (k < nchd) {
            uint32_t P[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                const uint8_t *q = s + (off[i] & ~3);
                P[i] = __funnelshift_r(lds32(q), lds32(q + 4), 8 * (off[i] & 3));
            }
            const uint32_t w0 = __byte_perm(P[0], P[1], sel0);
            const uint32_t w1 = ph < 2 ? __byte_perm(P[1], P[2], sel1) : __byte_perm(P[2], P[3], sel1);
            const uint32_t w2 = ph == 0 ? __byte_perm(P[2], P[3], sel2) : __byte_perm(P[3], P[4], sel2);
            const uint32_t w3 = __byte_perm(P[4], P[5], sel0);
            uint8_t *dc = dst + (int64_t)y * p.dpitch - dph + 16 * k;
            if (full) {
                *reinterpret_cast<uint4 *>(dc) = make_uint4(w0, w1, w2, w3);
            } else {
                const uint32_t w[4] = {w0, w1, w2, w3};
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (b0 + i >= 0 && b0 + i < dbytes) dc[i] = (uint8_t)(w[i >> 2] >> (8 * (i & 3)));
            }
        }
        __syncthreads();
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// The flip of 3-channel rows whose destination rows start on 16-byte boundaries (destination
// pitch, batch stride and base multiples of 16): thread g of a row writes output pixels
// 16g .. 16g+15 (48 bytes, three aligned 16-byte stores) from source pixels W-16-16g ..
// W-1-16g, a 48-byte window whose 16-byte phase is the same for every group of the row. The
// window is read as three or four aligned 16-byte loads and funnel-shifted by that phase, then
// reversed four pixels (12 bytes, four byte permutes) at a time. Groups whose loads would
// leave the source row (at some phases the row's first and last groups) and a partial last
// group copy pixel by pixel. No shared memory: loads and stores are independent per thread.
__global__ void __launch_bounds__(256) flip3_kernel(const __grid_constant__ GatherParams p)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (p.W + 15) >> 4) return;
    const uint8_t *srow = p.src + (int64_t)blockIdx.z * p.sbatch + (int64_t)blockIdx.y * p.spitch;
    uint8_t *drow = p.dst + (int64_t)blockIdx.z * p.dbatch + (int64_t)blockIdx.y * p.dpitch;
    const int sbytes = 3 * p.W;
    const int x0 = 16 * g;                                  // first output pixel of the group
    const int lo = 3 * (p.W - 16 - x0);                     // window start in the row (< 0: partial group)
    const int u = (int)(((uintptr_t)srow + (uintptr_t)(intptr_t)lo) & 15);
    const int la = lo - u;                                  // first aligned block of the window
    const int nb = u == 0 ? 3 : 4;
    if (x0 + 16 <= p.W && la >= 0 && la + 16 * nb <= sbytes) {
        const uint4 *q = reinterpret_cast<const uint4 *>(srow + la);
        const uint4 b0 = __ldg(q), b1 = __ldg(q + 1), b2 = __ldg(q + 2);
        const uint4 b3 = nb == 4 ? __ldg(q + 3) : make_uint4(0u, 0u, 0u, 0u);
        const uint32_t V[16] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w,
                                b2.x, b2.y, b2.z, b2.w, b3.x, b3.y, b3.z, b3.w};
        const int sh = 8 * (u & 3);
        uint32_t A[12];   // the window: source pixels S0 .. S15, S_m at bytes 3m .. 3m+2
        switch (u >> 2) {
        case 0:
#pragma unroll
            for (int j = 0; j < 12; ++j) A[j] = __funnelshift_r(V[j], V[j + 1], sh);
            break;
        case 1:
#pragma unroll
            for (int j = 0; j < 12; ++j) A[j] = __funnelshift_r(V[j + 1], V[j + 2], sh);
            break;
        case 2:
#pragma unroll
            for (int j = 0; j < 12; ++j) A[j] = __funnelshift_r(V[j + 2], V[j + 3], sh);
            break;
        default:
#pragma unroll
            for (int j = 0; j < 12; ++j) A[j] = __funnelshift_r(V[j + 3], V[j + 4], sh);
            break;
        }
        // output pixels 4k .. 4k+3 are S_{15-4k} .. S_{12-4k}: the 12 window bytes of words
        // x0 x1 x2 = A[9-3k] A[10-3k] A[11-3k], pixel order reversed, channel order kept
        uint32_t o[12];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t x0w = A[9 - 3 * k], x1w = A[10 - 3 * k], x2w = A[11 - 3 * k];
            o[3 * k] = __byte_perm(x1w, x2w, 0x2765);                         // S3.c0-2, S2.c0
            o[3 * k + 1] = __byte_perm(__byte_perm(x1w, x2w, 0x0043), x0w, 0x3710);   // S2.c1-2, S1.c0-1
            o[3 * k + 2] = __byte_perm(x0w, x1w, 0x2105);                     // S1.c2, S0.c0-2
        }
        uint4 *d = reinterpret_cast<uint4 *>(drow + 48 * g);
        d[0] = make_uint4(o[0], o[1], o[2], o[3]);
        d[1] = make_uint4(o[4], o[5], o[6], o[7]);
        d[2] = make_uint4(o[8], o[9], o[10], o[11]);
    } else {
        const int n = min(16, p.W - x0);
        for (int i = 0; i < n; ++i) {
            const uint8_t *s = srow + 3 * (p.W - 1 - x0 - i);
            uint8_t *d = drow + 3 * (x0 + i);
            d[0] = __ldg(s);
            d[1] = __ldg(s + 1);
            d[2] = __ldg(s + 2);
        }
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
    if (!NEAREST && d.C == 3 && d.dpitch % 16 == 0 && ((uintptr_t)d.dst & 15) == 0 &&
        (d.batch == 1 || d.dbatch % 16 == 0) && d.H <= 65535 && d.batch <= 65535) {
        const int ng = (d.W + 15) / 16;
        const int bx = std::min(256, 32 * ((ng + 31) / 32));
        const dim3 g3((ng + bx - 1) / bx, d.H, d.batch);
        flip3_kernel<<<g3, bx, 0, stream>>>(p);
        return cudaGetLastError();
    }
    // a staged row: up to 15 bytes of phase, the row, and 8 bytes that word reads may touch
    const long long buf = ((long long)d.W * d.C + 15 + 8 + 15) & ~15LL;
    if (buf <= kRowBufBytes && d.batch <= 65535) {
        // whole rows per CTA, a ring of row buffers (later rows are staged while this one is
        // written); as many CTAs as fit on the GPU at once, each taking rows in turn
        // a deeper ring for short rows: enough bytes in flight per SM to cover the latency
        const int nbuf = (int)std::min(4LL, std::max(2LL, (28LL * 1024) / buf));
        const size_t smem = (size_t)(nbuf * buf);
        // nearest: one chunk per thread when every row has the same phases (3 channels). The
        // flip keeps 256 threads taking chunks in turn: its chunks are cheap to map, and eight
        // CTAs per SM hide the shared-memory latency better than fewer, larger ones.
        const long long nchd = ((long long)((uintptr_t)d.dst & 15) + (long long)d.w * d.C + 15) / 16;
        const bool fixed = NEAREST && d.C == 3 && d.spitch % 16 == 0 && d.dpitch % 16 == 0 &&
                           (d.batch == 1 || (d.sbatch % 16 == 0 && d.dbatch % 16 == 0)) && nchd <= kChunkThreadsMax;
        auto k = fixed ? row_gather3_kernel<NEAREST> : d.C == 3 ? row_gather_kernel<3, NEAREST> : row_gather_kernel<1, NEAREST>;
        const int threads = fixed ? (int)std::max(64LL, 32 * ((nchd + 31) / 32)) : kGatherThreads;
        if (smem > 48 * 1024) {
            const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        int dev = 0, sms = 0, resident = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k, threads, smem);
        if (e != cudaSuccess) return e;
        const int total = std::max(1, resident) * sms;
        const int per_image = std::max(1, std::min(d.h, (total + d.batch - 1) / d.batch));
        const dim3 g2(per_image, d.batch);
        k<<<g2, threads, smem, stream>>>(p, (int)buf, nbuf);
        return cudaGetLastError();
    }
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
