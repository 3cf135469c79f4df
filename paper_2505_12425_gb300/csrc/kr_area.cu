// Area (antialiased) downscale, a variant of the paper's downsizing (Sec. III), which
// prints no interpolation rule: each output pixel is the overlap-weighted mean of the
// source over its footprint [x W/w, (x+1) W/w) x [y H/h, (y+1) H/h). In units of 1/w and
// 1/h of a pixel the overlaps are integers, so the weighted sum S is exact (32-bit when
// 255 W H < 2^32, else 64-bit) and u8 = floor((2 S + W H) / (2 W H)); f32 outputs take
// S / (W H) in fp32 and the fused normalisation.
//
// The sum is separable and every source row overlaps at most two output rows (H >= h), so a
// CTA streams source rows: it owns a strip of up to 768 / C output columns and a band of R
// output rows, and passes the band's source rows through a ring of shared-memory row buffers
// (16-byte cp.async copies of the strip's bytes; later rows are in flight while one is
// summed). For each source row, every (column, channel) value of the strip takes its
// horizontal sum over its column footprint (first and last taps partial, interior taps of
// weight w) and adds it, times the row's overlap, to the sums of the output rows the source
// row overlaps; an output row whose footprint is complete is written out. Each source byte
// is read from HBM once per band (the row shared by two bands twice).
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "kr_device.cuh"
#include "kr_internal.h"

namespace kr {
namespace {

constexpr int kStripValues = 768;   // (column, channel) values per CTA: a column (C = 3) or three (C = 1) per thread

struct AreaParams {
    const uint8_t *src;
    int64_t spitch, sbatch;
    int32_t H, W;
    uint8_t *dst;
    int64_t dpitch, dplane, dbatch;
    int32_t h, w;
    int32_t C;
    int32_t f32, chw;
    int32_t nx;                     // output columns per strip
    int32_t R;                      // output rows per band
    int32_t segrow;                 // bytes per staged row (a multiple of 16)
    int32_t K;                      // source rows per ring slot
    int32_t nbuf;                   // ring slots (2 .. 4)
    int32_t fin32;                  // 512 W H < 2^32: the u8 rounding runs in 32-bit integers
    float inv_wh;                   // 1 / (W H)
    float inv_2wh;                  // 1 / (2 W H)
    float scale[3], bias[3];
};

__device__ __forceinline__ void area_cp16(void *sdst, const void *gsrc)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
}

// Interior taps of a 3-channel column: the channel sums of the bytes [A, E) of a staged row
// (E - A a multiple of 3, byte A of channel 0). Aligned words are read and each word adds its
// bytes of one channel with one dp4a against a 0/1 byte mask; the word at A & ~3 starts
// (A & 3) bytes before channel 0, so the masks of word t follow t + (A & 3) modulo 3, and the
// bytes outside [A, E) are masked off in the first and last words.
__device__ __forceinline__ void interior3(const uint8_t *ring_base, int A, int E, unsigned (&S)[3])
{
    const int a0 = A & ~3;
    const int nw = (E - a0 + 3) >> 2;
    const uint32_t *wp = reinterpret_cast<const uint32_t *>(ring_base + a0);
    const uint32_t head = 0xFFFFFFFFu << (8 * (A - a0));                  // bytes >= A of word 0
    const int tail_bytes = E - (a0 + 4 * (nw - 1));                       // 1 .. 4 bytes of the last word
    const uint32_t tail = tail_bytes >= 4 ? 0xFFFFFFFFu : (1u << (8 * tail_bytes)) - 1u;
    // U[r]: sums of the bytes whose channel is (r - (A - a0)) mod 3 relative to word 0's byte 0
    unsigned U0 = 0, U1 = 0, U2 = 0;
    for (int t = 0; t < nw; t += 3) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (t + d < nw) {
                uint32_t v = wp[t + d];
                if (t + d == 0) v &= head;
                if (t + d == nw - 1) v &= tail;
                // word t + d: its byte j is at relative position 4 (t + d) + j, i.e. class (d + j) mod 3
                const uint32_t m0 = d == 0 ? 0x01000001u : d == 1 ? 0x00010000u : 0x00000100u;
                const uint32_t m1 = d == 0 ? 0x00000100u : d == 1 ? 0x01000001u : 0x00010000u;
                const uint32_t m2 = d == 0 ? 0x00010000u : d == 1 ? 0x00000100u : 0x01000001u;
                U0 = __dp4a(v, m0, U0);
                U1 = __dp4a(v, m1, U1);
                U2 = __dp4a(v, m2, U2);
            }
        }
    }
    // class r holds channel (r - (A - a0)) mod 3
    const int sft = A - a0;
    S[0] = sft == 0 ? U0 : sft == 1 ? U1 : sft == 2 ? U2 : U0;
    S[1] = sft == 0 ? U1 : sft == 1 ? U2 : sft == 2 ? U0 : U1;
    S[2] = sft == 0 ? U2 : sft == 1 ? U0 : sft == 2 ? U1 : U2;
}

// WIDE: 64-bit sums (255 W H >= 2^32). C = 3: a thread owns one output column (its three
// channels); C = 1: three columns, tid + 256 k.
template <bool WIDE, int C>
__global__ void __launch_bounds__(kThreads, 4) area_kernel(const __grid_constant__ AreaParams p)
{
    using Acc = typename std::conditional<WIDE, unsigned long long, unsigned>::type;
    using u64 = unsigned long long;
    constexpr int NCOL = C == 3 ? 1 : 3;
    extern __shared__ __align__(16) uint8_t ring[];
    // per source row of the current slot: overlap with the output row being summed, overlap
    // with the next one, whether the row completes the first, and the row's staged byte 0
    __shared__ int4 s_row[16];
    const int xs = blockIdx.x * p.nx, nx = min(p.nx, p.w - xs);
    const int ya = blockIdx.y * p.R, yb = min(ya + p.R, p.h);
    const uint8_t *src = p.src + (int64_t)blockIdx.z * p.sbatch;
    const u64 W = (u64)p.W, H = (u64)p.H, w = (u64)p.w, h = (u64)p.h;
    // the strip's source columns and the band's source rows
    const int i_lo = (int)((u64)xs * W / w);
    const int i_hi = (int)min(((u64)(xs + nx) * W - 1) / w, W - 1);
    const int sbytes = (i_hi - i_lo + 1) * C;                   // <= segrow - 15
    const int j_lo = (int)((u64)ya * H / h);
    const int j_hi = (int)min(((u64)yb * H - 1) / h, H - 1);
    const int nrows = j_hi - j_lo + 1;
    // this thread's columns: staged offset of the first tap, number of taps, first and last
    // overlaps (units of 1/w; interior taps: w)
    int off[NCOL], nt[NCOL];
    unsigned af[NCOL], al[NCOL];
#pragma unroll
    for (int m = 0; m < NCOL; ++m) {
        const int x = threadIdx.x + kThreads * m;
        const u64 xa = (u64)(xs + min(x, nx - 1)) * W, xb = xa + W;
        const int i0 = (int)(xa / w), i1 = (int)min((xb - 1) / w, W - 1);
        nt[m] = x < nx ? i1 - i0 + 1 : 0;                       // 0: no column
        af[m] = (unsigned)(min(xb, (u64)(i0 + 1) * w) - xa);     // W when the footprint is one column
        al[m] = (unsigned)(xb - (u64)i1 * w);
        off[m] = (i0 - i_lo) * C;
    }
    Acc cur[3] = {0, 0, 0}, nxt[3] = {0, 0, 0};
    auto row_of = [&](int j) { return src + (int64_t)j * p.spitch + (int64_t)i_lo * C; };
    // stage a source row's strip at its own 16-byte phase: whole aligned chunks by cp.async,
    // the partial head and tail chunks byte by byte (only the row's own bytes are read)
    auto stage = [&](int j, uint8_t *s) {
        const uint8_t *g = row_of(j);
        const int ph = (int)((uintptr_t)g & 15);
        const uint8_t *g0 = g - ph;
        const int nch = (ph + sbytes + 15) >> 4;
        for (int k = threadIdx.x; k < nch; k += kThreads) {
            const int o = 16 * k;
            if (o >= ph && o + 16 <= ph + sbytes) {
                area_cp16(s + o, g0 + o);
            } else {
                for (int b = 0; b < 16; ++b)
                    if (o + b >= ph && o + b < ph + sbytes) s[o + b] = __ldg(g0 + o + b);
            }
        }
    };
    // ring slot u holds source rows j_lo + K u .. j_lo + K u + K - 1
    const int nbuf = p.nbuf, K = p.K, slotb = K * p.segrow;
    const int nslots = (nrows + K - 1) / K;
    auto stage_slot = [&](int u, uint8_t *s) {
        for (int r = 0; r < K && K * u + r < nrows; ++r) stage(j_lo + K * u + r, s + r * p.segrow);
    };
    for (int i = 0; i < nbuf - 1; ++i) {
        if (i < nslots) stage_slot(i, ring + i * slotb);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    int y = ya, slot = 0;
    for (int u = 0; u < nslots; ++u) {
        const int sa = slot == 0 ? nbuf - 1 : slot - 1;        // the slot read one round ago
        if (u + nbuf - 1 < nslots) stage_slot(u + nbuf - 1, ring + sa * slotb);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        if ((int)threadIdx.x < K && K * u + (int)threadIdx.x < nrows) {
            // source row j: it starts in output row y = max(ya, floor(j h / H)), which it
            // completes when (j + 1) h >= (y + 1) H; it reaches into y + 1 past that
            const int r = threadIdx.x, j = j_lo + K * u + r;
            const u64 j0 = (u64)j * h, j1 = j0 + h;
            const u64 yr = max((u64)ya, j0 / H), y0 = yr * H, y1 = y0 + H;
            int4 e;
            e.x = (int)(min(y1, j1) - max(y0, j0));
            e.y = (j1 > y1 && (int)yr + 1 < yb) ? (int)(j1 - y1) : 0;
            e.z = j1 >= y1;
            e.w = (slot * slotb) + r * p.segrow + (int)((uintptr_t)row_of(j) & 15);
            s_row[r] = e;
        }
        // this slot's copies are done (later slots' may still be in flight)
        if (nbuf >= 4)
            asm volatile("cp.async.wait_group 3;\n" ::: "memory");
        else if (nbuf == 3)
            asm volatile("cp.async.wait_group 2;\n" ::: "memory");
        else
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        __syncthreads();
        slot = slot + 1 == nbuf ? 0 : slot + 1;
        const int kr = min(K, nrows - K * u);
        for (int r = 0; r < kr; ++r) {
            const int4 e = s_row[r];
            const int s0 = e.w;                                 // staged byte 0 of the row
            const unsigned wy = (unsigned)e.x, wn = (unsigned)e.y;   // units of 1/h
#pragma unroll
            for (int m = 0; m < NCOL; ++m) {
                if (nt[m] == 0) continue;
                const int a = s0 + off[m];
                const uint8_t *q = ring + a;
                if (C == 3) {
                    unsigned hs[3];
                    if (nt[m] == 1) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) hs[c] = af[m] * q[c];
                    } else {
                        unsigned S[3] = {0u, 0u, 0u};
                        const int last = 3 * (nt[m] - 1);
                        if (nt[m] > 4) {
                            interior3(ring, a + 3, a + last, S);
                        } else {
                            for (int i = 3; i < last; i += 3) {
                                S[0] += q[i];
                                S[1] += q[i + 1];
                                S[2] += q[i + 2];
                            }
                        }
#pragma unroll
                        for (int c = 0; c < 3; ++c) hs[c] = af[m] * q[c] + al[m] * q[last + c] + (unsigned)w * S[c];
                    }
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        cur[c] += (Acc)wy * hs[c];
                        nxt[c] += (Acc)wn * hs[c];
                    }
                } else {
                    unsigned hs;
                    if (nt[m] == 1) {
                        hs = af[m] * q[0];
                    } else {
                        unsigned m0 = 0, m1 = 0;   // interior taps, two independent sums
                        int i = 1;
                        for (; i + 1 < nt[m] - 1; i += 2) {
                            m0 += q[i];
                            m1 += q[i + 1];
                        }
                        if (i < nt[m] - 1) m0 += q[i];
                        hs = af[m] * q[0] + al[m] * q[nt[m] - 1] + (unsigned)w * (m0 + m1);
                    }
                    cur[m] += (Acc)wy * hs;
                    nxt[m] += (Acc)wn * hs;
                }
            }
            if (e.z) {   // output row y is complete (the last source row ends at H h)
                uint8_t *row = p.dst + (int64_t)blockIdx.z * p.dbatch + (int64_t)y * p.dpitch;
                const u64 wh = W * H;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const int m = C == 3 ? 0 : k;
                    if (nt[m] != 0) {
                        const int x = xs + threadIdx.x + (C == 3 ? 0 : kThreads * k), c = C == 3 ? k : 0;
                        if (!p.f32) {
                            // floor((2 S + W H) / (2 W H)) in [0, 255]: a float estimate is within
                            // one of the quotient; one step each way makes it exact
                            unsigned qv;
                            if (!WIDE && p.fin32) {
                                // 512 W H < 2^32: every product below fits 32 bits
                                const unsigned num = 2u * (unsigned)cur[k] + (unsigned)wh, den = 2u * (unsigned)wh;
                                qv = (unsigned)__fmul_rz(__uint2float_rn(num), p.inv_2wh);
                                const unsigned t = qv * den;
                                if (t > num) --qv;
                                else if (t + den <= num) ++qv;
                            } else {
                                const u64 num = 2ull * (u64)cur[k] + wh, den = 2ull * wh;
                                qv = (unsigned)__fmul_rz((float)num, p.inv_2wh);
                                if ((u64)qv * den > num) --qv;
                                else if ((u64)(qv + 1) * den <= num) ++qv;
                            }
                            row[x * C + c] = (uint8_t)qv;
                        } else {
                            const float mv = __fmul_rn((float)cur[k], p.inv_wh);   // mean in [0, 255]
                            const float o = __fmaf_rn(mv, p.scale[c], p.bias[c]);
                            if (p.chw)
                                reinterpret_cast<float *>(row + (int64_t)c * p.dplane)[x] = o;
                            else
                                reinterpret_cast<float *>(row)[x * C + c] = o;
                        }
                    }
                    cur[k] = nxt[k];
                    nxt[k] = 0;
                }
                ++y;
            }
        }
        __syncthreads();   // the slot is read before later rows are staged into it
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
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
    // strip width: at most 768 / C output columns, halved until two ring slots fit; a slot
    // holds the strip's source columns (at most ceil(nx W / w) + 1) and the 16-byte phase
    auto seg_of = [&](long long nx) { return ((((nx * d.W + d.w - 1) / d.w + 1) * d.C + 15) + 15) & ~15LL; };
    long long nx = std::min<long long>(d.w, kStripValues / d.C);
    while (nx > 1 && 2 * seg_of(nx) > (long long)kAreaSmemCap) nx = (nx + 1) / 2;
    const long long segrow = seg_of(nx);
    too_large = 2 * segrow > (long long)kAreaSmemCap;
    if (too_large) return cudaSuccess;
    // rows per slot: about 8 KB of source per slot, so that a CTA keeps tens of KB in flight
    const long long K = std::max(1LL, std::min(16LL, 8192 / segrow));
    int nbuf = 4;
    while (nbuf > 2 && nbuf * K * segrow > 48 * 1024) --nbuf;
    p.nx = (int)nx;
    p.segrow = (int)segrow;
    p.K = (int)K;
    p.nbuf = nbuf;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long strips = (d.w + nx - 1) / nx;
    // bands of R output rows: about eight CTAs per SM in all, R <= 32 (a band re-reads at
    // most one source row of its neighbour)
    p.R = (int)std::max(1LL, std::min(32LL, strips * d.h * d.batch / (8LL * std::max(1, sms))));
    const size_t smem = (size_t)nbuf * (size_t)(K * segrow);
    const bool wide = 255.0 * (double)d.W * (double)d.H >= 4294967296.0;
    p.fin32 = 512.0 * (double)d.W * (double)d.H < 4294967296.0;
    const void *k = d.C == 3 ? (wide ? (const void *)area_kernel<true, 3> : (const void *)area_kernel<false, 3>)
                             : (wide ? (const void *)area_kernel<true, 1> : (const void *)area_kernel<false, 1>);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAreaSmemCap);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)strips, (unsigned)((d.h + p.R - 1) / p.R), (unsigned)d.batch);
    void *args[] = {&p};
    e = cudaLaunchKernel(k, grid, dim3(kThreads), args, smem, stream);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace kr
