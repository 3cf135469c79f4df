// Device-side tile engine of the resampling kernels (sm_103a): bilinear resize and the
// affine and perspective warps of Sec. III / Sec. II-A, with the fused gray and u8 -> f32
// normalisation epilogues of Sec. III.
//
// One CTA of kThreads threads produces one TW x TH tile of output pixels:
//   1. plan: the source box of the tile (the bounding box of every tap, from the resize
//      axis tables or from the warp map at the tile corners) and a per-tile "fast" flag;
//   2. stage: the box's source rows are copied into shared memory by one 3-D TMA copy (a
//      {word, row, image} tensor map; the part of a warp box outside the image arrives as
//      zeros, the zero border), else by one bulk copy per row, else as 16-byte cp.async
//      chunks; the copies complete on an mbarrier with a bounded wait. TMA- and bulk-staged
//      rows share one 16-byte phase, so 3-channel tap pairs are read straight from them
//      ("raw taps"); cp.async-staged 3-channel rows are re-laid as one word per pixel. With
//      the replicated border a box crossing the image's edge is clipped to the image and
//      its taps are clamped into it;
//   3. compute: fast tiles (every tap inside the box, coordinates in the range where the
//      packed one-fma weight forms are exact) run a branch-free pixel loop; other tiles
//      (coordinates outside that range, boxes too large for shared memory, non-finite or
//      huge coordinates) take the medium or general per-pixel paths;
//   4. write-out: when the destination rows are whole 16-byte chunks at 16-byte aligned
//      addresses (Job::direct) the pixels go straight from registers to global memory; else
//      into a shared copy of the output tile (two bands of rows for f32) that leaves through
//      128-bit coalesced stores (head and tail bytes one per lane).
//
// Arithmetic (definitions shared with the C ABI documentation):
//   resize   sx = (x + 1/2) W / w - 1/2 as the exact rational num/den, clamp to
//            the edge; 11-bit weight of the second tap rounded half up;
//   warp     sx = fmaf(m00, x + 1/2, fmaf(m01, y + 1/2, m02)) - 1/2 in fp32,
//            taps floor(sx), floor(sx) + 1, zero outside the image, 11-bit
//            weight = round-half-up of 2048 * (sx - floor(sx));
//   u8       out = (v + 2^21) >> 22, v = sum of tap * wx * wy (exact integers);
//   f32      p/255 blended with fp32 weights, then * scale[c] + bias[c];
//   gray     (4899 R + 9617 G + 1868 B + 8192) >> 14 (u8), 0.299/0.587/0.114 (f32).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace kr {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

enum { OP_RESIZE = 0, OP_WARP = 1, OP_PERSP = 2 };
enum { OUT_U8 = 0, OUT_U8_GRAY = 1, OUT_F32 = 2, OUT_F32_GRAY = 3 };

// One image of one resampling operation, pointers already at that image.
struct Job {
    const uint8_t *src;
    int64_t spitch;
    int32_t H, W;
    uint8_t *dst;
    int64_t dpitch;
    int64_t dplane;       // CHW plane stride in bytes
    int32_t h, w;
    int32_t chw;          // f32 planar destination
    int32_t foot_budget;  // shared bytes of region A (staged box); 0 = never stage
    int32_t region_b;     // shared bytes of region B (raw rows of 3-channel boxes, then output tile)
    int32_t allow_fast;   // warp: the map's intermediate terms are small enough for the fast path
    int32_t raw_taps;     // region A is sized for raw boxes: 3-channel tiles staged by TMA or by
                          // bulk row copies read their taps from the raw rows, not re-laid words
    int32_t rows16;       // source base and pitch are 16-byte aligned (bulk row copies possible)
    int32_t replicate;    // warps: taps outside the image read the nearest edge pixel (else zero)
    // TMA source map (per-operation kernels; null in the ragged kernel): the images as
    // {32-bit word, row, image} tensors whose rows are a whole number of words.
    const CUtensorMap *tin;   // box {4 tin_nc words, tin_br rows, 1}; null = cp.async staging
    int32_t tin_nc, tin_br;   // box row in 16-byte chunks, box rows
    int32_t direct;           // destination rows are whole 16-byte chunks at 16-byte aligned
                              // addresses: tiles are written straight from registers
    int32_t zimg;             // image coordinate of this job in both maps
    unsigned *err;            // device error flags (bit 0: a bounded TMA wait ran out)
    uint64_t wait_ns;         // bound of the first wait for a staged box (0: give up at once)
    uint32_t rm[4];           // resize: floor((2^32-1)/d) for d = 2w, 4w, 2h, 4h (0: divide)
    float M[9];           // destination -> source map (warp: 2x3; perspective: 3x3), row-major
    float scale[3];       // f32: out = v255 * scale[c] + bias[c]
    float bias[3];
};

__host__ __device__ constexpr int round16(int x) { return (x + 15) & ~15; }
__host__ __device__ constexpr int round4(int x) { return (x + 3) & ~3; }

// Bytes per output element and channels of the destination.
template <int OUTK, int CIN> struct OutTraits {
    static constexpr int esize = (OUTK == OUT_F32 || OUTK == OUT_F32_GRAY) ? 4 : 1;
    static constexpr int dC = (OUTK == OUT_U8_GRAY || OUTK == OUT_F32_GRAY) ? 1 : CIN;
    static constexpr bool is_f32 = esize == 4;
};

// Output rows a tile stages at a time: f32 tiles leave in two bands of TH / 2 rows.
template <int OUTK, int CIN, int TH>
__host__ __device__ constexpr int out_band_rows()
{
    return OutTraits<OUTK, CIN>::is_f32 ? TH / 2 : TH;
}

// Shared bytes of the output staging buffer of a TW x TH tile: f32 tiles are
// sized for three planar rows of TW floats (which also covers one HWC row of
// 3*TW floats) per band row; u8 tiles hold TH rows of TW*dC bytes. Every row
// gets 15 bytes of room for its 16-byte phase.
template <int OUTK, int CIN, int TW, int TH>
__host__ __device__ constexpr int out_stage_bytes()
{
    return OutTraits<OUTK, CIN>::is_f32
               ? OutTraits<OUTK, CIN>::dC * out_band_rows<OUTK, CIN, TH>() * round16(TW * 4 + 15)
               : TH * round16(TW * OutTraits<OUTK, CIN>::dC + 15);
}

// Staged-box geometry of a box `cols` source pixels wide.
//   raw row:  the row's bytes as whole 16-byte chunks, with room for the 16-byte
//             phase and for the last 4-pixel group of the re-layout;
//   word row: one 32-bit word per pixel plus one spare, a multiple of 4 words.
__host__ __device__ constexpr int raw_row_bytes(int cols, int cin)
{
    return cin == 3 ? round16(15 + 12 * ((cols + 3) / 4) + 4) : round16(cols + 15 + 2);
}
__host__ __device__ constexpr int word_row(int cols) { return round4(cols + 1); }

// ---------------------------------------------------------------------------
// Coordinate maps
// ---------------------------------------------------------------------------

// Resize along one axis: sx = (i + 1/2) n_in / n_out - 1/2 = num / den exactly.
// i0/i1 taps, q = 11-bit weight of i1 rounded half up, f = fp32 weight of i1.
// 32-bit division when both sizes are below 2^15 (num < 2^31), else 64-bit.
__device__ __forceinline__ void resize_axis(int i, int n_in, int n_out, int &i0, int &i1, int &q,
                                            float &f)
{
    if (n_in < 32768 && n_out < 32768) {
        const int num = (2 * i + 1) * n_in - n_out;
        const unsigned den = 2u * (unsigned)n_out;
        if (num <= 0) {
            i0 = 0; q = 0; f = 0.f;
        } else {
            const unsigned k = (unsigned)num / den;
            const unsigned r = (unsigned)num - k * den;
            if ((int)k >= n_in - 1) {
                i0 = n_in - 1; q = 0; f = 0.f;
            } else {
                i0 = (int)k;
                q = (int)((4096u * r + den) / (2u * den));
                f = __fdiv_rn((float)r, (float)den);
            }
        }
    } else {
        const long long num = (2LL * i + 1) * (long long)n_in - (long long)n_out;
        const long long den = 2LL * (long long)n_out;
        if (num <= 0) {
            i0 = 0; q = 0; f = 0.f;
        } else {
            const long long k = num / den;
            const long long r = num - k * den;
            if (k >= n_in - 1) {
                i0 = n_in - 1; q = 0; f = 0.f;
            } else {
                i0 = (int)k;
                q = (int)((4096LL * r + den) / (2LL * den));
                f = __fdiv_rn((float)r, (float)den);
            }
        }
    }
    i1 = min(i0 + 1, n_in - 1);
}

// resize_axis for sizes below 2^15 with the divisions by den = 2 n_out and by 2 den done as a
// multiply-high by mden = floor((2^32 - 1) / den) (m2den for 2 den) and one correction step:
// for num < 2^32 the estimate floor(num mden / 2^32) is the quotient or one less.
__device__ __forceinline__ void resize_axis_m(int i, int n_in, int n_out, uint32_t mden, uint32_t m2den, int &i0,
                                              int &i1, int &q, float &f)
{
    const int num = (2 * i + 1) * n_in - n_out;
    const uint32_t den = 2u * (uint32_t)n_out;
    if (num <= 0) {
        i0 = 0; q = 0; f = 0.f;
    } else {
        uint32_t k = __umulhi((uint32_t)num, mden);
        uint32_t r = (uint32_t)num - k * den;
        if (r >= den) { ++k; r -= den; }
        if ((int)k >= n_in - 1) {
            i0 = n_in - 1; q = 0; f = 0.f;
        } else {
            i0 = (int)k;
            const uint32_t n2 = 4096u * r + den, d2 = 2u * den;
            uint32_t qq = __umulhi(n2, m2den);
            if (n2 - qq * d2 >= d2) ++qq;
            q = (int)qq;
            f = __fdiv_rn((float)r, (float)den);
        }
    }
    i1 = min(i0 + 1, n_in - 1);
}

// Warp coordinate: the fixed fp32 sequence, no contraction beyond the explicit fmas.
__device__ __forceinline__ bool warp_coord(const float *M, int x, int y, float &sx, float &sy)
{
    const float xc = __fadd_rn((float)x, 0.5f);
    const float yc = __fadd_rn((float)y, 0.5f);
    sx = __fsub_rn(__fmaf_rn(M[0], xc, __fmaf_rn(M[1], yc, M[2])), 0.5f);
    sy = __fsub_rn(__fmaf_rn(M[3], xc, __fmaf_rn(M[4], yc, M[5])), 0.5f);
    return fabsf(sx) < 4194304.f && fabsf(sy) < 4194304.f;
}

// Perspective coordinate: homogeneous X, Y, Z by fp32 fmas, q = 1/Z (rounded), s = X q - 1/2.
// No source (false) where Z <= 0, or beyond |s| < 2^22. With the last row (0, 0, 1) this is
// warp_coord bit for bit.
__device__ __forceinline__ bool persp_coord(const float *M, int x, int y, float &sx, float &sy)
{
    const float xc = __fadd_rn((float)x, 0.5f);
    const float yc = __fadd_rn((float)y, 0.5f);
    const float X = __fmaf_rn(M[0], xc, __fmaf_rn(M[1], yc, M[2]));
    const float Y = __fmaf_rn(M[3], xc, __fmaf_rn(M[4], yc, M[5]));
    const float Z = __fmaf_rn(M[6], xc, __fmaf_rn(M[7], yc, M[8]));
    if (!(Z > 0.f)) {
        sx = sy = 0.f;
        return false;
    }
    const float q = __frcp_rn(Z);
    sx = __fsub_rn(__fmul_rn(X, q), 0.5f);
    sy = __fsub_rn(__fmul_rn(Y, q), 0.5f);
    return fabsf(sx) < 4194304.f && fabsf(sy) < 4194304.f;
}

template <int OP> __device__ __forceinline__ bool map_coord(const float *M, int x, int y, float &sx, float &sy)
{
    return OP == OP_PERSP ? persp_coord(M, x, y, sx, sy) : warp_coord(M, x, y, sx, sy);
}

// floor and 11-bit weight (round half up of 2048 * frac, frac = s - floor(s) in fp32).
__device__ __forceinline__ void warp_weight(float s, int &i0, int &q)
{
    const float fl = floorf(s);
    i0 = (int)fl;
    const float t = __fmul_rn(__fsub_rn(s, fl), 2048.f);
    const float k = floorf(t);
    q = (int)k + (__fsub_rn(t, k) >= 0.5f ? 1 : 0);
}

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(void *sdst, const void *gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(sdst)), "l"(gsrc)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// ---------------------------------------------------------------------------
// TMA and mbarrier helpers (sm_90+ PTX, used here on sm_103a)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t *mbar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n"
                 "fence.mbarrier_init.release.cluster;\n" ::"r"(smem_addr(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(mbar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, uint32_t parity)
{
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done)
                 : "r"(smem_addr(mbar)), "r"(parity)
                 : "memory");
    return done != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the mbarrier phase `parity`, giving up after `limit_ns` nanoseconds.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *mbar, uint32_t parity, uint64_t limit_ns)
{
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(mbar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

// 3-D tensor load {x, y, image} of the map's box into shared memory, completing on mbar.
__device__ __forceinline__ void tma_load_3d(void *sdst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint64_t *mbar)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_addr(sdst)),
                 "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(mbar))
                 : "memory");
}

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned) from global to
// shared memory, completing on mbar.
__device__ __forceinline__ void bulk_load(void *sdst, const void *gsrc, uint32_t bytes, uint64_t *mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_addr(sdst)),
                 "l"(reinterpret_cast<uint64_t>(gsrc)), "r"(bytes), "r"(smem_addr(mbar))
                 : "memory");
}

// Make this thread's generic-proxy shared-memory writes visible to the TMA (async proxy).
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// Bound of every TMA wait: far above any copy's latency, far below a hang.
constexpr uint64_t kTmaWaitNs = 2000000000ull;

// One RGB pixel from global memory as a word R | G << 8 | B << 16 (outside the image: zero,
// or with `rep` the nearest edge pixel).
__device__ __forceinline__ uint32_t ldg_px3(const uint8_t *src, int64_t spitch, int H, int W, int y,
                                            int x, bool rep = false)
{
    if (rep) {
        x = min(max(x, 0), W - 1);
        y = min(max(y, 0), H - 1);
    }
    if ((unsigned)x >= (unsigned)W || (unsigned)y >= (unsigned)H) return 0u;
    const uint8_t *p = src + (int64_t)y * spitch + (int64_t)x * 3;
    return (uint32_t)__ldg(p) | ((uint32_t)__ldg(p + 1) << 8) | ((uint32_t)__ldg(p + 2) << 16);
}

__device__ __forceinline__ uint32_t ldg_px1(const uint8_t *src, int64_t spitch, int H, int W, int y,
                                            int x, bool rep = false)
{
    if (rep) {
        x = min(max(x, 0), W - 1);
        y = min(max(y, 0), H - 1);
    }
    if ((unsigned)x >= (unsigned)W || (unsigned)y >= (unsigned)H) return 0u;
    return (uint32_t)__ldg(src + (int64_t)y * spitch + x);
}

// Exact float of byte k of w (0..255): 2^23 + b has b in its low mantissa bits.
__device__ __forceinline__ float byte_f(uint32_t w, int k)
{
    const uint32_t sel = 0x7540u | (uint32_t)k;
    return __fsub_rn(__uint_as_float(__byte_perm(w, 0x4B000000u, sel)), 8388608.f);
}

// Two fp32 lanes in one 64-bit register pair (sm_100+ packed f32x2 arithmetic).
struct F2 {
    unsigned long long v;
};
__device__ __forceinline__ F2 f2_pack(float lo, float hi)
{
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ F2 f2_pack_bits(uint32_t lo, uint32_t hi)
{
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "r"(lo), "r"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(F2 a, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b)
{
    F2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 f2_sub(F2 a, F2 b)
{
    F2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b)
{
    F2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 f2_fma(F2 a, F2 b, F2 c)
{
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}

__device__ __forceinline__ void f2_unpack_bits(F2 a, uint32_t &lo, uint32_t &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(a.v));
}
// Rounded toward minus infinity, lane by lane.
__device__ __forceinline__ F2 f2_fma_rm(F2 a, F2 b, F2 c)
{
    F2 r;
    asm("fma.rm.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
__device__ __forceinline__ F2 f2_add_rm(F2 a, F2 b)
{
    F2 r;
    asm("add.rm.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}


// Packed 11-bit weight pair for dp2a: low half 2048 - q, high half q.
__device__ __forceinline__ uint32_t wpair(int q) { return 2048u + (uint32_t)q * 65535u; }

// Horizontal u8 blend of two RGB pixel words a, b (R | G<<8 | B<<16) with weight pair w.
struct U8x3 { uint32_t r, g, b; };

__device__ __forceinline__ U8x3 hblend_px(uint32_t a, uint32_t b, uint32_t w)
{
    const uint32_t rg = __byte_perm(a, b, 0x5140);   // Ra Rb Ga Gb
    const uint32_t bb = __byte_perm(a, b, 0x0062);   // Ba Bb
    U8x3 o;
    o.r = __dp2a_lo(w, rg, 0u);
    o.g = __dp2a_hi(w, rg, 0u);
    o.b = __dp2a_lo(w, bb, 0u);
    return o;
}

__device__ __forceinline__ uint32_t vblend(uint32_t top, uint32_t bot, int qy)
{
    return (top * (uint32_t)(2048 - qy) + bot * (uint32_t)qy + (1u << 21)) >> 22;
}

__device__ __forceinline__ uint32_t gray_u8(uint32_t r, uint32_t g, uint32_t b)
{
    return (4899u * r + 9617u * g + 1868u * b + 8192u) >> 14;
}

// ---------------------------------------------------------------------------
// Shared tile state
// ---------------------------------------------------------------------------
struct TileInfo {
    int fx0, fx1, fy0, fy1;   // staged source box (inclusive)
    int srow;                 // raw bytes per staged row
    int sw;                   // words per row of the re-laid 3-channel box
    int staged;               // the box is in shared memory
    int fast;                 // every tap of the tile is inside the box (and, for warp,
                              // every coordinate lies in [0, 4094))
    int tma_ok;               // the TMA copy of the box completed
    int zero;                 // warp: the box misses the image, every sample is 0
    int clamp;                // warp, replicated border: the box was clipped to the image and
                              // every tap is clamped into it
};

// The staging decision of a tile.
enum { TD_ZERO = 1, TD_STAGED = 2, TD_RAWBOX = 4, TD_FAST = 8, TD_TMA = 16, TD_BULK = 32 };
struct TileDec {
    int rows, cols;   // box size
    int srow, sw;     // raw bytes / words per row of the re-laid layout
    int bnc;          // 16-byte chunks of a bulk-copied box row
    int rstride;      // bytes between staged raw rows
    int flags;        // TD_*
};

template <int TW, int TH> struct TileShared {
    uint64_t mbar;         // completion barrier of the box's copies (one phase per staged tile)
    uint32_t mbar_phase;   // parity of the barrier's next phase
    int32_t mbar_ok;       // 0 after a wait ran out twice: the barrier is not used again
    TileInfo ti;
    int cx0[TW];     // column tap x0
    int cqd[TW];     // q | (x1 - x0) << 16
    float cf[TW];    // fp32 weight of x1
    int ry0[TH];
    int rqd[TH];
    float rf[TH];
};

// Once per CTA, before its first tile (the tile's first barrier publishes it).
template <int TW, int TH> __device__ __forceinline__ void tile_shared_init(TileShared<TW, TH> &ts)
{
    if (threadIdx.x == 0) {
        mbar_init(&ts.mbar);
        ts.mbar_phase = 0;
        ts.mbar_ok = 1;
    }
}

// One thread waits (bounded by first_ns; 0 gives up at once) for the current phase of the
// staging barrier and records the outcome in ti.tma_ok. A wait that runs out sets error bit 0
// and waits once more (bounded by kTmaWaitNs) for the copies to land before the tile is
// abandoned; if that runs out too the barrier is retired.
template <int TW, int TH>
__device__ __forceinline__ void stage_wait(TileShared<TW, TH> &ts, unsigned *err, uint64_t first_ns)
{
    const uint32_t ph = ts.mbar_phase;
    bool ok = first_ns != 0 && mbar_wait_bounded(&ts.mbar, ph, first_ns);
    ts.ti.tma_ok = ok ? 1 : 0;
    if (!ok) {
        atomicOr(err, 1u);
        ok = mbar_wait_bounded(&ts.mbar, ph, kTmaWaitNs);
    }
    if (ok) ts.mbar_phase = ph ^ 1u;
    else ts.mbar_ok = 0;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Where one output row of the tile goes in the shared output copy: the HWC row,
// or the three CHW plane rows (each keeping the 16-byte phase of its global row).
struct ORow {
    uint8_t *p0, *p1, *p2;
};

// Tap formats of a 3-channel pixel pair (x0, x0 + 1) of one source row:
//   TAPS_WORDS  p0 = R0 | G0<<8 | B0<<16, p1 = R1 | G1<<8 | B1<<16 (re-laid box);
//   TAPS_RAW    p0 = R0 | G0<<8 | B0<<16 | R1<<24, p1 = G1 | B1<<8 | .. (the six bytes
//               of the pair as they lie in a raw row, shifted down to byte 0).
enum { TAPS_WORDS = 0, TAPS_RAW = 1 };
template <int V> struct IntC {
    static constexpr int value = V;
};

// Raw pair at byte offset `off` of a staged box: three aligned words, two funnel shifts
// (which use the low five bits of the shift, so off * 8 needs no mask).
__device__ __forceinline__ void raw_pair(const uint8_t *wp, uint32_t sh, uint32_t &p0, uint32_t &p1)
{
    const uint32_t *w = reinterpret_cast<const uint32_t *>(wp);
    const uint32_t t0 = w[0], t1 = w[1], t2 = w[2];
    p0 = __funnelshift_r(t0, t1, sh);
    p1 = __funnelshift_r(t1, t2, sh);
}

// Horizontal u8 blend of the pair (p0, p1) in tap format F with weight pair w.
template <int F>
__device__ __forceinline__ U8x3 hblend_pair(uint32_t p0, uint32_t p1, uint32_t w)
{
    if (F == TAPS_WORDS) return hblend_px(p0, p1, w);
    const uint32_t rg = __byte_perm(p0, p1, 0x4130);   // R0 R1 G0 G1
    const uint32_t bb = __byte_perm(p0, p1, 0x0052);   // B0 B1
    U8x3 o;
    o.r = __dp2a_lo(w, rg, 0u);
    o.g = __dp2a_hi(w, rg, 0u);
    o.b = __dp2a_lo(w, bb, 0u);
    return o;
}


// The same taps as 2^23 + byte, not yet unbiased (exact floats; differences are exact).
__device__ __forceinline__ F2 rg_biased(uint32_t w)
{
    return f2_pack_bits(__byte_perm(w, 0x4B000000u, 0x7540), __byte_perm(w, 0x4B000000u, 0x7541));
}
template <int F> __device__ __forceinline__ F2 rg1_biased(uint32_t p0, uint32_t p1)
{
    if (F == TAPS_WORDS) return rg_biased(p1);
    return f2_pack_bits(__byte_perm(p0, 0x4B000000u, 0x7543), __byte_perm(p1, 0x4B000000u, 0x7540));
}
template <int F> __device__ __forceinline__ uint32_t b1_biased(uint32_t p1)
{
    return __byte_perm(p1, 0x4B000000u, F == TAPS_WORDS ? 0x7542 : 0x7541);
}

// ---------------------------------------------------------------------------
// Per-pixel output: blend the taps and put the result into the output tile.
// Taps are pixel pairs (p00, p01) of the top row and (p10, p11) of the bottom row in
// tap format F (3 channels), or single pixels in byte 0 (1 channel).
// ---------------------------------------------------------------------------
template <int CIN, int OUTK, int F = TAPS_WORDS>
__device__ __forceinline__ void emit(const Job &J, const ORow &o, int c, uint32_t p00, uint32_t p01,
                                     uint32_t p10, uint32_t p11, int qx, int qy, float fx, float fy)
{
    using OT = OutTraits<OUTK, CIN>;
    if (!OT::is_f32) {
        uint8_t *op = o.p0 + c * OT::dC;
        const uint32_t w = wpair(qx);
        if (CIN == 3) {
            const U8x3 a = hblend_pair<F>(p00, p01, w), b = hblend_pair<F>(p10, p11, w);
            const uint32_t r = vblend(a.r, b.r, qy), g = vblend(a.g, b.g, qy), bl = vblend(a.b, b.b, qy);
            if (OUTK == OUT_U8_GRAY) {
                op[0] = (uint8_t)gray_u8(r, g, bl);
            } else {
                op[0] = (uint8_t)r;
                op[1] = (uint8_t)g;
                op[2] = (uint8_t)bl;
            }
        } else {
            const uint32_t t = __dp2a_lo(w, __byte_perm(p00, p01, 0x0040), 0u);
            const uint32_t b = __dp2a_lo(w, __byte_perm(p10, p11, 0x0040), 0u);
            op[0] = (uint8_t)vblend(t, b, qy);
        }
    } else {
        float v[3];
        if (CIN == 3) {
            // Lerp along x on both rows, then along y: R and G of a row in one packed f32x2
            // pair, B alone. Taps are read as 2^23 + byte (exact); the
            // difference of two such taps is the difference of the bytes, and only the base
            // of each lerp is unbiased: fma(f, b - a, a) with the same operands as on bytes.
            const F2 K = f2_pack(8388608.f, 8388608.f);
            const F2 fx2 = f2_pack(fx, fx), fy2 = f2_pack(fy, fy);
            const F2 a = rg_biased(p00), b = rg1_biased<F>(p00, p01);
            const F2 cc = rg_biased(p10), d = rg1_biased<F>(p10, p11);
            const F2 h0 = f2_fma(fx2, f2_sub(b, a), f2_sub(a, K));
            const F2 h1 = f2_fma(fx2, f2_sub(d, cc), f2_sub(cc, K));
            f2_unpack(f2_fma(fy2, f2_sub(h1, h0), h0), v[0], v[1]);
            const float kb = 8388608.f;
            const float ba = __uint_as_float(__byte_perm(p00, 0x4B000000u, 0x7542));
            const float bb = __uint_as_float(b1_biased<F>(p01));
            const float bc = __uint_as_float(__byte_perm(p10, 0x4B000000u, 0x7542));
            const float bd = __uint_as_float(b1_biased<F>(p11));
            const float g0 = __fmaf_rn(fx, __fsub_rn(bb, ba), __fsub_rn(ba, kb));
            const float g1 = __fmaf_rn(fx, __fsub_rn(bd, bc), __fsub_rn(bc, kb));
            v[2] = __fmaf_rn(fy, __fsub_rn(g1, g0), g0);
        } else {
            const float a = byte_f(p00, 0), b = byte_f(p01, 0);
            const float cc = byte_f(p10, 0), d = byte_f(p11, 0);
            const float h0 = __fmaf_rn(fx, __fsub_rn(b, a), a);
            const float h1 = __fmaf_rn(fx, __fsub_rn(d, cc), cc);
            v[0] = __fmaf_rn(fy, __fsub_rn(h1, h0), h0);
        }
        if (OUTK == OUT_F32_GRAY) {
            const float g = __fmaf_rn(0.299f, v[0], __fmaf_rn(0.587f, v[1], __fmul_rn(0.114f, v[2])));
            reinterpret_cast<float *>(o.p0)[c] = __fmaf_rn(g, J.scale[0], J.bias[0]);
        } else if (CIN == 3 && o.p1) {
            reinterpret_cast<float *>(o.p0)[c] = __fmaf_rn(v[0], J.scale[0], J.bias[0]);
            reinterpret_cast<float *>(o.p1)[c] = __fmaf_rn(v[1], J.scale[1], J.bias[1]);
            reinterpret_cast<float *>(o.p2)[c] = __fmaf_rn(v[2], J.scale[2], J.bias[2]);
        } else {
#pragma unroll
            for (int k = 0; k < CIN; ++k)
                reinterpret_cast<float *>(o.p0)[c * CIN + k] = __fmaf_rn(v[k], J.scale[k], J.bias[k]);
        }
    }
}

}  // namespace kr
