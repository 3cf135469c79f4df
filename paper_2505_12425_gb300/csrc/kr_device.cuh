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
//   4. write-out: results go into a shared copy of the output tile (two bands of rows for
//      f32) and leave through a TMA store per band, else through 128-bit coalesced stores
//      (head and tail bytes one per lane).
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
    // TMA (per-operation kernels; null in the ragged kernel). Both maps view images as
    // {32-bit word, row, (plane,) image} tensors whose rows are a whole number of words.
    const CUtensorMap *tin;   // source map, box {4 tin_nc words, tin_br rows, 1}; null = cp.async staging
    int32_t tin_nc, tin_br;   // box row in 16-byte chunks, box rows
    const CUtensorMap *tout;  // destination map, box = one output tile; null = 128-bit stores
    int32_t zimg;             // image coordinate of this job in both maps
    unsigned *err;            // device error flags (bit 0: a bounded TMA wait ran out)
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

__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, int c0, int c1, int c2, const void *ssrc)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];\n" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(ssrc))
                 : "memory");
}

__device__ __forceinline__ void tma_store_4d(const CUtensorMap *map, int c0, int c1, int c2, int c3, const void *ssrc)
{
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];\n" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(ssrc))
                 : "memory");
}

__device__ __forceinline__ void tma_store_commit_and_wait_read()
{
    asm volatile("cp.async.bulk.commit_group;\ncp.async.bulk.wait_group.read 0;\n" ::: "memory");
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

// One thread waits (bounded) for the current phase of the staging barrier and records the
// outcome in ti.tma_ok. A wait that runs out sets error bit 0 and waits once more for the
// copies to land before the tile is abandoned; if that runs out too the barrier is retired.
template <int TW, int TH> __device__ __forceinline__ void stage_wait(TileShared<TW, TH> &ts, unsigned *err)
{
    const uint32_t ph = ts.mbar_phase;
    bool ok = mbar_wait_bounded(&ts.mbar, ph, kTmaWaitNs);
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

// ---------------------------------------------------------------------------
// The tile engine.
// ---------------------------------------------------------------------------
// ROWS: the bulk row-copy staging is compiled in. FRESH: the CTA runs this one tile, and the
// staging barrier is initialised right before its copies; otherwise the caller ran
// tile_shared_init once and the barrier's phase carries over from tile to tile.
template <int OP, int CIN, int OUTK, int TW, int TH, bool ROWS, bool FRESH>
__device__ __forceinline__ void process_tile(const Job &J, int tile_x, int tile_y, uint8_t *smem,
                                             TileShared<TW, TH> &ts)
{
    static_assert(TW % 32 == 0 && TH % (2 * kWarps) == 0, "tile shape");
    using OT = OutTraits<OUTK, CIN>;
    constexpr int dC = OT::dC;
    constexpr int ES = OT::esize;
    constexpr int CPL = TW / 32;     // columns per lane
    TileInfo &ti = ts.ti;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx0 = tile_x * TW, ty0 = tile_y * TH;
    const int nx = min(TW, J.w - tx0), ny = min(TH, J.h - ty0);

    // ---- 1. plan -----------------------------------------------------------------
    if (OP == OP_RESIZE) {
        static_assert(TW + TH <= kThreads, "one axis entry per thread");
        if (tid < TW) {
            int i0 = 0, i1 = 0, q = 0;
            float f = 0.f;
            if (tid < nx) resize_axis(tx0 + tid, J.W, J.w, i0, i1, q, f);
            ts.cx0[tid] = i0; ts.cqd[tid] = q | ((i1 - i0) << 16); ts.cf[tid] = f;
        } else if (tid < TW + TH) {
            const int r = tid - TW;
            int i0 = 0, i1 = 0, q = 0;
            float f = 0.f;
            if (r < ny) resize_axis(ty0 + r, J.H, J.h, i0, i1, q, f);
            ts.ry0[r] = i0; ts.rqd[r] = q | ((i1 - i0) << 16); ts.rf[r] = f;
        }
        __syncthreads();
        if (tid == 0) {
            ti.fx0 = ts.cx0[0];
            ti.fx1 = ts.cx0[nx - 1] + (ts.cqd[nx - 1] >> 16);
            ti.fy0 = ts.ry0[0];
            ti.fy1 = ts.ry0[ny - 1] + (ts.rqd[ny - 1] >> 16);
        }
    } else if (warp == 0) {
        // Lanes 0..3 map one tile corner each; the box is their hull, one pixel wider
        // on the low side and three on the high side (floor, second tap, the fast form's
        // (x0 + 1, x0 + 2) pair, fp32 rounding of interior pixels).
        const int cx = (lane & 1) ? tx0 + nx - 1 : tx0, cy = (lane & 2) ? ty0 + ny - 1 : ty0;
        float sx = 0.f, sy = 0.f;
        bool ok = true;
        // (perspective: Z is affine in the pixel position, so Z > 0 at the four corners means
        // Z > 0 over the tile, and the tile maps onto the convex hull of its corners' images)
        if (lane < 4) ok = map_coord<OP>(J.M, cx, cy, sx, sy) && fabsf(sx) < 1048576.f && fabsf(sy) < 1048576.f;
        float mnx = lane < 4 ? sx : 3.0e38f, mxx = lane < 4 ? sx : -3.0e38f;
        float mny = lane < 4 ? sy : 3.0e38f, mxy = lane < 4 ? sy : -3.0e38f;
#pragma unroll
        for (int o = 1; o < 4; o <<= 1) {
            mnx = fminf(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
            mxx = fmaxf(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
            mny = fminf(mny, __shfl_xor_sync(0xffffffffu, mny, o));
            mxy = fmaxf(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
        }
        const bool all_ok = __all_sync(0xffffffffu, ok);
        if (lane == 0) {
            // The box is NOT clipped to the image: staging fills its part outside the
            // image with zeros, which is the zero border, so every tap reads the box.
            int fx0 = 0, fx1 = -1, fy0 = 0, fy1 = -1, fast = 0, zero = 0, clamp = 0;
            if (all_ok) {
                fx0 = (int)floorf(mnx) - 1; fx1 = (int)floorf(mxx) + 3;
                fy0 = (int)floorf(mny) - 1; fy1 = (int)floorf(mxy) + 3;
                // (with the replicated border no tile is all zero)
                zero = !J.replicate && (fx1 < 0 || fx0 > J.W - 1 || fy1 < 0 || fy0 > J.H - 1);
                // the one-fma weight form needs every coordinate in [0, 4094)
                fast = J.allow_fast && mnx >= 1.f && mny >= 1.f && mxx < 4093.f && mxy < 4093.f;
                if (J.replicate && (fx0 < 0 || fy0 < 0 || fx1 > J.W - 1 || fy1 > J.H - 1)) {
                    // a tap clamped to the image lies in the box clipped to the image
                    fx0 = min(max(fx0, 0), J.W - 1); fx1 = min(max(fx1, 0), J.W - 1);
                    fy0 = min(max(fy0, 0), J.H - 1); fy1 = min(max(fy1, 0), J.H - 1);
                    clamp = 1;
                    fast = 0;
                }
            }
            ti.fx0 = fx0; ti.fx1 = fx1; ti.fy0 = fy0; ti.fy1 = fy1;
            ti.fast = fast;
            ti.zero = zero;
            ti.clamp = clamp;
        }
    }
    __syncthreads();
    // Every thread derives the staging decision from the planned box (no extra barrier).
    const int fx0 = ti.fx0, fx1 = ti.fx1, fy0 = ti.fy0, fy1 = ti.fy1;
    const int rows = fy1 - fy0 + 1, cols = fx1 - fx0 + 1;
    const int srow = raw_row_bytes(max(cols, 1), CIN), sw = word_row(max(cols, 1));
    const bool zero_tile = OP != OP_RESIZE && ti.zero != 0;
    bool staged = !zero_tile && cols >= 1 && rows >= 1 && J.foot_budget > 0;
    // The staged box holds zeros outside the image: with the replicated border only boxes
    // inside the image are staged, the others take the general path.
    if (OP != OP_RESIZE && J.replicate && (fx0 < 0 || fy0 < 0 || fx1 > J.W - 1 || fy1 > J.H - 1)) staged = false;
    const int bph = (fx0 * CIN) & 15;   // 16-byte phase of the box in every row of 16-byte aligned rows
    const bool mbar_ok = FRESH || ts.mbar_ok != 0;
    // (1) one TMA copy when the launch has a source map whose box holds this tile's box
    const bool tma_fits = staged && mbar_ok && J.tin != nullptr && rows <= J.tin_br && bph + cols * CIN <= 16 * J.tin_nc;
    // (2) else one bulk copy per box row when the rows are 16-byte aligned and region A holds
    // the box (3 channels, raw taps)
    const int bnc = (bph + cols * CIN + 15) >> 4;   // 16-byte chunks of a box row
    const bool bulk_fits = ROWS && staged && mbar_ok && !tma_fits && CIN == 3 && J.raw_taps && J.rows16 &&
                           (long long)rows * 16 * bnc + 16 <= J.foot_budget;
    // Raw taps: 3-channel taps are read straight from rows staged by (1) or (2) (region A),
    // whose 16-byte phase is the same for every row.
    const bool rawbox = CIN == 3 && J.raw_taps && (tma_fits || bulk_fits);
    if (staged && !rawbox) {
        if (CIN == 3)
            staged = (long long)rows * sw * 4 <= J.foot_budget && (long long)rows * srow <= J.region_b;
        else
            staged = (long long)rows * srow + 16 <= J.foot_budget;
    }
    const bool fast = staged && (OP == OP_RESIZE || ti.fast != 0);   // resize taps always lie in the box
    const bool use_tma = staged && tma_fits;
    const bool use_bulk = staged && bulk_fits;
    const int rstride = use_tma ? 16 * J.tin_nc : use_bulk ? 16 * bnc : srow;   // bytes between staged raw rows
    uint8_t *regA = smem;
    uint8_t *regB = smem + J.foot_budget;
    uint8_t *raw = (CIN == 3 && !rawbox) ? regB : regA;
    uint8_t *ostage = regB;
    const uint32_t *words = reinterpret_cast<const uint32_t *>(regA);

    // ---- 2. stage ----------------------------------------------------------------
    if (staged) {
        // Row r of the box is [a, a + L). It is staged as whole 16-byte chunks
        // [align16(a), align16up(a + L)), clipped to the image's own byte range
        // [ibeg, iend) so that every read stays inside the described buffer; bytes
        // between rows (pitch padding) may be read but are never used. Only a chunk
        // cut by ibeg or iend (the image's first or last 16 bytes) goes byte by byte.
        // The (row, chunk) pairs are spread over the whole CTA.
        const int L = cols * CIN;
        const uint8_t *row0 = J.src + (int64_t)fy0 * J.spitch + (int64_t)fx0 * CIN;
        if (use_tma) {
            // One TMA copy of the box: rows fy0.., from the 16-byte chunk holding byte fx0*CIN
            // of each row (rows are 16-byte aligned, so every row has the same phase). Words
            // outside the image (left of it, right of its last word, above, below) arrive as
            // zeros: the zero border of warp boxes.
            if (tid == 0) {
                if (FRESH) tile_shared_init(ts);
                mbar_expect_tx(&ts.mbar, (uint32_t)(16 * J.tin_nc * J.tin_br));
                tma_load_3d(raw, J.tin, 4 * ((fx0 * CIN) >> 4), fy0, J.zimg, &ts.mbar);
                stage_wait(ts, J.err);
            }
            __syncthreads();
            if (!ti.tma_ok) return;
        } else if (use_bulk) {
            // Box row r is the row's bytes [xb0, xb1) (16-byte chunks from the one holding byte
            // fx0*3). Warp 0 copies each row's whole chunks inside the image, [0, F), with one
            // bulk copy; the other warps write what the copies do not cover: zeros outside the
            // image (the warp's zero border; resize never reads there) and the bytes of a row's
            // last partial chunk [F, 3W), byte by byte.
            const int xb0 = 16 * ((fx0 * CIN) >> 4), xb1 = xb0 + 16 * bnc;
            const int F = (J.W * CIN) & ~15;
            const int c0 = max(xb0, 0), c1 = min(xb1, F);   // copied byte range of an image row
            if (warp == 0) {
                uint32_t bytes = 0;
                if (c1 > c0)
                    for (int r = lane; r < rows; r += 32)
                        if ((unsigned)(fy0 + r) < (unsigned)J.H) bytes += (uint32_t)(c1 - c0);
                bytes = warp_sum(bytes);
                if (lane == 0) {
                    if (FRESH) tile_shared_init(ts);
                    mbar_expect_tx(&ts.mbar, bytes);
                }
                __syncwarp();
                if (c1 > c0)
                    for (int r = lane; r < rows; r += 32) {
                        const int y = fy0 + r;
                        if ((unsigned)y < (unsigned)J.H)
                            bulk_load(raw + r * rstride + (c0 - xb0), J.src + (int64_t)y * J.spitch + c0,
                                      (uint32_t)(c1 - c0), &ts.mbar);
                    }
                if (lane == 0) stage_wait(ts, J.err);
            } else if (!(fy0 >= 0 && fy1 < J.H && xb0 >= 0 && xb1 <= F)) {
                const int L3 = J.W * CIN;
                for (int r = warp - 1; r < rows; r += kWarps - 1) {
                    const int y = fy0 + r;
                    const bool yin = (unsigned)y < (unsigned)J.H;
                    const uint8_t *grow = J.src + (int64_t)y * J.spitch;
                    uint8_t *srow_p = raw + r * rstride;
                    for (int j = lane; j < bnc; j += 32) {
                        const int b0 = xb0 + 16 * j;
                        if (yin && b0 >= c0 && b0 + 16 <= c1) continue;   // copied
                        uint8_t *d = srow_p + 16 * j;
                        if (!yin || b0 + 16 <= 0 || b0 >= L3) {
                            *reinterpret_cast<uint4 *>(d) = make_uint4(0u, 0u, 0u, 0u);
                        } else {
                            for (int k = 0; k < 16; ++k) {
                                const int b = b0 + k;
                                d[k] = (b >= 0 && b < L3) ? __ldg(grow + b) : (uint8_t)0;
                            }
                        }
                    }
                }
            }
            __syncthreads();
            if (!ti.tma_ok) return;
        } else {
        const int nchr = (L + 15 + 15) >> 4;                 // chunks a row can span
        const float inv_nchr = __frcp_rn((float)nchr);
        const uintptr_t ibeg = (uintptr_t)J.src;
        const uintptr_t iend = (uintptr_t)(J.src + (int64_t)(J.H - 1) * J.spitch + (int64_t)J.W * CIN);
        for (int i = tid; i < rows * nchr; i += kThreads) {
            const int r = (int)__fmul_rz((float)i + 0.5f, inv_nchr);   // i / nchr (exact: i < 2^16)
            const int j = i - r * nchr;
            const uintptr_t a = (uintptr_t)(row0 + (int64_t)r * J.spitch);
            const uintptr_t G = a & ~(uintptr_t)15;
            const uintptr_t c0 = G + 16 * (uintptr_t)j;
            const uintptr_t e16 = (a + L + 15) & ~(uintptr_t)15;
            if (c0 >= e16) continue;
            uint8_t *dstp = raw + r * rstride + 16 * j;
            uintptr_t lo = ibeg, hi = iend;   // bytes that may be read
            if (OP != OP_RESIZE) {
                // warp boxes may cross the image border: only the row's own pixels are
                // read, everything else is the zero border
                const int yi = fy0 + r;
                if (yi < 0 || yi >= J.H) {
                    *reinterpret_cast<uint4 *>(dstp) = make_uint4(0u, 0u, 0u, 0u);
                    continue;
                }
                lo = (uintptr_t)(J.src + (int64_t)yi * J.spitch);
                hi = lo + (uintptr_t)J.W * CIN;
            }
            if (c0 >= lo && c0 + 16 <= hi) {
                cp_async16(dstp, reinterpret_cast<const void *>(c0));
            } else if (c0 + 16 <= lo || c0 >= hi) {
                *reinterpret_cast<uint4 *>(dstp) = make_uint4(0u, 0u, 0u, 0u);
            } else {
                for (int k = 0; k < 16; ++k) {
                    const uintptr_t b = c0 + k;
                    dstp[k] = (b >= lo && b < hi) ? __ldg(reinterpret_cast<const uint8_t *>(b)) : (uint8_t)0;
                }
            }
        }
        cp_async_wait_all();
        __syncthreads();
        }
        if (CIN == 3 && !rawbox) {
            // Re-lay each row as one word per pixel, 4 pixels (12 bytes) per step.
            const int gpr = (cols + 3) >> 2;
            const float inv_gpr = __frcp_rn((float)gpr);
            const uint32_t rowphase0 = (uint32_t)(uintptr_t)row0;
            const uint32_t sp = (uint32_t)J.spitch;
            for (int i = tid; i < rows * gpr; i += kThreads) {
                const int r = (int)__fmul_rz((float)i + 0.5f, inv_gpr);
                const int g = i - r * gpr;
                const int o = (int)((rowphase0 + (uint32_t)r * sp) & 15u) + 12 * g;
                const uint32_t *wp = reinterpret_cast<const uint32_t *>(raw + r * rstride + (o & ~3));
                const uint32_t sh = (uint32_t)(o & 3) * 8u;
                const uint32_t w0 = wp[0], w1 = wp[1], w2 = wp[2], w3 = wp[3];
                const uint32_t b0 = __funnelshift_r(w0, w1, sh);
                const uint32_t b1 = __funnelshift_r(w1, w2, sh);
                const uint32_t b2 = __funnelshift_r(w2, w3, sh);
                uint4 px;
                px.x = b0;                              // R0 G0 B0 (R1)
                px.y = __byte_perm(b0, b1, 0x6543);     // R1 G1 B1 (B1)
                px.z = __byte_perm(b1, b2, 0x0432);     // R2 G2 B2
                px.w = b2 >> 8;                         // R3 G3 B3
                *reinterpret_cast<uint4 *>(regA + (r * sw + 4 * g) * 4) = px;
            }
            __syncthreads();
        }
    }

    // ---- 3. compute and 4. write-out, by bands of BH rows: f32 tiles leave in two bands,
    // so that the output stage holds half a tile (more CTAs per SM).
    constexpr int BH = out_band_rows<OUTK, CIN, TH>();
    constexpr int NBAND = TH / BH;
    const bool chw = OT::is_f32 && dC == 3 && J.chw;
    const int rph = (fx0 * CIN) & 15;   // phase of every raw-staged row (raw taps)
    // output rows: dense when the tile leaves through a TMA store (its rows are 16-byte
    // aligned), else with room for each row's 16-byte phase
    const bool tma_out = J.tout != nullptr;
    const int orow = tma_out ? (chw ? TW * 4 : TW * dC * ES) : (chw ? round16(TW * 4 + 15) : round16(TW * dC * ES + 15));
    // low address bits of output row 0 of the tile (plane 0): staging rows keep their phase
    const uint32_t obase = (uint32_t)(uintptr_t)(J.dst + (int64_t)ty0 * J.dpitch +
                                                 (chw ? (int64_t)tx0 * 4 : (int64_t)tx0 * dC * ES));
    const uint32_t opitch = (uint32_t)J.dpitch, oplane = (uint32_t)J.dplane;
    int r0 = 0;   // first tile row of the current band
    auto orow_of = [&](int r) -> ORow {
        ORow o;
        const uint32_t a = obase + (uint32_t)r * opitch;
        const int sr = r - r0;
        o.p0 = ostage + sr * orow + (a & 15u);
        if (chw) {
            o.p1 = ostage + (BH + sr) * orow + ((a + oplane) & 15u);
            o.p2 = ostage + (2 * BH + sr) * orow + ((a + 2u * oplane) & 15u);
        } else {
            o.p1 = o.p2 = nullptr;
        }
        return o;
    };

    for (int band = 0; band < NBAND; ++band) {
        r0 = band * BH;
        if (r0 >= ny) break;
        const int r1 = min(ny, r0 + BH);
        if (band > 0) __syncthreads();   // the previous band has left the output stage

        if (zero_tile) {
            // every tap lies outside the image: every output pixel is the zero sample, which is
            // 0 for u8 and (0 - mean[c]) / std[c] = bias[c] (bias[0] for gray) for f32
            for (int r = r0 + warp; r < r1; r += kWarps) {
                const ORow o = orow_of(r);
#pragma unroll
                for (int j = 0; j < CPL; ++j) {
                    const int c = lane + 32 * j;
                    if (c >= nx) continue;
                    if (!OT::is_f32) {
#pragma unroll
                        for (int k = 0; k < dC; ++k) o.p0[c * dC + k] = 0;
                    } else if (chw) {
                        reinterpret_cast<float *>(o.p0)[c] = J.bias[0];
                        reinterpret_cast<float *>(o.p1)[c] = J.bias[1];
                        reinterpret_cast<float *>(o.p2)[c] = J.bias[2];
                    } else {
#pragma unroll
                        for (int k = 0; k < dC; ++k) reinterpret_cast<float *>(o.p0)[c * dC + k] = J.bias[k];
                    }
                }
            }
        } else if (fast && CIN == 3) {
            // Taps are addressed box-relative: word index into the re-laid box (TAPS_WORDS) or
            // byte offset into the raw rows, every row starting at phase rph (TAPS_RAW).
            auto fast3 = [&](auto fmt) {
                constexpr int F = decltype(fmt)::value;
                if (OP == OP_RESIZE) {
                    int xo[CPL], xo1[CPL], qxs[CPL];   // left tap (word index / byte offset), right tap
                    float fxs[CPL];
#pragma unroll
                    for (int j = 0; j < CPL; ++j) {
                        const int c = lane + 32 * j;
                        const int xr = ts.cx0[c] - fx0;
                        xo[j] = F == TAPS_RAW ? rph + 3 * xr : xr;
                        xo1[j] = xr + (ts.cqd[c] >> 16);
                        qxs[j] = ts.cqd[c] & 0xFFFF;
                        fxs[j] = ts.cf[c];
                    }
                    for (int r = r0 + warp; r < r1; r += kWarps) {
                        const int y0 = ts.ry0[r], qy = ts.rqd[r] & 0xFFFF, dy = ts.rqd[r] >> 16;
                        const float fy = ts.rf[r];
                        const ORow o = orow_of(r);
                        if (F == TAPS_RAW) {
                            // the pair (x0, x0 + 1) even where x1 = x0 (right edge): there q = 0
                            const uint8_t *b0 = raw + (y0 - fy0) * rstride;
                            const int d1 = dy * rstride;
#pragma unroll
                            for (int j = 0; j < CPL; ++j) {
                                const int c = lane + 32 * j;
                                if (c < nx) {
                                    uint32_t p00, p01, p10, p11;
                                    const uint8_t *wp = b0 + (xo[j] & ~3);
                                    const uint32_t sh = (uint32_t)xo[j] << 3;
                                    raw_pair(wp, sh, p00, p01);
                                    raw_pair(wp + d1, sh, p10, p11);
                                    emit<CIN, OUTK, F>(J, o, c, p00, p01, p10, p11, qxs[j], qy, fxs[j], fy);
                                }
                            }
                        } else {
                            const uint32_t *w0 = words + (y0 - fy0) * sw;
                            const uint32_t *w1 = w0 + dy * sw;
#pragma unroll
                            for (int j = 0; j < CPL; ++j) {
                                const int c = lane + 32 * j;
                                if (c < nx)
                                    emit<CIN, OUTK>(J, o, c, w0[xo[j]], w0[xo1[j]], w1[xo[j]], w1[xo1[j]], qxs[j], qy,
                                                    fxs[j], fy);
                            }
                        }
                    }
                } else {
                    // warp: (ax, ay) = (m00, m10) (x + 1/2) + row terms, the two axes in one packed
                    // lane pair (fp32 fmas, lane by lane as in the definition), then the fast forms,
                    // both rounded toward minus infinity (exact on [0, 4094), checked exhaustively
                    // on the host):
                    //   u8   fma(a, 2048, 2^23 - 1023.5) = 2^23 + 2048 x0 + q  (bits 0x4B000000 + ..;
                    //        q = 2048 comes out as x0 + 1 with q = 0, the same sample)
                    //   f32  a + (2^23 - 1/2) = 2^23 + x0; the weight of x0 + 1 is a - (x0 + 1/2)
                    F2 xc2[CPL];
#pragma unroll
                    for (int j = 0; j < CPL; ++j) {
                        const float xc = __fadd_rn((float)(tx0 + lane + 32 * j), 0.5f);
                        xc2[j] = f2_pack(xc, xc);
                    }
                    const F2 mx = f2_pack(J.M[0], J.M[3]), my = f2_pack(J.M[1], J.M[4]), m2 = f2_pack(J.M[2], J.M[5]);
                    const F2 kq = f2_pack(2048.f, 2048.f), kt = f2_pack(8387584.5f, 8387584.5f);
                    const F2 kf = f2_pack(8388607.5f, 8388607.5f);
                    // The coordinate bits give x0 + xb (and y0 + xb); the top-left tap is word
                    // y sw + x + abase, or byte y rstride + 3 x + abase (mod 2^32).
                    const uint32_t xb = OT::is_f32 ? 0x4B000000u : (0x4B000000u >> 11);
                    const uint32_t abase = F == TAPS_RAW
                                               ? (uint32_t)(rph - fy0 * rstride - 3 * fx0) - xb * (uint32_t)(rstride + 3)
                                               : (uint32_t)(-(fy0 * sw + fx0)) - xb * (uint32_t)(sw + 1);
                    for (int r = r0 + warp; r < r1; r += kWarps) {
                        const float yc = __fadd_rn((float)(ty0 + r), 0.5f);
                        const F2 rxy = f2_fma(my, f2_pack(yc, yc), m2);
                        const float rz = OP == OP_PERSP ? __fmaf_rn(J.M[7], yc, J.M[8]) : 0.f;
                        const ORow o = orow_of(r);
#pragma unroll
                        for (int j = 0; j < CPL; ++j) {
                            const int c = lane + 32 * j;
                            if (c < nx) {
                                F2 a2 = f2_fma(mx, xc2[j], rxy);
                                if (OP == OP_PERSP) {
                                    // (X, Y) q with q = 1/Z: Z > 0 over the tile (its corners)
                                    float xc, xc_hi;
                                    f2_unpack(xc2[j], xc, xc_hi);
                                    const float q = __frcp_rn(__fmaf_rn(J.M[6], xc, rz));
                                    a2 = f2_mul(a2, f2_pack(q, q));
                                }
                                uint32_t xi, yi;
                                int qx = 0, qy = 0;
                                float fx = 0.f, fy = 0.f;
                                if (!OT::is_f32) {
                                    uint32_t tx, ty;
                                    f2_unpack_bits(f2_fma_rm(a2, kq, kt), tx, ty);
                                    xi = tx >> 11; qx = (int)(tx & 2047u);
                                    yi = ty >> 11; qy = (int)(ty & 2047u);
                                } else {
                                    const F2 fl = f2_add_rm(a2, kf);
                                    f2_unpack(f2_sub(a2, f2_sub(fl, kf)), fx, fy);
                                    f2_unpack_bits(fl, xi, yi);
                                }
                                if (F == TAPS_RAW) {
                                    const int off = (int)(yi * (uint32_t)rstride + 3u * xi + abase);
                                    const uint8_t *wp = raw + (off & ~3);
                                    const uint32_t sh = (uint32_t)off << 3;
                                    uint32_t p00, p01, p10, p11;
                                    raw_pair(wp, sh, p00, p01);
                                    raw_pair(wp + rstride, sh, p10, p11);
                                    emit<CIN, OUTK, F>(J, o, c, p00, p01, p10, p11, qx, qy, fx, fy);
                                } else {
                                    const uint32_t *w0 = words + (int)(yi * (uint32_t)sw + xi + abase);
                                    emit<CIN, OUTK>(J, o, c, w0[0], w0[1], w0[sw], w0[sw + 1], qx, qy, fx, fy);
                                }
                            }
                        }
                    }
                }
            };
            if (rawbox) fast3(IntC<TAPS_RAW>{}); else fast3(IntC<TAPS_WORDS>{});
        } else if (OP != OP_RESIZE && CIN == 3 && staged && ti.clamp) {
            // Replicated border, tile whose footprint crosses the image's edge: the box is the
            // footprint clipped to the image; each tap is clamped into the image (its nearest
            // edge pixel), which lies in the box, and read as one pixel word.
            const int bx = J.W - 1 - fx0, by = J.H - 1 - fy0;   // box-relative image edges
            auto px_at = [&](int yb, int xb) -> uint32_t {
                if (rawbox) {
                    const int off = yb * rstride + rph + 3 * xb;
                    const uint32_t *wp = reinterpret_cast<const uint32_t *>(raw + (off & ~3));
                    return __funnelshift_r(wp[0], wp[1], (uint32_t)off << 3);
                }
                return words[yb * sw + xb];
            };
            for (int r = r0 + warp; r < r1; r += kWarps) {
                const ORow o = orow_of(r);
#pragma unroll
                for (int j = 0; j < CPL; ++j) {
                    const int c = lane + 32 * j;
                    if (c < nx) {
                        float sx, sy;
                        map_coord<OP>(J.M, tx0 + c, ty0 + r, sx, sy);   // valid: the tile's corners are
                        int x0, y0, qx, qy;
                        warp_weight(sx, x0, qx);
                        warp_weight(sy, y0, qy);
                        float fx = 0.f, fy = 0.f;
                        if (OT::is_f32) {
                            fx = __fsub_rn(sx, floorf(sx));
                            fy = __fsub_rn(sy, floorf(sy));
                        }
                        const int xa = min(max(x0 - fx0, -fx0), bx), xb = min(max(x0 + 1 - fx0, -fx0), bx);
                        const int ya = min(max(y0 - fy0, -fy0), by), yb = min(max(y0 + 1 - fy0, -fy0), by);
                        emit<CIN, OUTK>(J, o, c, px_at(ya, xa), px_at(ya, xb), px_at(yb, xa), px_at(yb, xb), qx, qy,
                                        fx, fy);
                    }
                }
            }
        } else if (OP != OP_RESIZE && CIN == 3 && staged) {
            // Medium path (warp tiles with coordinates outside [0, 4094)): the exact weight
            // formula per pixel; every tap still lies in the zero-filled box.
            auto medium3 = [&](auto fmt) {
                constexpr int F = decltype(fmt)::value;
                for (int r = r0 + warp; r < r1; r += kWarps) {
                    const float yc = __fadd_rn((float)(ty0 + r), 0.5f);
                    const float rx = __fmaf_rn(J.M[1], yc, J.M[2]);
                    const float ry = __fmaf_rn(J.M[4], yc, J.M[5]);
                    const ORow o = orow_of(r);
#pragma unroll
                    for (int j = 0; j < CPL; ++j) {
                        const int c = lane + 32 * j;
                        if (c < nx) {
                            float sx, sy;
                            if (OP == OP_PERSP) {
                                persp_coord(J.M, tx0 + c, ty0 + r, sx, sy);   // valid: Z > 0 over the tile
                            } else {
                                const float xc = __fadd_rn((float)(tx0 + c), 0.5f);
                                sx = __fsub_rn(__fmaf_rn(J.M[0], xc, rx), 0.5f);
                                sy = __fsub_rn(__fmaf_rn(J.M[3], xc, ry), 0.5f);
                            }
                            int x0, y0, qx, qy;
                            warp_weight(sx, x0, qx);
                            warp_weight(sy, y0, qy);
                            float fx = 0.f, fy = 0.f;
                            if (OT::is_f32) {
                                fx = __fsub_rn(sx, floorf(sx));
                                fy = __fsub_rn(sy, floorf(sy));
                            }
                            if (F == TAPS_RAW) {
                                const int off = (y0 - fy0) * rstride + 3 * (x0 - fx0) + rph;
                                const uint8_t *wp = raw + (off & ~3);
                                const uint32_t sh = (uint32_t)off << 3;
                                uint32_t p00, p01, p10, p11;
                                raw_pair(wp, sh, p00, p01);
                                raw_pair(wp + rstride, sh, p10, p11);
                                emit<CIN, OUTK, F>(J, o, c, p00, p01, p10, p11, qx, qy, fx, fy);
                            } else {
                                const uint32_t *w0 = words + ((y0 - fy0) * sw + (x0 - fx0));
                                emit<CIN, OUTK>(J, o, c, w0[0], w0[1], w0[sw], w0[sw + 1], qx, qy, fx, fy);
                            }
                        }
                    }
                }
            };
            if (rawbox) medium3(IntC<TAPS_RAW>{}); else medium3(IntC<TAPS_WORDS>{});
        } else {
            // General path: per-pixel coordinates with the full rules; taps from the
            // staged box when inside it, else from global memory (zero outside the image).
            const uint32_t rowphase0 = (uint32_t)(uintptr_t)(J.src + (int64_t)fx0 * CIN);
            for (int r = r0 + warp; r < r1; r += kWarps) {
                const int y = ty0 + r;
                const ORow o = orow_of(r);
                for (int j = 0; j < CPL; ++j) {
                    const int c = lane + 32 * j;
                    if (c >= nx) continue;
                    const int x = tx0 + c;
                    int x0 = 0, y0 = 0, qx = 0, qy = 0, dx = 1, dy = 1;
                    float fx = 0.f, fy = 0.f;
                    bool valid = true;
                    if (OP == OP_RESIZE) {
                        x0 = ts.cx0[c]; dx = ts.cqd[c] >> 16; qx = ts.cqd[c] & 0xFFFF; fx = ts.cf[c];
                        y0 = ts.ry0[r]; dy = ts.rqd[r] >> 16; qy = ts.rqd[r] & 0xFFFF; fy = ts.rf[r];
                    } else {
                        float sx, sy;
                        valid = map_coord<OP>(J.M, x, y, sx, sy);
                        if (valid) {
                            warp_weight(sx, x0, qx);
                            warp_weight(sy, y0, qy);
                            fx = __fsub_rn(sx, floorf(sx));
                            fy = __fsub_rn(sy, floorf(sy));
                        }
                    }
                    uint32_t p00 = 0, p01 = 0, p10 = 0, p11 = 0;
                    if (valid) {
                        const bool in_box = staged && x0 >= fx0 && x0 + dx <= fx1 && y0 >= fy0 && y0 + dy <= fy1;
                        // (3-channel tiles get here only unstaged: staged ones take the fast or
                        // medium path)
                        if (in_box && CIN == 3) {
                            const uint32_t *w0 = words + ((y0 - fy0) * sw + (x0 - fx0));
                            const uint32_t *w1 = w0 + dy * sw;
                            p00 = w0[0]; p01 = w0[dx]; p10 = w1[0]; p11 = w1[dx];
                        } else if (in_box) {
                            const int r0 = y0 - fy0, r1 = r0 + dy;
                            const int ph0 = (int)((rowphase0 + (uint32_t)((int64_t)y0 * J.spitch)) & 15u);
                            const int ph1 = (int)((rowphase0 + (uint32_t)((int64_t)(y0 + dy) * J.spitch)) & 15u);
                            const uint8_t *s0 = raw + r0 * rstride + ph0 + (x0 - fx0);
                            const uint8_t *s1 = raw + r1 * rstride + ph1 + (x0 - fx0);
                            p00 = s0[0]; p01 = s0[dx]; p10 = s1[0]; p11 = s1[dx];
                        } else if (CIN == 3) {
                            const bool rp = OP != OP_RESIZE && J.replicate;
                            p00 = ldg_px3(J.src, J.spitch, J.H, J.W, y0, x0, rp);
                            p01 = ldg_px3(J.src, J.spitch, J.H, J.W, y0, x0 + dx, rp);
                            p10 = ldg_px3(J.src, J.spitch, J.H, J.W, y0 + dy, x0, rp);
                            p11 = ldg_px3(J.src, J.spitch, J.H, J.W, y0 + dy, x0 + dx, rp);
                        } else {
                            const bool rp = OP != OP_RESIZE && J.replicate;
                            p00 = ldg_px1(J.src, J.spitch, J.H, J.W, y0, x0, rp);
                            p01 = ldg_px1(J.src, J.spitch, J.H, J.W, y0, x0 + dx, rp);
                            p10 = ldg_px1(J.src, J.spitch, J.H, J.W, y0 + dy, x0, rp);
                            p11 = ldg_px1(J.src, J.spitch, J.H, J.W, y0 + dy, x0 + dx, rp);
                        }
                    }
                    emit<CIN, OUTK>(J, o, c, p00, p01, p10, p11, qx, qy, fx, fy);
                }
            }
        }
        if (tma_out) fence_proxy_async_smem();
        __syncthreads();

        if (tma_out) {
            // write-out through TMA stores of the band (rows and chunks past the image's edge
            // are clipped by the copy engine)
            if (tid == 0) {
                if (chw) {
                    for (int pl = 0; pl < 3; ++pl)
                        tma_store_4d(J.tout, tx0, ty0 + r0, pl, J.zimg, ostage + pl * BH * orow);
                } else {
                    tma_store_3d(J.tout, (tx0 * dC * ES) >> 2, ty0 + r0, J.zimg, ostage);
                }
                tma_store_commit_and_wait_read();
            }
            // After the last band no closing barrier: this path runs one tile per CTA, the
            // storing thread waits for the copy engine to finish reading the stage, and a
            // CTA's shared memory lives until its last thread exits.
            if (r1 >= ny) return;
            continue;
        }

        // write-out: 16-byte chunks of every (plane, row) segment of the band spread over the
        // CTA; a second pass, only when some row is not 16-byte aligned at both ends, moves
        // the (at most 15 + 15) head and tail bytes of each segment, one per thread.
        const int nplanes = chw ? 3 : 1;
        const int nrow = r1 - r0;
        const int seglen = chw ? nx * 4 : nx * dC * ES;
        const int nseg = nplanes * nrow;
        const int ncs = (seglen + 15 + 15) >> 4;           // chunks a segment can span
        const float inv_ncs = __frcp_rn((float)ncs);
        const int64_t tile_off = chw ? (int64_t)tx0 * 4 : (int64_t)tx0 * dC * ES;
        uint8_t *drow0 = J.dst + (int64_t)(ty0 + r0) * J.dpitch + tile_off;
        // segment sidx = (plane, band row rr): its global start and its stage row
        auto seg_base = [&](int sidx, int &srow_off) -> uint8_t * {
            const int pl = chw ? (sidx >= nrow) + (sidx >= 2 * nrow) : 0;
            const int rr = sidx - pl * nrow;
            srow_off = (pl * BH + rr) * orow;
            return drow0 + (int64_t)rr * J.dpitch + (int64_t)pl * J.dplane;
        };
        for (int i = tid; i < nseg * ncs; i += kThreads) {
            const int sidx = (int)__fmul_rz((float)i + 0.5f, inv_ncs);
            const int j = i - sidx * ncs;
            int so;
            uint8_t *g = seg_base(sidx, so);
            const int phase = (int)((uintptr_t)g & 15);
            const int b0 = 16 * j;
            if (b0 >= phase && b0 + 16 <= phase + seglen)
                *reinterpret_cast<uint4 *>(g - phase + b0) = *reinterpret_cast<const uint4 *>(ostage + so + b0);
        }
        const bool aligned_rows = ((obase | opitch | (chw ? oplane : 0u) | (uint32_t)seglen) & 15u) == 0;
        if (!aligned_rows) {
            for (int i = tid; i < nseg * 32; i += kThreads) {
                const int sidx = i >> 5, k = i & 31;
                int so;
                uint8_t *g = seg_base(sidx, so);
                const int phase = (int)((uintptr_t)g & 15);
                const int end = phase + seglen;
                const int jf = (phase + 15) >> 4, jl = end >> 4;   // full chunks: [jf, jl)
                int b;
                if (k < 16) {
                    b = phase + k;
                    if (b >= min(jf * 16, end)) continue;
                } else {
                    if (jl < jf) continue;
                    b = jl * 16 + (k - 16);
                    if (b >= end) continue;
                }
                g[b - phase] = ostage[so + b];
            }
        }
        __syncthreads();
    }
}

}  // namespace kr
