// Quad fast path shared by the tile engines: each lane blends 4 adjacent output pixels of one
// row of a full-width 64-column tile from a box staged as raw rows (all rows at one 16-byte
// phase), and stores them into the output stage as packed words. The arithmetic is the
// definition of kr_device.cuh (resize: exact rational axis tables; warp / perspective: the
// fixed fp32 coordinate sequence and the fast forms exact on [0, 4094); u8: 11-bit weights,
// (v + 2^21) >> 22; f32: lerps of p/255 then * scale + bias), only laid out for fewer
// instructions: 32-bit shared-memory offsets, one pixel quad per lane, and the u8 rounding
// taken as byte 3 of 4 (v + 2^21).
#pragma once

#include "kr_device.cuh"

namespace kr {

// The dynamic shared memory of a tile kernel, addressed by 32-bit byte offsets.
extern __shared__ __align__(128) uint8_t kr_pipe_smem[];

__device__ __forceinline__ uint32_t lds32(uint32_t off) { return *reinterpret_cast<const uint32_t *>(kr_pipe_smem + off); }

// NW words at byte offset off of the shared memory: 16-byte stores where off is 16-byte aligned
// (NW a multiple of 4), else 4-byte stores where it is 4-byte aligned, else byte stores.
template <int NW> __device__ __forceinline__ void sts_words(uint32_t off, const uint32_t (&w)[NW])
{
    if ((NW % 4) == 0 && (off & 15u) == 0) {
#pragma unroll
        for (int i = 0; i < NW / 4; ++i)
            *reinterpret_cast<uint4 *>(kr_pipe_smem + off + 16 * i) = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
    } else if ((off & 3u) == 0) {
#pragma unroll
        for (int i = 0; i < NW; ++i) *reinterpret_cast<uint32_t *>(kr_pipe_smem + off + 4 * i) = w[i];
    } else {
#pragma unroll
        for (int i = 0; i < NW; ++i)
#pragma unroll
            for (int b = 0; b < 4; ++b) kr_pipe_smem[off + 4 * i + b] = (uint8_t)(w[i] >> (8 * b));
    }
}

// The four taps of a raw pixel pair: byte offset o of the pair's first byte in the top staged
// row, d from the top row to the bottom row (three aligned words and two funnel shifts a row).
__device__ __forceinline__ void raw_taps4(uint32_t o, uint32_t d, uint32_t &p00, uint32_t &p01, uint32_t &p10,
                                          uint32_t &p11)
{
    const uint32_t a = o & ~3u, sh = o << 3;
    const uint32_t t0 = lds32(a), t1 = lds32(a + 4), t2 = lds32(a + 8);
    const uint32_t b0 = lds32(a + d), b1 = lds32(a + d + 4), b2 = lds32(a + d + 8);
    p00 = __funnelshift_r(t0, t1, sh);
    p01 = __funnelshift_r(t1, t2, sh);
    p10 = __funnelshift_r(b0, b1, sh);
    p11 = __funnelshift_r(b1, b2, sh);
}

// u8 bilinear blend of raw taps with the weight pair wx (wpair(qx)) and wy1 = 4 qy: each
// channel's 4 (v + 2^21) = top (8192 - 4 qy) + bottom 4 qy + 2^23 < 2^32, so the rounded
// result (v + 2^21) >> 22 is byte 3 of the returned word.
struct Q3 {
    uint32_t r, g, b;
};
__device__ __forceinline__ Q3 blend_u8_b3(uint32_t p00, uint32_t p01, uint32_t p10, uint32_t p11, uint32_t wx,
                                          uint32_t wy1)
{
    const U8x3 a = hblend_pair<TAPS_RAW>(p00, p01, wx), b = hblend_pair<TAPS_RAW>(p10, p11, wx);
    const uint32_t wy0 = 8192u - wy1;
    Q3 o;
    o.r = a.r * wy0 + (b.r * wy1 + (1u << 23));
    o.g = a.g * wy0 + (b.g * wy1 + (1u << 23));
    o.b = a.b * wy0 + (b.b * wy1 + (1u << 23));
    return o;
}

// f32 bilinear blend of raw taps (values p/255 scaled by 255: the bytes), as in emit.
__device__ __forceinline__ void blend_f32_raw(uint32_t p00, uint32_t p01, uint32_t p10, uint32_t p11, float fx,
                                              float fy, float (&v)[3])
{
    const F2 K = f2_pack(8388608.f, 8388608.f);
    const F2 fx2 = f2_pack(fx, fx), fy2 = f2_pack(fy, fy);
    const F2 a = rg_biased(p00), b = rg1_biased<TAPS_RAW>(p00, p01);
    const F2 cc = rg_biased(p10), d = rg1_biased<TAPS_RAW>(p10, p11);
    const F2 h0 = f2_fma(fx2, f2_sub(b, a), f2_sub(a, K));
    const F2 h1 = f2_fma(fx2, f2_sub(d, cc), f2_sub(cc, K));
    f2_unpack(f2_fma(fy2, f2_sub(h1, h0), h0), v[0], v[1]);
    const float kb = 8388608.f;
    const float ba = __uint_as_float(__byte_perm(p00, 0x4B000000u, 0x7542));
    const float bb = __uint_as_float(b1_biased<TAPS_RAW>(p01));
    const float bc = __uint_as_float(__byte_perm(p10, 0x4B000000u, 0x7542));
    const float bd = __uint_as_float(b1_biased<TAPS_RAW>(p11));
    const float g0 = __fmaf_rn(fx, __fsub_rn(bb, ba), __fsub_rn(ba, kb));
    const float g1 = __fmaf_rn(fx, __fsub_rn(bd, bc), __fsub_rn(bc, kb));
    v[2] = __fmaf_rn(fy, __fsub_rn(g1, g0), g0);
}

// Blended values of a lane's 4 adjacent output pixels, before the store.
template <int OUTK> struct QuadOut {
    Q3 u[4];          // u8 kinds: byte 3 of each channel
    float f[4][3];    // f32 kinds: v255 per channel
};

template <int OUTK>
__device__ __forceinline__ void quad_blend(QuadOut<OUTK> &Q, int j, uint32_t p00, uint32_t p01, uint32_t p10,
                                           uint32_t p11, uint32_t wx, uint32_t wy1, float fx, float fy)
{
    if (OUTK == OUT_U8 || OUTK == OUT_U8_GRAY)
        Q.u[j] = blend_u8_b3(p00, p01, p10, p11, wx, wy1);
    else
        blend_f32_raw(p00, p01, p10, p11, fx, fy, Q.f[j]);
}

// Store a lane's 4 adjacent output pixels (columns cb .. cb + 3 of the tile) into the output
// stage: off0 = byte offset of the pixels' row (planar: of plane 0's row), oplane_off = the
// offset between planes' rows in the stage.
template <int OUTK>
__device__ __forceinline__ void quad_store(const QuadOut<OUTK> &Q, const Job &J, bool chw, uint32_t off0,
                                           uint32_t off1, uint32_t off2, int cb)
{
    if (OUTK == OUT_U8) {
        uint32_t w[3];
        const uint32_t a0 = __byte_perm(Q.u[0].r, Q.u[0].g, 0x0073), a1 = __byte_perm(Q.u[0].b, Q.u[1].r, 0x0073);
        const uint32_t b0 = __byte_perm(Q.u[1].g, Q.u[1].b, 0x0073), b1 = __byte_perm(Q.u[2].r, Q.u[2].g, 0x0073);
        const uint32_t c0 = __byte_perm(Q.u[2].b, Q.u[3].r, 0x0073), c1 = __byte_perm(Q.u[3].g, Q.u[3].b, 0x0073);
        w[0] = __byte_perm(a0, a1, 0x5410);
        w[1] = __byte_perm(b0, b1, 0x5410);
        w[2] = __byte_perm(c0, c1, 0x5410);
        sts_words<3>(off0 + 3 * cb, w);
    } else if (OUTK == OUT_U8_GRAY) {
        uint32_t g[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            g[j] = __dp2a_lo(4899u | (9617u << 16), __byte_perm(Q.u[j].r, Q.u[j].g, 0x0073),
                             8192u + 1868u * (Q.u[j].b >> 24)) >> 14;
        uint32_t w[1];
        w[0] = __byte_perm(__byte_perm(g[0], g[1], 0x0040), __byte_perm(g[2], g[3], 0x0040), 0x5410);
        sts_words<1>(off0 + cb, w);
    } else if (OUTK == OUT_F32_GRAY) {
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float g = __fmaf_rn(0.299f, Q.f[j][0], __fmaf_rn(0.587f, Q.f[j][1], __fmul_rn(0.114f, Q.f[j][2])));
            w[j] = __float_as_uint(__fmaf_rn(g, J.scale[0], J.bias[0]));
        }
        sts_words<4>(off0 + 4 * cb, w);
    } else if (chw) {
        uint32_t w0[4], w1[4], w2[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            w0[j] = __float_as_uint(__fmaf_rn(Q.f[j][0], J.scale[0], J.bias[0]));
            w1[j] = __float_as_uint(__fmaf_rn(Q.f[j][1], J.scale[1], J.bias[1]));
            w2[j] = __float_as_uint(__fmaf_rn(Q.f[j][2], J.scale[2], J.bias[2]));
        }
        sts_words<4>(off0 + 4 * cb, w0);
        sts_words<4>(off1 + 4 * cb, w1);
        sts_words<4>(off2 + 4 * cb, w2);
    } else {
        uint32_t w[12];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) w[3 * j + k] = __float_as_uint(__fmaf_rn(Q.f[j][k], J.scale[k], J.bias[k]));
        sts_words<12>(off0 + 12 * cb, w);
    }
}

// Per-tile state of a lane's quad (columns cb .. cb + 3 of a full-width tile).
struct QuadTile {
    uint32_t xo[4], wq[4];   // resize: byte offset of the tap pair in a staged row, weight pair
    float fxs[4];            // resize: fp32 weight of x1
    F2 xc2[4];               // warp: x + 1/2 in both lanes
    F2 mx, my, m2;           // warp: the map's columns, both axes
    uint32_t abase;          // warp: shared-memory offset bias of the top-left tap
};

// Set-up of the quad state: cx0/cqd/cf are the resize column tables of the tile (shared
// memory), sraw the offset of the staged box, rph the phase of its rows. Columns at or past nx
// (a tile at the image's right edge) repeat column nx - 1: their taps stay inside the box, and
// the values they produce land in stage columns that are never written out.
template <int OP, int OUTK>
__device__ __forceinline__ void quad_setup(QuadTile &T, const Job &J, const int *cx0, const int *cqd, const float *cf,
                                           int tx0, int fx0, int fy0, int rstride, uint32_t sraw, int rph, int cb,
                                           int nx)
{
    if (OP == OP_RESIZE) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = min(cb + j, nx - 1);
            T.xo[j] = sraw + (uint32_t)(rph + 3 * (cx0[c] - fx0));
            T.wq[j] = wpair(cqd[c] & 0xFFFF);
            T.fxs[j] = cf[c];
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float xc = __fadd_rn((float)(tx0 + min(cb + j, nx - 1)), 0.5f);
            T.xc2[j] = f2_pack(xc, xc);
        }
        T.mx = f2_pack(J.M[0], J.M[3]);
        T.my = f2_pack(J.M[1], J.M[4]);
        T.m2 = f2_pack(J.M[2], J.M[5]);
        // the coordinate bits give x0 + xb (and y0 + xb); the top-left tap is byte
        // y rstride + 3 x + abase (mod 2^32) of the shared memory
        constexpr uint32_t xb = OutTraits<OUTK, 3>::is_f32 ? 0x4B000000u : (0x4B000000u >> 11);
        T.abase = sraw + (uint32_t)(rph - fy0 * rstride - 3 * fx0) - xb * (uint32_t)(rstride + 3);
    }
}

// The packed bytes of a lane's 4 adjacent u8 output pixels: 12 (3 words) for RGB, 4 for gray.
template <int OUTK> struct QuadWords {
    static constexpr int n = OUTK == OUT_U8 ? 3 : 1;
};
template <int OUTK>
__device__ __forceinline__ void quad_pack_u8(const QuadOut<OUTK> &Q, uint32_t (&w)[QuadWords<OUTK>::n])
{
    if constexpr (OUTK == OUT_U8) {
        const uint32_t a0 = __byte_perm(Q.u[0].r, Q.u[0].g, 0x0073), a1 = __byte_perm(Q.u[0].b, Q.u[1].r, 0x0073);
        const uint32_t b0 = __byte_perm(Q.u[1].g, Q.u[1].b, 0x0073), b1 = __byte_perm(Q.u[2].r, Q.u[2].g, 0x0073);
        const uint32_t c0 = __byte_perm(Q.u[2].b, Q.u[3].r, 0x0073), c1 = __byte_perm(Q.u[3].g, Q.u[3].b, 0x0073);
        w[0] = __byte_perm(a0, a1, 0x5410);
        w[1] = __byte_perm(b0, b1, 0x5410);
        w[2] = __byte_perm(c0, c1, 0x5410);
    } else if constexpr (OUTK == OUT_U8_GRAY) {
        uint32_t g[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            g[j] = __dp2a_lo(4899u | (9617u << 16), __byte_perm(Q.u[j].r, Q.u[j].g, 0x0073),
                             8192u + 1868u * (Q.u[j].b >> 24)) >> 14;
        w[0] = __byte_perm(__byte_perm(g[0], g[1], 0x0040), __byte_perm(g[2], g[3], 0x0040), 0x5410);
    }
}

// A run of L bytes at g (any alignment) held by the 16 lanes of a half-warp, NW words each
// (lane l16 holds bytes [4 NW l16, 4 NW (l16 + 1))), written with aligned 4-byte stores: the
// aligned word k of the run's span (bytes [4k - p, 4k - p + 4) of the run, p = g mod 4) is
// built from the two words that hold its bytes (the first from the lane below, by a shuffle)
// and stored by the lane that holds its last bytes; a word the run covers only in part (its
// first and last) goes byte by byte. Every lane of the warp calls this (L = 0: no stores).
template <int NW>
__device__ __forceinline__ void store_run_u8(uint8_t *g, int L, const uint32_t (&x)[NW], int l16)
{
    const uint32_t p = (uint32_t)(uintptr_t)g & 3u;
    uint32_t *A = reinterpret_cast<uint32_t *>(g - p);
    const uint32_t prev = __shfl_up_sync(0xffffffffu, x[NW - 1], 1, 16);
    const uint32_t sh = 32u - 8u * p;   // (p = 0: the clamped shift gives the upper word)
#pragma unroll
    for (int i = 0; i <= NW; ++i) {
        if (i == NW && l16 != 15) break;   // (the next lane's first word)
        const uint32_t lo = i == 0 ? prev : x[i - 1], hi = i < NW ? x[i] : 0u;
        const uint32_t v = __funnelshift_rc(lo, hi, sh);
        const int k = NW * l16 + i;
        const int s0 = 4 * k - (int)p;   // run byte of the word's first byte
        if (s0 >= 0 && s0 + 4 <= L) {
            A[k] = v;
        } else {
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if (s0 + b >= 0 && s0 + b < L) g[s0 + b] = (uint8_t)(v >> (8 * b));
        }
    }
}

// Store a lane's 4 adjacent output pixels straight to global memory: g0 = the pixels' row
// (planar: plane 0's row; planes oplane bytes apart), 16-byte aligned (f32: 16-byte stores of
// each 4-pixel group; u8: 4-byte stores).
template <int OUTK>
__device__ __forceinline__ void quad_store_global(const QuadOut<OUTK> &Q, const Job &J, bool chw, uint8_t *g0,
                                                  int64_t oplane, int cb)
{
    if constexpr (OUTK == OUT_U8) {
        uint32_t w[3];
        quad_pack_u8<OUTK>(Q, w);
        uint32_t *d = reinterpret_cast<uint32_t *>(g0 + 3 * cb);
        d[0] = w[0];
        d[1] = w[1];
        d[2] = w[2];
    } else if constexpr (OUTK == OUT_U8_GRAY) {
        uint32_t w[1];
        quad_pack_u8<OUTK>(Q, w);
        *reinterpret_cast<uint32_t *>(g0 + cb) = w[0];
    } else if constexpr (OUTK == OUT_F32_GRAY) {
        float g[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float v = __fmaf_rn(0.299f, Q.f[j][0], __fmaf_rn(0.587f, Q.f[j][1], __fmul_rn(0.114f, Q.f[j][2])));
            g[j] = __fmaf_rn(v, J.scale[0], J.bias[0]);
        }
        *reinterpret_cast<float4 *>(g0 + 4 * cb) = make_float4(g[0], g[1], g[2], g[3]);
    } else if constexpr (OUTK == OUT_F32) {
        if (chw) {
#pragma unroll
            for (int k = 0; k < 3; ++k)
                *reinterpret_cast<float4 *>(g0 + k * oplane + 4 * cb) =
                    make_float4(__fmaf_rn(Q.f[0][k], J.scale[k], J.bias[k]), __fmaf_rn(Q.f[1][k], J.scale[k], J.bias[k]),
                                __fmaf_rn(Q.f[2][k], J.scale[k], J.bias[k]), __fmaf_rn(Q.f[3][k], J.scale[k], J.bias[k]));
        } else {
            float w[12];
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int k = 0; k < 3; ++k) w[3 * j + k] = __fmaf_rn(Q.f[j][k], J.scale[k], J.bias[k]);
            float4 *d = reinterpret_cast<float4 *>(g0 + 12 * cb);
            d[0] = make_float4(w[0], w[1], w[2], w[3]);
            d[1] = make_float4(w[4], w[5], w[6], w[7]);
            d[2] = make_float4(w[8], w[9], w[10], w[11]);
        }
    }
}

// One row r of the lane's quad: the blended values of its 4 pixels. ry0/rqd/rf are the resize
// row tables.
template <int OP, int OUTK>
__device__ __forceinline__ void quad_eval(QuadOut<OUTK> &Q, const QuadTile &T, const Job &J, const int *ry0,
                                          const int *rqd, const float *rf, int r, int ty0, int fy0, int rstride)
{
    using OT = OutTraits<OUTK, 3>;
    if (OP == OP_RESIZE) {
        const int rq = rqd[r];
        const uint32_t wy1 = (uint32_t)(rq & 0xFFFF) << 2;
        const float fy = rf[r];
        const uint32_t rb = (uint32_t)((ry0[r] - fy0) * rstride);
        const uint32_t d1 = (uint32_t)((rq >> 16) * rstride);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t p00, p01, p10, p11;
            raw_taps4(rb + T.xo[j], d1, p00, p01, p10, p11);
            quad_blend<OUTK>(Q, j, p00, p01, p10, p11, T.wq[j], wy1, T.fxs[j], fy);
        }
    } else {
        // warp: both axes in one packed lane pair, then the fast forms rounded toward minus
        // infinity (exact on [0, 4094), checked exhaustively on the host): u8
        // fma(a, 2048, 2^23 - 1023.5) = 2^23 + 2048 x0 + q; f32 a + (2^23 - 1/2) = 2^23 + x0,
        // weight of x0 + 1 = a - (x0 + 1/2)
        const F2 kq = f2_pack(2048.f, 2048.f), kt = f2_pack(8387584.5f, 8387584.5f);
        const F2 kf = f2_pack(8388607.5f, 8388607.5f);
        const float yc = __fadd_rn((float)(ty0 + r), 0.5f);
        const F2 rxy = f2_fma(T.my, f2_pack(yc, yc), T.m2);
        const float rz = OP == OP_PERSP ? __fmaf_rn(J.M[7], yc, J.M[8]) : 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            F2 a2 = f2_fma(T.mx, T.xc2[j], rxy);
            if (OP == OP_PERSP) {
                float xc, xc_hi;
                f2_unpack(T.xc2[j], xc, xc_hi);
                const float q = __frcp_rn(__fmaf_rn(J.M[6], xc, rz));
                a2 = f2_mul(a2, f2_pack(q, q));
            }
            uint32_t xi, yi, wx = 0, wy1 = 0;
            float fx = 0.f, fy = 0.f;
            if (!OT::is_f32) {
                uint32_t tx, ty;
                f2_unpack_bits(f2_fma_rm(a2, kq, kt), tx, ty);
                xi = tx >> 11;
                yi = ty >> 11;
                wx = wpair((int)(tx & 2047u));
                wy1 = (ty & 2047u) << 2;
            } else {
                const F2 fl = f2_add_rm(a2, kf);
                f2_unpack(f2_sub(a2, f2_sub(fl, kf)), fx, fy);
                f2_unpack_bits(fl, xi, yi);
            }
            uint32_t p00, p01, p10, p11;
            raw_taps4(yi * (uint32_t)rstride + 3u * xi + T.abase, (uint32_t)rstride, p00, p01, p10, p11);
            quad_blend<OUTK>(Q, j, p00, p01, p10, p11, wx, wy1, fx, fy);
        }
    }
}

// One row r of the lane's quad: blend and store into the output stage at off0 (planar f32:
// plane rows off0, off1, off2).
template <int OP, int OUTK>
__device__ __forceinline__ void quad_row(const QuadTile &T, const Job &J, const int *ry0, const int *rqd,
                                         const float *rf, int r, int ty0, int fy0, int rstride, uint32_t sraw,
                                         bool chw, uint32_t off0, uint32_t off1, uint32_t off2, int cb)
{
    QuadOut<OUTK> Q;
    quad_eval<OP, OUTK>(Q, T, J, ry0, rqd, rf, r, ty0, fy0, rstride);
    quad_store<OUTK>(Q, J, chw, off0, off1, off2, cb);
}

}  // namespace kr
