// Device-side tile engine of the resampling kernels (sm_103a).
//
// One CTA of kThreads threads produces one TW x TH tile of output pixels:
//   1. the source footprint of the tile (the bounding box of every tap) is
//      copied into shared memory: 16-byte cp.async for the aligned body of
//      each source row, byte loads for its unaligned head and tail;
//   2. every output pixel takes its four taps from shared memory (global
//      memory at the zero border, or when the footprint does not fit) and
//      blends them: u8 with 11-bit weights through dp2a, f32 with fp32 FMAs;
//   3. results are written into a shared-memory copy of the output tile whose
//      rows carry the same 16-byte phase as their global rows, so the tile
//      leaves through 128-bit coalesced stores (byte stores only for the
//      unaligned head and tail of a row).
//
// The arithmetic follows the definitions stated in include/kr.h (half-pixel
// centres, clamp-to-edge resize, zero-border warp with the fixed fp32
// coordinate sequence, 11-bit round-half-up weights, BT.601 gray).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace kr {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

enum { OP_RESIZE = 0, OP_WARP = 1 };
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
    int32_t foot_budget;  // shared bytes available for the source footprint (0: never stage)
    float M[6];           // destination -> source map (warp)
    float scale[3];       // f32: out = v255 * scale[c] + bias[c]
    float bias[3];
};

__host__ __device__ constexpr int round16(int x) { return (x + 15) & ~15; }

// Bytes per output element and channels of the destination.
template <int OUTK, int CIN> struct OutTraits {
    static constexpr int esize = (OUTK == OUT_F32 || OUTK == OUT_F32_GRAY) ? 4 : 1;
    static constexpr int dC = (OUTK == OUT_U8_GRAY || OUTK == OUT_F32_GRAY) ? 1 : CIN;
    static constexpr bool is_f32 = esize == 4;
};

// Shared bytes of the output staging buffer of a TW x TH tile: f32 tiles are
// sized for three planar rows of TW floats (which also covers one HWC row of
// 3*TW floats); u8 tiles hold TH rows of TW*dC bytes. Every row gets 15 bytes
// of room for its 16-byte phase.
template <int OUTK, int CIN, int TW, int TH>
__host__ __device__ constexpr int out_stage_bytes()
{
    return OutTraits<OUTK, CIN>::is_f32
               ? OutTraits<OUTK, CIN>::dC * TH * round16(TW * 4 + 15)
               : TH * round16(TW * OutTraits<OUTK, CIN>::dC + 15);
}

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

// Six bytes starting at shared byte offset o (two RGB pixels): lo = bytes 0..3, hi = bytes 4..5.
__device__ __forceinline__ void lds6(const uint8_t *s, int o, uint32_t &lo, uint32_t &hi)
{
    const uint32_t *wp = reinterpret_cast<const uint32_t *>(s + (o & ~3));
    const uint32_t sh = (uint32_t)(o & 3) * 8u;
    const uint32_t w0 = wp[0], w1 = wp[1];
    const uint32_t w2 = (o & 3) > 2 ? wp[2] : 0u;
    lo = __funnelshift_r(w0, w1, sh);
    hi = __funnelshift_r(w1, w2, sh);
}

// One RGB pixel from global memory (zero outside the image).
__device__ __forceinline__ uint32_t ldg_px3(const uint8_t *src, int64_t spitch, int H, int W, int y,
                                            int x)
{
    if ((unsigned)x >= (unsigned)W || (unsigned)y >= (unsigned)H) return 0u;
    const uint8_t *p = src + (int64_t)y * spitch + (int64_t)x * 3;
    return (uint32_t)__ldg(p) | ((uint32_t)__ldg(p + 1) << 8) | ((uint32_t)__ldg(p + 2) << 16);
}

__device__ __forceinline__ uint32_t ldg_px1(const uint8_t *src, int64_t spitch, int H, int W, int y,
                                            int x)
{
    if ((unsigned)x >= (unsigned)W || (unsigned)y >= (unsigned)H) return 0u;
    return (uint32_t)__ldg(src + (int64_t)y * spitch + x);
}

// Exact float of byte k of w (0..255): 2^23 + b has b in its low mantissa bits.
__device__ __forceinline__ float byte_f(uint32_t w, int k)
{
    const uint32_t sel = 0x7540u | (uint32_t)k;
    return __fsub_rn(__uint_as_float(__byte_perm(w, 0x4B000000u, sel)), 8388608.f);
}

// Byte i (0..7) of the pair (lo, hi) as an exact float; i is a compile-time constant.
__device__ __forceinline__ float pair_f(uint32_t lo, uint32_t hi, int i)
{
    return i < 4 ? byte_f(lo, i) : byte_f(hi, i - 4);
}

// u8 blend of two rows of RGB tap pairs. lo/hi: bytes R0 G0 B0 R1 | G1 B1 of a row.
struct U8x3 { uint32_t r, g, b; };

__device__ __forceinline__ U8x3 hblend3(uint32_t lo, uint32_t hi, uint32_t wx)
{
    const uint32_t rg = __byte_perm(lo, hi, 0x4130);   // R0 R1 G0 G1
    const uint32_t bb = __byte_perm(lo, hi, 0x0052);   // B0 B1
    U8x3 o;
    o.r = __dp2a_lo(wx, rg, 0u);
    o.g = __dp2a_hi(wx, rg, 0u);
    o.b = __dp2a_lo(wx, bb, 0u);
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

// Shared tile-level state of the engine: the staged source box and, for
// resize, the per-column and per-row axis maps of the current tile.
struct TileInfo {
    int fx0, fx1, fy0, fy1;   // staged source box (inclusive)
    int srow;                 // shared bytes per staged row
    int staged;               // 1 if the footprint is in shared memory
};

template <int TW, int TH> struct TileShared {
    TileInfo ti;
    int cx0[TW];     // column tap x0
    int cqd[TW];     // q | (x1 - x0) << 16
    float cf[TW];    // fp32 weight of x1
    int ry0[TH];
    int rqd[TH];
    float rf[TH];
};

// ---------------------------------------------------------------------------
// The tile engine.
// ---------------------------------------------------------------------------
template <int OP, int CIN, int OUTK, int TW, int TH>
__device__ __forceinline__ void process_tile(const Job &J, int tile_x, int tile_y, uint8_t *smem,
                                             TileShared<TW, TH> &ts)
{
    TileInfo &ti = ts.ti;
    static_assert(TW % 32 == 0 && TH % kWarps == 0, "tile shape");
    using OT = OutTraits<OUTK, CIN>;
    constexpr int dC = OT::dC;
    constexpr int ES = OT::esize;
    constexpr int NPL = (OT::is_f32 && dC == 3) ? 3 : 1;   // planes when CHW
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx0 = tile_x * TW, ty0 = tile_y * TH;
    const int nx = min(TW, J.w - tx0), ny = min(TH, J.h - ty0);

    // ---- 1. axis tables (resize) and source footprint ----------------------------
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
    }
    if (tid == 0) {
        int fx0, fx1, fy0, fy1;
        bool ok = true;
        if (OP == OP_RESIZE) {
            fx0 = ts.cx0[0];
            fx1 = ts.cx0[nx - 1] + (ts.cqd[nx - 1] >> 16);
            fy0 = ts.ry0[0];
            fy1 = ts.ry0[ny - 1] + (ts.rqd[ny - 1] >> 16);
        } else {
            float mnx = 3.4e38f, mxx = -3.4e38f, mny = 3.4e38f, mxy = -3.4e38f;
            const int cx[2] = {tx0, tx0 + nx - 1}, cy[2] = {ty0, ty0 + ny - 1};
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) {
                    float sx, sy;
                    ok = ok && warp_coord(J.M, cx[a], cy[b], sx, sy) && fabsf(sx) < 1048576.f &&
                         fabsf(sy) < 1048576.f;
                    mnx = fminf(mnx, sx); mxx = fmaxf(mxx, sx);
                    mny = fminf(mny, sy); mxy = fmaxf(mxy, sy);
                }
            if (ok) {
                fx0 = max((int)floorf(mnx) - 1, 0);
                fx1 = min((int)floorf(mxx) + 2, J.W - 1);
                fy0 = max((int)floorf(mny) - 1, 0);
                fy1 = min((int)floorf(mxy) + 2, J.H - 1);
                ok = fx0 <= fx1 && fy0 <= fy1;
            }
        }
        int srow = 0;
        if (ok) {
            srow = round16((fx1 - fx0 + 1) * CIN + 15);
            const long long need = (long long)(fy1 - fy0 + 1) * srow + 16;
            ok = need <= J.foot_budget;
        }
        ti.fx0 = ok ? fx0 : 0; ti.fx1 = ok ? fx1 : -1;
        ti.fy0 = ok ? fy0 : 0; ti.fy1 = ok ? fy1 : -1;
        ti.srow = srow;
        ti.staged = ok ? 1 : 0;
    }
    __syncthreads();
    const int fx0 = ti.fx0, fx1 = ti.fx1, fy0 = ti.fy0, fy1 = ti.fy1, srow = ti.srow;
    const bool staged = ti.staged != 0;
    uint8_t *foot = smem;
    uint8_t *ostage = smem + J.foot_budget;

    if (staged) {
        const int L = (fx1 - fx0 + 1) * CIN;
        for (int r = warp; r <= fy1 - fy0; r += kWarps) {
            const uint8_t *a = J.src + (int64_t)(fy0 + r) * J.spitch + (int64_t)fx0 * CIN;
            const uint8_t *G = reinterpret_cast<const uint8_t *>((uintptr_t)a & ~(uintptr_t)15);
            const int phase = (int)((uintptr_t)a & 15);
            const int nch = (phase + L + 15) >> 4;
            uint8_t *srowp = foot + r * srow;
            for (int j = lane; j < nch; j += 32) {
                const int b0 = j * 16, b1 = b0 + 16;   // chunk bytes relative to G
                if (b0 >= phase && b1 <= phase + L) {
                    cp_async16(srowp + b0, G + b0);
                } else {
                    const int lo = max(b0, phase), hi = min(b1, phase + L);
                    for (int b = lo; b < hi; ++b) srowp[b] = __ldg(G + b);
                }
            }
        }
        cp_async_wait_all();
    }
    __syncthreads();

    // ---- 2. per-pixel compute into the output staging ---------------------------
    // Output staging geometry: HWC -> one plane of rows of TW*dC*ES bytes;
    // CHW (f32, 3 channels) -> three planes of rows of TW*4 bytes.
    const bool chw = OT::is_f32 && dC == 3 && J.chw;
    const int orow = chw ? round16(TW * 4 + 15) : round16(TW * dC * ES + 15);
    auto ophase = [&](int plane, int r) -> int {
        const uint8_t *g = J.dst + (int64_t)(ty0 + r) * J.dpitch +
                           (chw ? (int64_t)plane * J.dplane + (int64_t)tx0 * 4
                                : (int64_t)tx0 * dC * ES);
        return (int)((uintptr_t)g & 15);
    };

    // Per-lane column parameters (resize), read once from the tile tables.
    constexpr int CPL = TW / 32;
    int cx0[CPL], cdx[CPL], cq[CPL];
    float cf[CPL];
    if (OP == OP_RESIZE) {
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
            const int c = lane + 32 * j;
            cx0[j] = ts.cx0[c]; cq[j] = ts.cqd[c] & 0xFFFF; cdx[j] = ts.cqd[c] >> 16; cf[j] = ts.cf[c];
        }
    }

    const uint32_t sbase = (uint32_t)(uintptr_t)(J.src + (int64_t)fx0 * CIN);

    for (int r = warp; r < ny; r += kWarps) {
        const int y = ty0 + r;
        int ry0 = 0, rdy = 0, rq = 0;
        float rf = 0.f;
        if (OP == OP_RESIZE) {
            ry0 = ts.ry0[r]; rq = ts.rqd[r] & 0xFFFF; rdy = ts.rqd[r] >> 16; rf = ts.rf[r];
        }
        const int oph = ophase(0, r);
        uint8_t *orowp = ostage + r * orow;
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
            const int c = lane + 32 * j;
            if (c >= nx) continue;
            const int x = tx0 + c;
            int x0, y0, qx, qy, dx, dy;
            float fx, fy;
            bool valid = true;   // false: sample outside the coordinate range -> 0
            if (OP == OP_RESIZE) {
                x0 = cx0[j]; dx = cdx[j]; qx = cq[j]; fx = cf[j];
                y0 = ry0; dy = rdy; qy = rq; fy = rf;
            } else {
                float sx, sy;
                valid = warp_coord(J.M, x, y, sx, sy);
                x0 = y0 = qx = qy = 0; fx = fy = 0.f;
                if (valid) {
                    warp_weight(sx, x0, qx);
                    warp_weight(sy, y0, qy);
                    if (OT::is_f32) {
                        fx = __fsub_rn(sx, floorf(sx));
                        fy = __fsub_rn(sy, floorf(sy));
                    }
                }
                dx = 1; dy = 1;
            }
            // ---- fetch taps as byte pairs of each source row:
            //   CIN 3: lo = R0 G0 B0 R1, hi = G1 B1 (taps x0 and x0 + 1);
            //   CIN 1: lo = p0 | p1 << 8.
            // Resize at the right/bottom edge has dx or dy = 0 and a zero weight on
            // the second tap, so reading x0 + 1 (or row y0) there changes nothing.
            uint32_t lo0 = 0, hi0 = 0, lo1 = 0, hi1 = 0;
            if (valid) {
                const bool in_box = staged && x0 >= fx0 && x0 + dx <= fx1 && y0 >= fy0 && y0 + dy <= fy1;
                if (in_box) {
                    const int r0 = y0 - fy0, r1 = r0 + dy;
                    const int ph0 = (int)((sbase + (uint32_t)((int64_t)y0 * J.spitch)) & 15u);
                    const int ph1 = (int)((sbase + (uint32_t)((int64_t)(y0 + dy) * J.spitch)) & 15u);
                    const int xo = (x0 - fx0) * CIN;
                    if (CIN == 3) {
                        lds6(foot + r0 * srow, ph0 + xo, lo0, hi0);
                        lds6(foot + r1 * srow, ph1 + xo, lo1, hi1);
                    } else {
                        const uint8_t *s0 = foot + r0 * srow + ph0 + xo;
                        const uint8_t *s1 = foot + r1 * srow + ph1 + xo;
                        lo0 = (uint32_t)s0[0] | ((uint32_t)s0[1] << 8);
                        lo1 = (uint32_t)s1[0] | ((uint32_t)s1[1] << 8);
                    }
                } else if (CIN == 3) {
                    const uint32_t a = ldg_px3(J.src, J.spitch, J.H, J.W, y0, x0);
                    const uint32_t b = ldg_px3(J.src, J.spitch, J.H, J.W, y0, x0 + dx);
                    const uint32_t c2 = ldg_px3(J.src, J.spitch, J.H, J.W, y0 + dy, x0);
                    const uint32_t d = ldg_px3(J.src, J.spitch, J.H, J.W, y0 + dy, x0 + dx);
                    lo0 = a | (b << 24); hi0 = b >> 8;
                    lo1 = c2 | (d << 24); hi1 = d >> 8;
                } else {
                    lo0 = ldg_px1(J.src, J.spitch, J.H, J.W, y0, x0) |
                          (ldg_px1(J.src, J.spitch, J.H, J.W, y0, x0 + dx) << 8);
                    lo1 = ldg_px1(J.src, J.spitch, J.H, J.W, y0 + dy, x0) |
                          (ldg_px1(J.src, J.spitch, J.H, J.W, y0 + dy, x0 + dx) << 8);
                }
            }
            // ---- blend and stage
            if (!OT::is_f32) {
                const uint32_t wx = (uint32_t)(2048 - qx) | ((uint32_t)qx << 16);
                uint32_t o0, o1 = 0, o2 = 0;
                if (CIN == 3) {
                    const U8x3 a = hblend3(lo0, hi0, wx), b = hblend3(lo1, hi1, wx);
                    o0 = vblend(a.r, b.r, qy); o1 = vblend(a.g, b.g, qy); o2 = vblend(a.b, b.b, qy);
                } else {
                    o0 = vblend(__dp2a_lo(wx, lo0, 0u), __dp2a_lo(wx, lo1, 0u), qy);
                }
                uint8_t *op = orowp + oph + c * dC;
                if (OUTK == OUT_U8_GRAY) {
                    op[0] = (uint8_t)gray_u8(o0, o1, o2);
                } else {
                    op[0] = (uint8_t)o0;
                    if (CIN == 3) { op[1] = (uint8_t)o1; op[2] = (uint8_t)o2; }
                }
            } else {
                float v[3];
#pragma unroll
                for (int k = 0; k < CIN; ++k) {
                    const float a = pair_f(lo0, hi0, k), b = pair_f(lo0, hi0, CIN + k);
                    const float d0 = pair_f(lo1, hi1, k), d1 = pair_f(lo1, hi1, CIN + k);
                    const float h0 = __fmaf_rn(fx, __fsub_rn(b, a), a);
                    const float h1 = __fmaf_rn(fx, __fsub_rn(d1, d0), d0);
                    v[k] = __fmaf_rn(fy, __fsub_rn(h1, h0), h0);
                }
                if (OUTK == OUT_F32_GRAY) {
                    const float g = __fmaf_rn(0.299f, v[0], __fmaf_rn(0.587f, v[1], __fmul_rn(0.114f, v[2])));
                    *reinterpret_cast<float *>(orowp + oph + c * 4) = __fmaf_rn(g, J.scale[0], J.bias[0]);
                } else if (chw) {
#pragma unroll
                    for (int k = 0; k < CIN; ++k) {
                        uint8_t *pl = ostage + k * TH * orow + r * orow + ophase(k, r);
                        *reinterpret_cast<float *>(pl + c * 4) = __fmaf_rn(v[k], J.scale[k], J.bias[k]);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < CIN; ++k)
                        *reinterpret_cast<float *>(orowp + oph + (c * CIN + k) * 4) =
                            __fmaf_rn(v[k], J.scale[k], J.bias[k]);
                }
            }
        }
    }
    __syncthreads();

    // ---- 3. write-out: one warp per (plane, row), 16-byte chunks --------------------
    const int nplanes = chw ? NPL : 1;
    const int seglen = chw ? nx * 4 : nx * dC * ES;
    for (int s = warp; s < nplanes * ny; s += kWarps) {
        const int pl = s / ny, r = s - pl * ny;
        uint8_t *g = J.dst + (int64_t)(ty0 + r) * J.dpitch +
                     (chw ? (int64_t)pl * J.dplane + (int64_t)tx0 * 4 : (int64_t)tx0 * dC * ES);
        const int phase = (int)((uintptr_t)g & 15);
        uint8_t *G = g - phase;
        const uint8_t *S = ostage + (pl * TH + r) * orow;
        const int nch = (phase + seglen + 15) >> 4;
        for (int j = lane; j < nch; j += 32) {
            const int b0 = j * 16, b1 = b0 + 16;
            if (b0 >= phase && b1 <= phase + seglen) {
                *reinterpret_cast<uint4 *>(G + b0) = *reinterpret_cast<const uint4 *>(S + b0);
            } else {
                const int lo = max(b0, phase), hi = min(b1, phase + seglen);
                for (int b = lo; b < hi; ++b) G[b] = S[b];
            }
        }
    }
    __syncthreads();
}

}  // namespace kr
