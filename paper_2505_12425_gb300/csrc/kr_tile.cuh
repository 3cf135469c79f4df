// The one-tile-per-CTA engine of the resampling kernels (see kr_device.cuh for the steps
// and the arithmetic): plan, stage, compute, write-out of one TW x TH output tile.
#pragma once

#include "kr_quad.cuh"

namespace kr {

// ---------------------------------------------------------------------------
// The tile engine.
// ---------------------------------------------------------------------------
// The staging decision for the planned box ti; every thread takes it from the shared plan.
template <int OP, int CIN, bool ROWS, bool FRESH, int TW, int TH>
__device__ __forceinline__ TileDec decide_staging(const Job &J, const TileShared<TW, TH> &ts)
{
    const TileInfo &ti = ts.ti;
    TileDec d;
    const int fx0 = ti.fx0, fx1 = ti.fx1, fy0 = ti.fy0, fy1 = ti.fy1;
    d.rows = fy1 - fy0 + 1;
    d.cols = fx1 - fx0 + 1;
    d.srow = raw_row_bytes(max(d.cols, 1), CIN);
    d.sw = word_row(max(d.cols, 1));
    const bool zero_tile = OP != OP_RESIZE && ti.zero != 0;
    bool staged = !zero_tile && d.cols >= 1 && d.rows >= 1 && J.foot_budget > 0;
    // The staged box holds zeros outside the image: with the replicated border only boxes
    // inside the image are staged, the others take the general path.
    if (OP != OP_RESIZE && J.replicate && (fx0 < 0 || fy0 < 0 || fx1 > J.W - 1 || fy1 > J.H - 1)) staged = false;
    const int bph = (fx0 * CIN) & 15;   // 16-byte phase of the box in every row of 16-byte aligned rows
    const bool mbar_ok = FRESH || ts.mbar_ok != 0;
    // (1) one TMA copy when the launch has a source map whose box holds this tile's box
    const bool tma_fits =
        staged && mbar_ok && J.tin != nullptr && d.rows <= J.tin_br && bph + d.cols * CIN <= 16 * J.tin_nc;
    // (2) else one bulk copy per box row when the rows are 16-byte aligned and region A holds
    // the box (3 channels, raw taps)
    d.bnc = (bph + d.cols * CIN + 15) >> 4;
    const bool bulk_fits = ROWS && staged && mbar_ok && !tma_fits && CIN == 3 && J.raw_taps && J.rows16 &&
                           (long long)d.rows * 16 * d.bnc + 16 <= J.foot_budget;
    // Raw taps: 3-channel taps are read straight from rows staged by (1) or (2) (region A),
    // whose 16-byte phase is the same for every row.
    const bool rawbox = CIN == 3 && J.raw_taps && (tma_fits || bulk_fits);
    if (staged && !rawbox) {
        if (CIN == 3)
            staged = (long long)d.rows * d.sw * 4 <= J.foot_budget && (long long)d.rows * d.srow <= J.region_b;
        else
            staged = (long long)d.rows * d.srow + 16 <= J.foot_budget;
    }
    const bool fast = staged && (OP == OP_RESIZE || ti.fast != 0);   // resize taps always lie in the box
    const bool use_tma = staged && tma_fits;
    const bool use_bulk = staged && bulk_fits;
    d.rstride = use_tma ? 16 * J.tin_nc : use_bulk ? 16 * d.bnc : d.srow;
    d.flags = (zero_tile ? TD_ZERO : 0) | (staged ? TD_STAGED : 0) | (rawbox ? TD_RAWBOX : 0) | (fast ? TD_FAST : 0) |
              (use_tma ? TD_TMA : 0) | (use_bulk ? TD_BULK : 0);
    return d;
}

// One tile per CTA: the thread that planned the box takes the staging decision at once and, when
// the box is one TMA copy, initialises the staging barrier and starts the copy, so that the copy
// runs while the other threads finish the plan (the box's origin and size are the same values
// every thread later decides on).
template <int OP, int CIN, bool ROWS, int TW, int TH>
__device__ __forceinline__ void early_tma(const Job &J, TileShared<TW, TH> &ts, uint8_t *smem)
{
    const TileDec d = decide_staging<OP, CIN, ROWS, true>(J, ts);
    if (!(d.flags & TD_TMA)) return;
    uint8_t *raw = (CIN == 3 && !(d.flags & TD_RAWBOX)) ? smem + J.foot_budget : smem;
    mbar_init(&ts.mbar);
    ts.mbar_phase = 0;
    ts.mbar_ok = 1;
    mbar_expect_tx(&ts.mbar, (uint32_t)(16 * J.tin_nc * J.tin_br));
    tma_load_3d(raw, J.tin, 4 * ((ts.ti.fx0 * CIN) >> 4), ts.ti.fy0, J.zimg, &ts.mbar);
}

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
    // The thread that starts a one-tile CTA's box copy early (after planning the box itself).
    constexpr int kIssuer = (FRESH && OP == OP_RESIZE) ? (TW + TH + 31) / 32 * 32 : 0;
    if (OP == OP_RESIZE) {
        static_assert(TW + TH <= kThreads && (!FRESH || kIssuer + 32 <= kThreads),
                      "one axis entry per thread (and a spare warp for one-tile CTAs)");
        if (tid < TW) {
            int i0 = 0, i1 = 0, q = 0;
            float f = 0.f;
            if (tid < nx) {
                if (J.rm[0]) resize_axis_m(tx0 + tid, J.W, J.w, J.rm[0], J.rm[1], i0, i1, q, f);
                else resize_axis(tx0 + tid, J.W, J.w, i0, i1, q, f);
            }
            ts.cx0[tid] = i0; ts.cqd[tid] = q | ((i1 - i0) << 16); ts.cf[tid] = f;
        } else if (tid < TW + TH) {
            const int r = tid - TW;
            int i0 = 0, i1 = 0, q = 0;
            float f = 0.f;
            if (r < ny) {
                if (J.rm[0]) resize_axis_m(ty0 + r, J.H, J.h, J.rm[2], J.rm[3], i0, i1, q, f);
                else resize_axis(ty0 + r, J.H, J.h, i0, i1, q, f);
            }
            ts.ry0[r] = i0; ts.rqd[r] = q | ((i1 - i0) << 16); ts.rf[r] = f;
        } else if (FRESH && warp == kIssuer / 32) {
            // the box from the first and last column and row of the tile (their taps are the
            // tables' first and last entries; lanes 0..3 take one each), then its copy
            const bool col = lane < 2;
            const int i = col ? tx0 + (lane & 1) * (nx - 1) : ty0 + (lane & 1) * (ny - 1);
            int i0 = 0, i1 = 0, q = 0;
            float f = 0.f;
            if (lane < 4) {
                const int n_in = col ? J.W : J.H, n_out = col ? J.w : J.h;
                if (J.rm[0]) resize_axis_m(i, n_in, n_out, J.rm[col ? 0 : 2], J.rm[col ? 1 : 3], i0, i1, q, f);
                else resize_axis(i, n_in, n_out, i0, i1, q, f);
            }
            const int b0 = __shfl_sync(0xffffffffu, i0, 0), b1 = __shfl_sync(0xffffffffu, i1, 1);
            const int b2 = __shfl_sync(0xffffffffu, i0, 2), b3 = __shfl_sync(0xffffffffu, i1, 3);
            if (lane == 0) {
                ti.fx0 = b0;
                ti.fx1 = b1;
                ti.fy0 = b2;
                ti.fy1 = b3;
                early_tma<OP, CIN, ROWS>(J, ts, smem);
            }
        }
        if (!FRESH) {
            __syncthreads();
            if (tid == 0) {
                ti.fx0 = ts.cx0[0];
                ti.fx1 = ts.cx0[nx - 1] + (ts.cqd[nx - 1] >> 16);
                ti.fy0 = ts.ry0[0];
                ti.fy1 = ts.ry0[ny - 1] + (ts.rqd[ny - 1] >> 16);
            }
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
            if (FRESH) early_tma<OP, CIN, ROWS>(J, ts, smem);
        }
    }
    __syncthreads();
    // Every thread derives the staging decision from the planned box (no extra barrier).
    const int fx0 = ti.fx0, fx1 = ti.fx1, fy0 = ti.fy0, fy1 = ti.fy1;
    const TileDec dec = decide_staging<OP, CIN, ROWS, FRESH>(J, ts);
    const int rows = dec.rows, cols = dec.cols, sw = dec.sw, bnc = dec.bnc;
    const bool zero_tile = (dec.flags & TD_ZERO) != 0;
    bool staged = (dec.flags & TD_STAGED) != 0;
    const bool rawbox = (dec.flags & TD_RAWBOX) != 0;
    const bool fast = (dec.flags & TD_FAST) != 0;
    const bool use_tma = (dec.flags & TD_TMA) != 0;
    const bool use_bulk = (dec.flags & TD_BULK) != 0;
    const int rstride = dec.rstride;
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
            if (tid == kIssuer) {
                if (!FRESH) {   // (one tile per CTA: started right after the plan)
                    mbar_expect_tx(&ts.mbar, (uint32_t)(16 * J.tin_nc * J.tin_br));
                    tma_load_3d(raw, J.tin, 4 * ((fx0 * CIN) >> 4), fy0, J.zimg, &ts.mbar);
                }
                stage_wait(ts, J.err, J.wait_ns);
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
                if (lane == 0) stage_wait(ts, J.err, J.wait_ns);
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
    // output stage rows (tiles not written straight to global memory), with room for each
    // row's 16-byte phase
    const int orow = chw ? round16(TW * 4 + 15) : round16(TW * dC * ES + 15);
    // low address bits of output row 0 of the tile (plane 0): staging rows keep their phase
    const uint32_t obase = (uint32_t)(uintptr_t)(J.dst + (int64_t)ty0 * J.dpitch +
                                                 (chw ? (int64_t)tx0 * 4 : (int64_t)tx0 * dC * ES));
    const uint32_t opitch = (uint32_t)J.dpitch, oplane = (uint32_t)J.dplane;
    // Rows that are whole 16-byte chunks are written straight to global memory by every path
    // (the quad path with 4- or 16-byte stores, the others pixel by pixel): no output stage.
    const bool direct = J.direct != 0;
    int r0 = 0;   // first tile row of the current band
    auto orow_of = [&](int r) -> ORow {
        ORow o;
        if (direct) {
            uint8_t *g = J.dst + (int64_t)(ty0 + r) * J.dpitch + (chw ? (int64_t)tx0 * 4 : (int64_t)tx0 * dC * ES);
            o.p0 = g;
            o.p1 = chw ? g + J.dplane : nullptr;
            o.p2 = chw ? g + 2 * J.dplane : nullptr;
            return o;
        }
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

    const bool quad = CIN == 3 && TW == 64 && fast && rawbox && nx == TW;
    if constexpr (CIN == 3 && TW == 64) {
        if (quad && direct) {
            // each lane stores its 4 pixels straight to global memory, all rows of the tile in
            // one pass, with no barrier after the staging one
            const int half = lane >> 4, cb = 4 * (lane & 15);
            const uint32_t sraw = (uint32_t)(raw - smem);
            QuadTile T;
            quad_setup<OP, OUTK>(T, J, ts.cx0, ts.cqd, ts.cf, tx0, fx0, fy0, rstride, sraw, rph, cb, nx);
            uint8_t *g = J.dst + (int64_t)ty0 * J.dpitch + (chw ? (int64_t)tx0 * 4 : (int64_t)tx0 * dC * ES);
            for (int r = 2 * warp + half; r < ny; r += 2 * kWarps) {
                QuadOut<OUTK> Q;
                quad_eval<OP, OUTK>(Q, T, J, ts.ry0, ts.rqd, ts.rf, r, ty0, fy0, rstride);
                quad_store_global<OUTK>(Q, J, chw, g + (int64_t)r * J.dpitch, J.dplane, cb);
            }
            return;
        }
    }
    for (int band = 0; band < (direct ? 1 : NBAND); ++band) {
        r0 = band * BH;
        if (r0 >= ny) break;
        const int r1 = direct ? ny : min(ny, r0 + BH);
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
        } else if (quad) {
            // Full-width tile with raw taps: each lane blends 4 adjacent pixels of a row (half-
            // warps on neighbouring rows) and stores them as packed words.
            if constexpr (CIN == 3 && TW == 64) {
                const int half = lane >> 4, cb = 4 * (lane & 15);
                const uint32_t sraw = (uint32_t)(raw - smem);
                const uint32_t sost = (uint32_t)(ostage - smem);
                QuadTile T;
                quad_setup<OP, OUTK>(T, J, ts.cx0, ts.cqd, ts.cf, tx0, fx0, fy0, rstride, sraw, rph, cb, nx);
                for (int rr = 2 * warp + half; rr < BH; rr += 2 * kWarps) {
                    const int r = r0 + rr;
                    if (r >= r1) break;
                    auto off = [&](int pl) -> uint32_t {
                        const uint32_t a = obase + (uint32_t)r * opitch + (uint32_t)pl * oplane;
                        return sost + (uint32_t)((pl * BH + rr) * orow) + (a & 15u);
                    };
                    quad_row<OP, OUTK>(T, J, ts.ry0, ts.rqd, ts.rf, r, ty0, fy0, rstride, sraw, chw, off(0),
                                       chw ? off(1) : 0u, chw ? off(2) : 0u, cb);
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
                        } else if (CIN == 3 && !(OP != OP_RESIZE && J.replicate) && dx == 1 && dy == 1 &&
                                   x0 >= 0 && x0 + 1 < J.W && y0 >= 0 && y0 + 2 < J.H &&
                                   (((uintptr_t)J.src | (uintptr_t)J.spitch) & 3) == 0) {
                            // both taps inside and both rows followed by a row of the image: each
                            // row's pair from three aligned words (at most 11 bytes past the pair,
                            // inside the next row), read as a raw pair
                            const uint8_t *a = J.src + (int64_t)y0 * J.spitch + 3 * x0;
                            const uint32_t *w0 = reinterpret_cast<const uint32_t *>((uintptr_t)a & ~(uintptr_t)3);
                            const uint32_t *w1 = reinterpret_cast<const uint32_t *>((uintptr_t)(a + J.spitch) & ~(uintptr_t)3);
                            const uint32_t sh8 = (uint32_t)(uintptr_t)a << 3;
                            p00 = __funnelshift_r(__ldg(w0), __ldg(w0 + 1), sh8);
                            p01 = __funnelshift_r(__ldg(w0 + 1), __ldg(w0 + 2), sh8);
                            p10 = __funnelshift_r(__ldg(w1), __ldg(w1 + 1), sh8);
                            p11 = __funnelshift_r(__ldg(w1 + 1), __ldg(w1 + 2), sh8);
                            emit<CIN, OUTK, TAPS_RAW>(J, o, c, p00, p01, p10, p11, qx, qy, fx, fy);
                            continue;
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
        if (direct) return;   // (written straight to global memory)
        __syncthreads();

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
