// Warp-specialised persistent tile pipeline of the 3-channel resampling kernels: bilinear
// resize and the affine and perspective warps of Sec. III / Sec. II-A, with the fused gray
// and u8 -> f32 normalisation epilogues of Sec. III (arithmetic as in kr_device.cuh).
//
// A CTA holds kPipeConsumers threads (8 warps) that blend tiles and one producer warp that
// runs ahead of them over the CTA's tiles (claimed from the launch's tile counter):
//
//   producer  for tile k: plan the tile (resize axis tables, or the warp map at the four tile
//             corners -> source box; fast flag; staging mode), wait until ring slot
//             s = k mod NS is free ("empty" mbarrier, one arrival per consumer warp), write the
//             plan into the slot, start the copy of the box into the slot's staging buffer (one TMA tensor copy,
//             or one bulk copy per box row with the bytes the copies do not cover written by
//             the warp: zeros outside the image, the row's last partial 16-byte chunk), then
//             every lane arrives on the slot's "full" mbarrier (which also completes on the
//             copies' bytes);
//   consumers each warp waits on "full" by itself, blends its units of the tile (4 rows for
//             u8, 2 for f32) from the staged raw rows (the quad path, or the exact per-pixel
//             weights for a tile outside the fast forms' range) or, for a tile that is not
//             staged, from global memory, writes u8 rows straight to global memory and f32 units
//             through its own two unit stages in turn (bulk copies of each row's aligned
//             middle, head and tail bytes by lanes), and releases the slot when it has read it.
//
// While tile k is blended the copies of tiles k+1 .. k+NS-1 are in flight, and the bulk
// stores of a unit drain while the warp blends the next: no CTA-wide barrier after set-up.
// Every wait sleeps on its mbarrier and is bounded: a staging wait that runs out sets error
// bit 0, waits once more (bounded) for the copies to land and abandons the warp's rows of
// the tile without writing them; if that also runs out the warp stops.
#pragma once

#include "kr_quad.cuh"

namespace kr {

constexpr int kPipeConsumers = 256;
constexpr int kPipeThreads = kPipeConsumers + 32;

enum { PM_END = 0, PM_ZERO = 1, PM_STAGED = 2, PM_GLOBAL = 3 };

// A planned tile, written by the producer and read by the consumers.
template <int TW, int TH> struct PipeSlot {
    int mode;                 // PM_*
    int job;                  // image of the launch / item of the work list
    int tx0, ty0;             // first output column and row of the tile
    int fx0, fy0, fx1, fy1;   // source box (inclusive)
    int rstride;              // bytes between staged rows
    int fast;                 // every coordinate of the tile is in the fast forms' range
    int clamp;                // replicated border: box clipped to the image, taps clamped
    int pad;
    int cx0[TW];              // resize: column tap x0
    int cqd[TW];              //         q | (x1 - x0) << 16
    float cf[TW];             //         fp32 weight of x1
    int ry0[TH];
    int rqd[TH];
    float rf[TH];
};

template <int TW, int TH, int NS> struct PipeShared {
    uint64_t full[NS];
    uint64_t empty[NS];
    PipeSlot<TW, TH> slot[NS];
};

// ---------------------------------------------------------------------------
// Synchronisation helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init_count(uint64_t *mbar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// Plain arrive (release): the calling thread's earlier writes are visible to a thread whose
// wait on this phase succeeds.
__device__ __forceinline__ void mbar_arrive(uint64_t *mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(mbar)) : "memory");
}

// Raise the phase's expected transaction bytes without arriving.
__device__ __forceinline__ void mbar_expect_bytes(uint64_t *mbar, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(mbar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }

// try_wait that may suspend the thread until the phase completes or hint_ns pass.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *mbar, uint32_t parity, uint32_t hint_ns)
{
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done)
                 : "r"(smem_addr(mbar)), "r"(parity), "r"(hint_ns)
                 : "memory");
    return done != 0;
}

// Wait for phase `parity`, sleeping on the barrier between checks of the bound limit_ns (so a
// waiting warp takes no issue slots from the warps that work).
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t *mbar, uint32_t parity, uint64_t limit_ns)
{
    if (mbar_try_wait(mbar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait_sleep(mbar, parity, 1000000u))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

// First wait of a staging slot: limit_ns = 0 gives up at once (used to test the timeout
// path), otherwise the wait is bounded by limit_ns.
__device__ __forceinline__ bool pipe_first_wait(uint64_t *mbar, uint32_t parity, uint64_t limit_ns)
{
    if (limit_ns == 0) return false;
    return mbar_wait_sleep(mbar, parity, limit_ns);
}

// ---------------------------------------------------------------------------
// Producer
// ---------------------------------------------------------------------------
// Pol provides (warp-uniform):
//   bool tile(int k, int lane, int &job, int &tx, int &ty)   the CTA's k-th tile (k = 0, 1, ...
//                                                            in order), false past the last
//   void job(int job, Job &J)                                the tile's image
//   unsigned *err()                                          device error flags
//   kSameGeometry                                            every job of the launch has the same
//                                                            sizes (resize column tables depend
//                                                            on the tile column only)
template <int OP, int TW, int TH, int NS, class Pol>
__device__ __forceinline__ void pipe_produce(Pol &P, PipeShared<TW, TH, NS> &sh, uint8_t *stage0, int stage_bytes)
{
    constexpr int CPL = TW / 32, RPL = (TH + 31) / 32;
    const int lane = threadIdx.x & 31;
    Job J;
    int cur_job = -1;                             // image held in J
    bool small = false;                           // resize: every size below 2^15
    uint32_t mx1 = 0, mx2 = 0, my1 = 0, my2 = 0;  // floor((2^32-1)/d) for d = 2w, 4w, 2h, 4h
    int col_tx = -1, col_job = -1;                // resize: tile column (and job) of the held column entries
    int ccx[CPL], ccq[CPL], crx[RPL], crq[RPL];
    float ccf[CPL], crf[RPL];
    // The tile is planned before its slot is free (the plan's loads overlap the consumers'
    // work); only the slot's writes and the copies wait for the slot.
    auto wait_slot = [&](int k) -> bool {
        if (k < NS) return true;
        int ok = 1;
        if (lane == 0) ok = mbar_wait_sleep(&sh.empty[k % NS], (uint32_t)((k / NS) - 1) & 1u, kTmaWaitNs) ? 1 : 0;
        if (__shfl_sync(0xffffffffu, ok, 0)) return true;
        if (lane == 0) atomicOr(P.err(), 1u);
        return false;
    };
    for (int k = 0;; ++k) {
        const int s = k % NS;
        PipeSlot<TW, TH> &sl = sh.slot[s];
        int job = 0, tx = 0, ty = 0;
        if (!P.tile(k, lane, job, tx, ty)) {
            if (!wait_slot(k)) return;
            if (lane == 0) sl.mode = PM_END;
            mbar_arrive(&sh.full[s]);
            return;
        }
        if (job != cur_job) {
            P.job(job, J);
            cur_job = job;
            if (OP == OP_RESIZE) {
                small = J.W < 32768 && J.w < 32768 && J.H < 32768 && J.h < 32768;
                // lanes 0..3 each take one reciprocal
                const uint32_t d = lane == 0 ? 2u * J.w : lane == 1 ? 4u * J.w : lane == 2 ? 2u * J.h : 4u * J.h;
                const uint32_t m = (small && lane < 4) ? 0xFFFFFFFFu / d : 0u;
                mx1 = __shfl_sync(0xffffffffu, m, 0);
                mx2 = __shfl_sync(0xffffffffu, m, 1);
                my1 = __shfl_sync(0xffffffffu, m, 2);
                my2 = __shfl_sync(0xffffffffu, m, 3);
            }
        }
        const int tx0 = tx * TW, ty0 = ty * TH;
        const int nx = min(TW, J.w - tx0), ny = min(TH, J.h - ty0);

        // ---- plan: the tile's source box ----
        int fx0 = 0, fx1 = -1, fy0 = 0, fy1 = -1, fast = 0, zero = 0, clamp = 0;
        if (OP == OP_RESIZE) {
            // column entries are held in registers and rewritten into every slot; they are
            // recomputed only when the tile column (or, across different sizes, the job) changes
            if (tx != col_tx || (!Pol::kSameGeometry && job != col_job)) {
#pragma unroll
                for (int j = 0; j < CPL; ++j) {
                    const int c = lane + 32 * j;
                    int i0 = 0, i1 = 0, q = 0;
                    float f = 0.f;
                    if (c < nx) {
                        if (small) resize_axis_m(tx0 + c, J.W, J.w, mx1, mx2, i0, i1, q, f);
                        else resize_axis(tx0 + c, J.W, J.w, i0, i1, q, f);
                    }
                    ccx[j] = i0;
                    ccq[j] = q | ((i1 - i0) << 16);
                    ccf[j] = f;
                }
                col_tx = tx;
                col_job = job;
            }
#pragma unroll
            for (int j = 0; j < RPL; ++j) {
                const int r = lane + 32 * j;
                int i0 = 0, i1 = 0, q = 0;
                float f = 0.f;
                if (r < ny) {
                    if (small) resize_axis_m(ty0 + r, J.H, J.h, my1, my2, i0, i1, q, f);
                    else resize_axis(ty0 + r, J.H, J.h, i0, i1, q, f);
                }
                crx[j] = i0;
                crq[j] = q | ((i1 - i0) << 16);
                crf[j] = f;
            }
            // the box from the first and last entries of both tables
            int lx = ccx[0], lq = ccq[0], ly = crx[0], lr = crq[0];
#pragma unroll
            for (int j = 1; j < CPL; ++j)
                if (j == ((nx - 1) >> 5)) { lx = ccx[j]; lq = ccq[j]; }
#pragma unroll
            for (int j = 1; j < RPL; ++j)
                if (j == ((ny - 1) >> 5)) { ly = crx[j]; lr = crq[j]; }
            fx0 = __shfl_sync(0xffffffffu, ccx[0], 0);
            fx1 = __shfl_sync(0xffffffffu, lx + (lq >> 16), (nx - 1) & 31);
            fy0 = __shfl_sync(0xffffffffu, crx[0], 0);
            fy1 = __shfl_sync(0xffffffffu, ly + (lr >> 16), (ny - 1) & 31);
            fast = 1;
        } else {
            // lanes 0..3 map one tile corner each; the box is their hull, one pixel wider on
            // the low side and three on the high side (floor, second tap, the fast form's
            // pair, fp32 rounding of interior pixels). Perspective: Z is affine in the pixel
            // position, so Z > 0 at the corners means Z > 0 over the tile, and the tile maps
            // onto the convex hull of its corners' images.
            const int cx = (lane & 1) ? tx0 + nx - 1 : tx0, cy = (lane & 2) ? ty0 + ny - 1 : ty0;
            float sx = 0.f, sy = 0.f;
            bool ok = true;
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
            mnx = __shfl_sync(0xffffffffu, mnx, 0);
            mxx = __shfl_sync(0xffffffffu, mxx, 0);
            mny = __shfl_sync(0xffffffffu, mny, 0);
            mxy = __shfl_sync(0xffffffffu, mxy, 0);
            if (__all_sync(0xffffffffu, ok)) {
                // not clipped to the image: the staged box is zero outside it (zero border)
                fx0 = (int)floorf(mnx) - 1;
                fx1 = (int)floorf(mxx) + 3;
                fy0 = (int)floorf(mny) - 1;
                fy1 = (int)floorf(mxy) + 3;
                zero = !J.replicate && (fx1 < 0 || fx0 > J.W - 1 || fy1 < 0 || fy0 > J.H - 1);
                fast = J.allow_fast && mnx >= 1.f && mny >= 1.f && mxx < 4093.f && mxy < 4093.f;
                if (J.replicate && (fx0 < 0 || fy0 < 0 || fx1 > J.W - 1 || fy1 > J.H - 1)) {
                    // a tap clamped into the image lies in the box clipped to the image
                    fx0 = min(max(fx0, 0), J.W - 1);
                    fx1 = min(max(fx1, 0), J.W - 1);
                    fy0 = min(max(fy0, 0), J.H - 1);
                    fy1 = min(max(fy1, 0), J.H - 1);
                    clamp = 1;
                    fast = 0;
                }
            }
        }

        // ---- staging mode ----
        const int rows = fy1 - fy0 + 1, cols = fx1 - fx0 + 1;
        const int bph = (fx0 * 3) & 15;                 // 16-byte phase of the box in its rows
        const int bnc = (bph + cols * 3 + 15) >> 4;    // 16-byte chunks of a box row
        bool staged = !zero && cols >= 1 && rows >= 1 && J.raw_taps;
        const bool tma = staged && J.tin != nullptr && rows <= J.tin_br && bph + cols * 3 <= 16 * J.tin_nc;
        const bool bulk = staged && !tma && J.rows16 && (long long)rows * 16 * bnc + 16 <= stage_bytes;
        staged = tma || bulk;
        const int mode = zero ? PM_ZERO : staged ? PM_STAGED : PM_GLOBAL;
        const int rstride = tma ? 16 * J.tin_nc : 16 * bnc;

        // ---- the slot is free: write it, start the copies ----
        if (!wait_slot(k)) return;
        if (OP == OP_RESIZE) {
#pragma unroll
            for (int j = 0; j < CPL; ++j) {
                sl.cx0[lane + 32 * j] = ccx[j];
                sl.cqd[lane + 32 * j] = ccq[j];
                sl.cf[lane + 32 * j] = ccf[j];
            }
#pragma unroll
            for (int j = 0; j < RPL; ++j) {
                const int r = lane + 32 * j;
                if (r < TH) {
                    sl.ry0[r] = crx[j];
                    sl.rqd[r] = crq[j];
                    sl.rf[r] = crf[j];
                }
            }
        }
        if (lane == 0) {
            sl.mode = mode;
            sl.job = job;
            sl.tx0 = tx0;
            sl.ty0 = ty0;
            sl.fx0 = fx0;
            sl.fy0 = fy0;
            sl.fx1 = fx1;
            sl.fy1 = fy1;
            sl.rstride = rstride;
            sl.fast = staged && fast;
            sl.clamp = clamp;
        }

        // ---- start the copies ----
        uint8_t *stage = stage0 + s * stage_bytes;
        if (tma) {
            if (lane == 0) {
                mbar_expect_bytes(&sh.full[s], (uint32_t)(16 * J.tin_nc * J.tin_br));
                tma_load_3d(stage, J.tin, 4 * ((fx0 * 3) >> 4), fy0, J.zimg, &sh.full[s]);
            }
        } else if (bulk) {
            // Box row r is the row's bytes [xb0, xb1). The whole chunks of the row inside the
            // image, [c0, c1), come by one bulk copy; the warp writes the rest: zeros outside
            // the image (the warp's zero border; resize never reads there) and the bytes of
            // the row's last partial chunk [F, 3W).
            const int xb0 = 16 * ((fx0 * 3) >> 4), xb1 = xb0 + 16 * bnc;
            const int F = (J.W * 3) & ~15;
            const int c0 = max(xb0, 0), c1 = min(xb1, F);
            uint32_t bytes = 0;
            if (c1 > c0)
                for (int r = lane; r < rows; r += 32)
                    if ((unsigned)(fy0 + r) < (unsigned)J.H) bytes += (uint32_t)(c1 - c0);
            bytes = warp_sum(bytes);
            if (lane == 0 && bytes) mbar_expect_bytes(&sh.full[s], bytes);
            __syncwarp();
            if (c1 > c0)
                for (int r = lane; r < rows; r += 32) {
                    const int y = fy0 + r;
                    if ((unsigned)y < (unsigned)J.H)
                        bulk_load(stage + r * rstride + (c0 - xb0), J.src + (int64_t)y * J.spitch + c0,
                                  (uint32_t)(c1 - c0), &sh.full[s]);
                }
            if (!(fy0 >= 0 && fy1 < J.H && xb0 >= 0 && xb1 <= F)) {
                // a lane per box row: rows outside the image are zeros; inside, the chunks left
                // of the image are zeros and those from F on hold the row's last bytes [F, 3W)
                // (one 16-byte load, the bytes past the row masked to zero: every row but the
                // image's last is followed by at least its 16-byte aligned pitch; the last row
                // byte by byte) and zeros after them
                const int L3 = J.W * 3;
                for (int r = lane; r < rows; r += 32) {
                    const int y = fy0 + r;
                    uint8_t *srow = stage + r * rstride;
                    if ((unsigned)y >= (unsigned)J.H) {
                        for (int j = 0; j < bnc; ++j) *reinterpret_cast<uint4 *>(srow + 16 * j) = make_uint4(0u, 0u, 0u, 0u);
                        continue;
                    }
                    for (int b0 = xb0; b0 < min(0, xb1); b0 += 16)
                        *reinterpret_cast<uint4 *>(srow + (b0 - xb0)) = make_uint4(0u, 0u, 0u, 0u);
                    const uint8_t *grow = J.src + (int64_t)y * J.spitch;
                    for (int b0 = max(F, xb0); b0 < xb1; b0 += 16) {
                        uint4 v = make_uint4(0u, 0u, 0u, 0u);
                        if (b0 < L3) {
                            const int n = L3 - b0;   // bytes of the row in this chunk, 1..15
                            if (y < J.H - 1) {
                                v = __ldg(reinterpret_cast<const uint4 *>(grow + b0));
                                const uint32_t m[4] = {n >= 4 ? ~0u : (1u << (8 * n)) - 1u,
                                                       n >= 8 ? ~0u : n <= 4 ? 0u : (1u << (8 * (n - 4))) - 1u,
                                                       n >= 12 ? ~0u : n <= 8 ? 0u : (1u << (8 * (n - 8))) - 1u,
                                                       n <= 12 ? 0u : (1u << (8 * (n - 12))) - 1u};
                                v.x &= m[0];
                                v.y &= m[1];
                                v.z &= m[2];
                                v.w &= m[3];
                            } else {
                                uint32_t w[4] = {0u, 0u, 0u, 0u};
                                for (int q = 0; q < n; ++q) w[q >> 2] |= (uint32_t)__ldg(grow + b0 + q) << (8 * (q & 3));
                                v = make_uint4(w[0], w[1], w[2], w[3]);
                            }
                        }
                        *reinterpret_cast<uint4 *>(srow + (b0 - xb0)) = v;
                    }
                }
            }
        }
        // every lane arrives: releases the slot's plan, tables and the lanes' own writes
        mbar_arrive(&sh.full[s]);
    }
}

// ---------------------------------------------------------------------------
// Consumers
// ---------------------------------------------------------------------------
// A unit is UR adjacent output rows of a tile, owned by one consumer warp: each half-warp
// takes every other row of it, its 16 lanes 4 columns each (TW = 64). Warp w takes rows
// UR w .. UR w + UR - 1, then the rows 8 UR further down. Each warp writes its u8 rows straight
// to global memory, and blends f32 units into its own two unit stages in turn, writing each
// unit out itself: the consumer warps never wait for one another.

// Rows of a unit: u8 kinds 4, f32 kinds 2.
template <int OUTK> __host__ __device__ constexpr int pipe_unit_rows()
{
    return OutTraits<OUTK, 3>::is_f32 ? 2 : 4;
}

// Bytes of one unit stage (UR rows; three planes of UR rows for planar f32), a multiple of 128.
template <int OUTK, int TW> __host__ __device__ constexpr int pipe_unit_bytes()
{
    // (u8 rows go straight to global memory: no unit stage)
    return (OUTK == OUT_U8 || OUTK == OUT_U8_GRAY) ? 0
           : (OutTraits<OUTK, 3>::is_f32 && OutTraits<OUTK, 3>::dC == 3)
               ? (((pipe_unit_rows<OUTK>() * round16(TW * 12 + 15) > 3 * pipe_unit_rows<OUTK>() * round16(TW * 4 + 15)
                        ? pipe_unit_rows<OUTK>() * round16(TW * 12 + 15)
                        : 3 * pipe_unit_rows<OUTK>() * round16(TW * 4 + 15)) + 127) & ~127)
               : ((pipe_unit_rows<OUTK>() * round16(TW * OutTraits<OUTK, 3>::dC * OutTraits<OUTK, 3>::esize + 15) + 127) &
                  ~127);
}

__device__ __forceinline__ void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory"); }

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned) from shared to
// global memory, in the thread's current bulk group.
__device__ __forceinline__ void bulk_store(void *gdst, const void *ssrc, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(reinterpret_cast<uint64_t>(gdst)),
                 "r"(smem_addr(ssrc)), "r"(bytes)
                 : "memory");
}

template <int OP, int OUTK, int TW, int TH, int NS, class Pol>
__device__ __forceinline__ void pipe_consume(Pol &P, PipeShared<TW, TH, NS> &sh, int stage_bytes, int obuf_off,
                                             int unit_bytes)
{
    using OT = OutTraits<OUTK, 3>;
    constexpr int UR = pipe_unit_rows<OUTK>();
    static_assert(TW == 64 && TH % (8 * UR) == 0, "a half-warp covers a 64-column row, 8 warps 8 units");
    constexpr int CIN = 3;
    constexpr int dC = OT::dC;
    constexpr int ES = OT::esize;
    constexpr int NWARP = kPipeConsumers / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int half = lane >> 4, l16 = lane & 15, cb = 4 * l16;
    const uint64_t first_limit = P.first_wait_ns();
    const uint32_t wbuf = (uint32_t)(obuf_off + 2 * warp * unit_bytes);   // this warp's two unit stages
    int u = 0;   // units written by this warp: unit u uses stage u & 1
    for (int k = 0;; ++k) {
        const int s = k % NS;
        const uint32_t par = (uint32_t)(k / NS) & 1u;
        bool ok = pipe_first_wait(&sh.full[s], par, first_limit);
        if (!__all_sync(0xffffffffu, ok)) {
            // a wait ran out: record it, wait (bounded) for the slot's copies, abandon the tile
            if (lane == 0) atomicOr(P.err(), 1u);
            if (!ok) ok = mbar_wait_sleep(&sh.full[s], par, kTmaWaitNs);
            if (!__all_sync(0xffffffffu, ok)) break;   // copies may still land: stop
            if (sh.slot[s].mode == PM_END) break;
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh.empty[s]);
            continue;
        }
        const PipeSlot<TW, TH> &sl = sh.slot[s];
        const int mode = sl.mode;
        if (mode == PM_END) break;
        Job J;
        P.job(sl.job, J);
        const int tx0 = sl.tx0, ty0 = sl.ty0;
        const int nx = min(TW, J.w - tx0), ny = min(TH, J.h - ty0);
        const int fx0 = sl.fx0, fy0 = sl.fy0;
        const int rstride = sl.rstride;
        const bool fast = sl.fast != 0, clamp = sl.clamp != 0;
        const uint32_t sraw = (uint32_t)(s * stage_bytes);
        const uint8_t *raw = kr_pipe_smem + sraw;
        const int rph = (fx0 * 3) & 15;   // phase of every staged row
        const bool chw = OT::is_f32 && dC == 3 && J.chw;
        const int orow = chw ? round16(TW * 4 + 15) : round16(TW * dC * ES + 15);
        const uint32_t obase = (uint32_t)(uintptr_t)(J.dst + (int64_t)ty0 * J.dpitch +
                                                     (chw ? (int64_t)tx0 * 4 : (int64_t)tx0 * dC * ES));
        const uint32_t opitch = (uint32_t)J.dpitch, oplane = (uint32_t)J.dplane;
        // staged fast tiles take the quad path, full width or not (quad_setup); zero tiles write
        // the zero sample in the same layout
        const bool quad = mode == PM_STAGED && fast;

        QuadTile T;
        if (quad) quad_setup<OP, OUTK>(T, J, sl.cx0, sl.cqd, sl.cf, tx0, fx0, fy0, rstride, sraw, rph, cb, nx);

        // u8 rows of quad and zero tiles go straight to global memory (aligned 4-byte stores
        // built across each half-warp, any row alignment): no unit stage, no write-out
        constexpr bool kRunKind = OUTK == OUT_U8 || OUTK == OUT_U8_GRAY;
        const bool run = kRunKind && (quad || mode == PM_ZERO);
        if constexpr (kRunKind) {
            if (run) {
                constexpr int NW = QuadWords<OUTK>::n;
                for (int ra = UR * warp; ra < ny; ra += UR * NWARP) {
#pragma unroll 1
                    for (int hr = half; hr < UR; hr += 2) {
                        const int r = ra + hr;
                        const bool live = r < ny;
                        uint32_t w[NW];
#pragma unroll
                        for (int i = 0; i < NW; ++i) w[i] = 0u;
                        if (live && quad) {
                            QuadOut<OUTK> Q;
                            quad_eval<OP, OUTK>(Q, T, J, sl.ry0, sl.rqd, sl.rf, r, ty0, fy0, rstride);
                            quad_pack_u8<OUTK>(Q, w);
                        }
                        uint8_t *g = live ? J.dst + (int64_t)(ty0 + r) * J.dpitch + (int64_t)tx0 * dC : J.dst;
                        store_run_u8<NW>(g, live ? nx * dC : 0, w, l16);
                    }
                }
            }
        }
        for (int ra = UR * warp; ra < (run ? 0 : ny); ra += UR * NWARP) {
            const uint32_t ub = wbuf + (uint32_t)((u & 1) * unit_bytes);
            // byte offset of (tile row ra + h, plane pl) in the unit stage, keeping the 16-byte
            // phase of the row in global memory
            auto row_off = [&](int h, int pl) -> uint32_t {
                const uint32_t a = obase + (uint32_t)(ra + h) * opitch + (uint32_t)pl * oplane;
                return ub + (uint32_t)((pl * UR + h) * orow) + (a & 15u);
            };
            auto orow_of = [&](int h) -> ORow {
                ORow o;
                if (kRunKind) {   // u8: straight to the destination row
                    o.p0 = J.dst + (int64_t)(ty0 + ra + h) * J.dpitch + (int64_t)tx0 * dC;
                    o.p1 = o.p2 = nullptr;
                    return o;
                }
                o.p0 = kr_pipe_smem + row_off(h, 0);
                if (chw) {
                    o.p1 = kr_pipe_smem + row_off(h, 1);
                    o.p2 = kr_pipe_smem + row_off(h, 2);
                } else {
                    o.p1 = o.p2 = nullptr;
                }
                return o;
            };
#pragma unroll 1
            for (int hr = half; hr < UR; hr += 2) {
            const int r = ra + hr;   // this half-warp's tile row
            if (r < ny) {
                if (quad) {
                    quad_row<OP, OUTK>(T, J, sl.ry0, sl.rqd, sl.rf, r, ty0, fy0, rstride, sraw, chw, row_off(hr, 0),
                                       chw ? row_off(hr, 1) : 0u, chw ? row_off(hr, 2) : 0u, cb);
                } else if (mode == PM_ZERO) {
                    // every tap lies outside the image: the zero sample, 0 for u8 and
                    // (0 - mean[c]) / std[c] = bias[c] for f32 (bias[0] for gray): the quad store of
                    // zero interpolants
                    QuadOut<OUTK> Z;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        Z.u[j].r = Z.u[j].g = Z.u[j].b = 0u;
                        Z.f[j][0] = Z.f[j][1] = Z.f[j][2] = 0.f;
                    }
                    quad_store<OUTK>(Z, J, chw, row_off(hr, 0), chw ? row_off(hr, 1) : 0u, chw ? row_off(hr, 2) : 0u, cb);
                } else {
                    // per-pixel paths: columns l16 + 16 j of row r
                    const ORow o = orow_of(hr);
                    const int y = ty0 + r;
                    if (OP != OP_RESIZE && mode == PM_STAGED && clamp) {
                        // replicated border, footprint crossing the image's edge: the box is the
                        // footprint clipped to the image; each tap is clamped into the image
                        const int bx = J.W - 1 - fx0, by = J.H - 1 - fy0;   // box-relative image edges
                        auto px_at = [&](int yb, int xb) -> uint32_t {
                            const int off = yb * rstride + rph + 3 * xb;
                            const uint32_t *wp = reinterpret_cast<const uint32_t *>(raw + (off & ~3));
                            return __funnelshift_r(wp[0], wp[1], (uint32_t)off << 3);
                        };
#pragma unroll
                        for (int j = 0; j < TW / 16; ++j) {
                            const int c = l16 + 16 * j;
                            if (c >= nx) continue;
                            float sx, sy;
                            map_coord<OP>(J.M, tx0 + c, y, sx, sy);   // valid: the tile's corners are
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
                            emit<CIN, OUTK>(J, o, c, px_at(ya, xa), px_at(ya, xb), px_at(yb, xa), px_at(yb, xb), qx,
                                            qy, fx, fy);
                        }
                    } else if (OP != OP_RESIZE && mode == PM_STAGED) {
                        // staged tile outside the fast forms' range (its box crosses the image's
                        // edge): the exact weight formula per pixel, every tap read from the
                        // zero-filled box
                        const float yc = __fadd_rn((float)y, 0.5f);
                        const float rx = __fmaf_rn(J.M[1], yc, J.M[2]), ry = __fmaf_rn(J.M[4], yc, J.M[5]);
#pragma unroll
                        for (int j = 0; j < TW / 16; ++j) {
                            const int c = l16 + 16 * j;
                            if (c >= nx) continue;
                            float sx, sy;
                            if (OP == OP_PERSP) {
                                persp_coord(J.M, tx0 + c, y, sx, sy);   // valid: Z > 0 over the tile
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
                            const int off = (y0 - fy0) * rstride + 3 * (x0 - fx0) + rph;
                            const uint8_t *wp = raw + (off & ~3);
                            const uint32_t sh = (uint32_t)off << 3;
                            uint32_t p00, p01, p10, p11;
                            raw_pair(wp, sh, p00, p01);
                            raw_pair(wp + rstride, sh, p10, p11);
                            emit<CIN, OUTK, TAPS_RAW>(J, o, c, p00, p01, p10, p11, qx, qy, fx, fy);
                        }
                    } else {
                        // not staged: per-pixel coordinates with the full rules, taps from global
                        // memory (zero outside the image, or the nearest edge pixel)
                        const bool rp = OP != OP_RESIZE && J.replicate;
                        const bool words_ok = (((uintptr_t)J.src | (uintptr_t)J.spitch) & 3) == 0;
#pragma unroll
                        for (int j = 0; j < TW / 16; ++j) {
                            const int c = l16 + 16 * j;
                            if (c >= nx) continue;
                            int x0 = 0, y0 = 0, qx = 0, qy = 0, dx = 1, dy = 1;
                            float fx = 0.f, fy = 0.f;
                            bool valid = true;
                            if (OP == OP_RESIZE) {
                                x0 = sl.cx0[c]; dx = sl.cqd[c] >> 16; qx = sl.cqd[c] & 0xFFFF; fx = sl.cf[c];
                                y0 = sl.ry0[r]; dy = sl.rqd[r] >> 16; qy = sl.rqd[r] & 0xFFFF; fy = sl.rf[r];
                            } else {
                                float sx, sy;
                                valid = map_coord<OP>(J.M, tx0 + c, y, sx, sy);
                                if (valid) {
                                    warp_weight(sx, x0, qx);
                                    warp_weight(sy, y0, qy);
                                    fx = __fsub_rn(sx, floorf(sx));
                                    fy = __fsub_rn(sy, floorf(sy));
                                }
                            }
                            uint32_t p00 = 0, p01 = 0, p10 = 0, p11 = 0;
                            if (valid && words_ok && !rp && x0 >= 0 && x0 + 1 < J.W && y0 >= 0 && y0 + 2 < J.H) {
                                // both taps inside, both rows followed by a row of the image: the
                                // pair's six bytes of each row from three aligned words (at most 11
                                // bytes past the pair, inside the next row)
                                const uint8_t *a = J.src + (int64_t)y0 * J.spitch + 3 * x0;
                                const uint32_t *w0 = reinterpret_cast<const uint32_t *>((uintptr_t)a & ~(uintptr_t)3);
                                const uint32_t *w1 = reinterpret_cast<const uint32_t *>(
                                    (uintptr_t)(a + (int64_t)dy * J.spitch) & ~(uintptr_t)3);
                                const uint32_t sh8 = (uint32_t)(uintptr_t)a << 3;
                                p00 = __funnelshift_r(__ldg(w0), __ldg(w0 + 1), sh8);
                                p01 = __funnelshift_r(__ldg(w0 + 1), __ldg(w0 + 2), sh8);
                                p10 = __funnelshift_r(__ldg(w1), __ldg(w1 + 1), sh8);
                                p11 = __funnelshift_r(__ldg(w1 + 1), __ldg(w1 + 2), sh8);
                                emit<CIN, OUTK, TAPS_RAW>(J, o, c, p00, p01, p10, p11, qx, qy, fx, fy);
                                continue;
                            }
                            if (valid) {
                                p00 = ldg_px3(J.src, J.spitch, J.H, J.W, y0, x0, rp);
                                p01 = ldg_px3(J.src, J.spitch, J.H, J.W, y0, x0 + dx, rp);
                                p10 = ldg_px3(J.src, J.spitch, J.H, J.W, y0 + dy, x0, rp);
                                p11 = ldg_px3(J.src, J.spitch, J.H, J.W, y0 + dy, x0 + dx, rp);
                            }
                            emit<CIN, OUTK>(J, o, c, p00, p01, p10, p11, qx, qy, fx, fy);
                        }
                    }
                }
            }
            }
            if (kRunKind) continue;   // (written straight to global memory)
            __syncwarp();

            // ---- write-out of the unit ----
            {
                // every (plane, row) segment of the unit: its 16-byte aligned middle leaves by one
                // bulk copy from the unit stage (whose rows keep the global rows' 16-byte phase),
                // the (at most 15 + 15) head and tail bytes by the lanes
                fence_proxy_async_smem();
                __syncwarp();
                const int nplanes = chw ? 3 : 1;
                const int nrow = min(UR, ny - ra);
                const int seglen = chw ? nx * 4 : nx * dC * ES;
                const int nseg = nplanes * nrow;
                const int64_t tile_off = chw ? (int64_t)tx0 * 4 : (int64_t)tx0 * dC * ES;
                uint8_t *drow0 = J.dst + (int64_t)(ty0 + ra) * J.dpitch + tile_off;
                auto seg_base = [&](int sidx, int &srow_off) -> uint8_t * {
                    const int pl = chw ? (sidx >= nrow) + (sidx >= 2 * nrow) : 0;
                    const int h = sidx - pl * nrow;
                    srow_off = (int)ub + (pl * UR + h) * orow;
                    return drow0 + (int64_t)h * J.dpitch + (int64_t)pl * J.dplane;
                };
                for (int sidx = 0; sidx < nseg; ++sidx) {
                    int so;
                    uint8_t *g = seg_base(sidx, so);
                    const int phase = (int)((uintptr_t)g & 15);
                    const int m0 = min((16 - phase) & 15, seglen);   // head bytes
                    const int mlen = (seglen - m0) & ~15;             // aligned middle
                    if (lane == 0 && mlen > 0) bulk_store(g + m0, kr_pipe_smem + so + phase + m0, (uint32_t)mlen);
                    const int b = lane < 16 ? lane : m0 + mlen + (lane - 16);
                    if ((lane < 16 && b < m0) || (lane >= 16 && b < seglen)) g[b] = kr_pipe_smem[so + phase + b];
                }
                if (lane == 0) {
                    bulk_commit();
                    // the copies of the unit before this one have read the other stage
                    bulk_wait_read_1();
                }
                __syncwarp();
            }
            ++u;
        }
        // this warp has read the slot and its box
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.empty[s]);
    }
    // the unit stages' last stores have been read before the CTA's shared memory goes away
    if (lane == 0) bulk_wait_read_all();
}

// The whole CTA: barrier set-up, then the producer warp and the consumer warps.
template <int OP, int OUTK, int TW, int TH, int NS, class Pol>
__device__ __forceinline__ void pipe_run(Pol &P, PipeShared<TW, TH, NS> &sh, uint8_t *smem, int stage_bytes,
                                         int unit_bytes)
{
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init_count(&sh.full[s], 32);
            mbar_init_count(&sh.empty[s], kPipeConsumers / 32);
        }
        mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x >= kPipeConsumers)
        pipe_produce<OP, TW, TH, NS>(P, sh, smem, stage_bytes);
    else
        pipe_consume<OP, OUTK, TW, TH, NS>(P, sh, stage_bytes, NS * stage_bytes, unit_bytes);
}

}  // namespace kr
