// Ragged batches: many independent resize / warp / gray items of different
// sizes, matrices and output sizes in one submission.
//
//   host:   validate every item -> pack a work list {header, items grouped by
//           kind (op, channels, output kind), tile prefix} into a pinned staging
//           slot -> one async H2D copy into the caller's workspace -> one
//           persistent kernel per kind present, specialised for that kind, the
//           launches overlapping (programmatic dependent launch on a stream,
//           parallel branches in a CUDA graph);
//   device: #SM x k CTAs of each kernel pull tile indices of their kind from an
//           atomic counter in the workspace header, find the owning item by
//           binary search over the tile prefix, and run the same tile engine as
//           the single-image kernels.
//
// The tile shape and CTAs per SM (which sets the shared-memory cap of the
// launch) come from a small autotuner that times the candidates on the batch
// and caches the winner per batch class.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "kr_tile.cuh"
#include "kr_internal.h"
#include "kr_pipe.cuh"

namespace kr {

// ---------------------------------------------------------------------------
// Device work list
// ---------------------------------------------------------------------------
struct alignas(16) WorkItem {
    const uint8_t *src;
    uint8_t *dst;
    int64_t spitch, dpitch, dplane;
    int32_t H, W, h, w;
    int32_t kind;          // KIND_* below
    int32_t tiles_x;
    int32_t foot_budget;
    int32_t region_b;
    int32_t chw;
    int32_t flags;         // ITEM_* below
    float M[6];
    float scale[3], bias[3];
};
static_assert(sizeof(WorkItem) == 128, "work item is 128 bytes");

constexpr int kind_of(int op, int cin, int outk) { return op | (cin << 4) | (outk << 8); }
constexpr int KIND_GRAY = 0x1000;
// The kinds of work item, one specialised kernel (and one group of the work list) each.
constexpr int kGroups = 13;
constexpr int kKinds[kGroups] = {
    kind_of(OP_RESIZE, 3, OUT_U8), kind_of(OP_RESIZE, 3, OUT_U8_GRAY), kind_of(OP_RESIZE, 3, OUT_F32),
    kind_of(OP_RESIZE, 3, OUT_F32_GRAY), kind_of(OP_RESIZE, 1, OUT_U8), kind_of(OP_RESIZE, 1, OUT_F32),
    kind_of(OP_WARP, 3, OUT_U8), kind_of(OP_WARP, 3, OUT_U8_GRAY), kind_of(OP_WARP, 3, OUT_F32),
    kind_of(OP_WARP, 3, OUT_F32_GRAY), kind_of(OP_WARP, 1, OUT_U8), kind_of(OP_WARP, 1, OUT_F32), KIND_GRAY};
static int group_of(int kind)
{
    for (int g = 0; g < kGroups; ++g)
        if (kKinds[g] == kind) return g;
    return -1;
}

struct alignas(16) WsHeader {
    unsigned next[16];        // per-group tile counters (0 in every freshly copied header)
    int n;                    // items
    int total_tiles;
    int pad0[2];
    int first_item[16];       // group g: items [first_item[g], first_item[g] + items[g])
    int items[16];
    int first_tile[16];       // group g: tiles [first_tile[g], first_tile[g] + tiles[g])
    int tiles[16];
    int stage_bytes[16];      // group g, pipelined kernel: bytes of one staging slot
    int pad1[28];
};
static_assert(sizeof(WsHeader) == 512, "header is 512 bytes");
// item flags: the warp map allows the fast path; region A is sized for raw boxes; the
// source rows are 16-byte aligned (bulk row copies); the warp replicates the border
constexpr int ITEM_FAST = 1, ITEM_RAW = 2, ITEM_ROWS16 = 4, ITEM_REPLICATE = 8;

// Device error flags of the ragged kernel (bit 0: a bounded staging wait ran out).
static __device__ unsigned g_kr_batch_err;

// Bound of the first wait for a tile's staged box in the pipelined ragged kernels (0: give
// up at once); the second wait, for copies still in flight, always has the full bound.
static __device__ unsigned long long g_kr_stage_wait_ns = kTmaWaitNs;

// Staging ring depth and tile shape of the pipelined ragged kernels.
constexpr int kPipeStages = 2;
constexpr int kPipeTW = 64, kPipeTH = 64;

// Kinds that run on the pipelined engine (3-channel resize and warp).
constexpr bool pipe_kind(int kind) { return kind != KIND_GRAY && ((kind >> 4) & 15) == 3; }

static constexpr size_t prefix_bytes(int n) { return ((size_t)(n + 1) * 4 + 15) & ~(size_t)15; }
static constexpr size_t worklist_bytes(int n)
{
    return sizeof(WsHeader) + (size_t)n * sizeof(WorkItem) + prefix_bytes(n);
}

// Gray tile: TW x TH pixels, no staging (3 bytes in, 1 byte out per pixel).
template <int TW, int TH>
__device__ __forceinline__ void gray_tile(const WorkItem &it, int tx, int ty)
{
    const int x0 = tx * TW, y0 = ty * TH;
    const int nx = min(TW, it.w - x0), ny = min(TH, it.h - y0);
    for (int i = threadIdx.x; i < nx * ny; i += kThreads) {
        const int r = i / nx, c = i - r * nx;
        const uint8_t *s = it.src + (int64_t)(y0 + r) * it.spitch + (int64_t)(x0 + c) * 3;
        it.dst[(int64_t)(y0 + r) * it.dpitch + x0 + c] = (uint8_t)gray_u8(__ldg(s), __ldg(s + 1), __ldg(s + 2));
    }
}

__device__ __forceinline__ Job job_of(const WorkItem &it)
{
    Job J;
    J.src = it.src;
    J.spitch = it.spitch;
    J.H = it.H;
    J.W = it.W;
    J.dst = it.dst;
    J.dpitch = it.dpitch;
    J.dplane = it.dplane;
    J.h = it.h;
    J.w = it.w;
    J.chw = it.chw;
    J.foot_budget = it.foot_budget;
    J.region_b = it.region_b;
    J.allow_fast = (it.flags & ITEM_FAST) ? 1 : 0;
    J.tin = nullptr;
    J.tin_nc = J.tin_br = 0;
    J.raw_taps = (it.flags & ITEM_RAW) ? 1 : 0;
    J.rows16 = (it.flags & ITEM_ROWS16) ? 1 : 0;
    J.replicate = (it.flags & ITEM_REPLICATE) ? 1 : 0;
    J.direct = 0;
    J.zimg = 0;
    J.err = &g_kr_batch_err;
    J.wait_ns = g_kr_stage_wait_ns;
    J.rm[0] = J.rm[1] = J.rm[2] = J.rm[3] = 0u;
#pragma unroll
    for (int k = 0; k < 6; ++k) J.M[k] = it.M[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        J.scale[k] = it.scale[k];
        J.bias[k] = it.bias[k];
    }
    return J;
}

// Register budgets: f32 kinds 64 (4 CTAs per SM), the others 48 (5).
constexpr bool kind_is_f32(int kind) { return kind != KIND_GRAY && ((kind >> 8) & 15) >= OUT_F32; }

template <int TW, int TH, int G>
__global__ void __launch_bounds__(kThreads, kind_is_f32(kKinds[G]) ? 4 : 5) ragged_kernel(uint8_t *ws)
{
    // The next kind's kernel in the stream may start now: the kinds share no data.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    constexpr int KIND = kKinds[G];
    constexpr int OP = KIND & 15, CIN = (KIND >> 4) & 15, OUTK = (KIND >> 8) & 15;
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ TileShared<TW, TH> ts;
    __shared__ int s_tile;
    WsHeader *hdr = reinterpret_cast<WsHeader *>(ws);
    const WorkItem *items = reinterpret_cast<const WorkItem *>(ws + sizeof(WsHeader));
    const int n = hdr->n;
    const int *prefix = reinterpret_cast<const int *>(items + n);
    const int i0 = hdr->first_item[G], i1 = i0 + hdr->items[G] - 1;
    const int t0 = hdr->first_tile[G], tiles = hdr->tiles[G];
    if (KIND != KIND_GRAY) tile_shared_init(ts);
    for (;;) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(&hdr->next[G], 1u);
        __syncthreads();
        const int tl = s_tile;
        if (tl >= tiles) break;
        const int t = t0 + tl;
        int lo = i0, hi = i1;   // last item of the group whose first tile is <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(prefix + mid) <= t) lo = mid; else hi = mid - 1;
        }
        const WorkItem &it = items[lo];
        const int local = t - __ldg(prefix + lo);
        const int ty = local / it.tiles_x, tx = local - ty * it.tiles_x;
        if (KIND == KIND_GRAY) {
            gray_tile<TW, TH>(it, tx, ty);
        } else {
            process_tile<OP, CIN, OUTK, TW, TH, true, false>(job_of(it), tx, ty, smem, ts);
        }
        __syncthreads();   // everyone has read s_tile before thread 0 rewrites it
        // a staging wait ran out twice: copies may still be in flight into this CTA's shared
        // memory, so it takes no further tiles (the others finish the list; error bit set)
        if (KIND != KIND_GRAY && !ts.mbar_ok) break;
    }
}

// Tiles of one kind group of a ragged work list for the pipelined kernels: the producer
// claims kClaim consecutive tiles at a time from the group's counter in the work-list header
// (so CTAs that drew cheap tiles take more), and since a CTA's tile indices only grow, the
// owning item is found by a forward scan of the tile prefix from the previous tile's item,
// 32 entries per warp-wide read.
struct RaggedPipeTiles {
    static constexpr bool kSameGeometry = false;
    static constexpr int kClaim = 2;
    unsigned *next;   // the group's tile counter
    const WorkItem *items;
    const int *prefix;
    int t0, tiles, last_item;
    int cur;          // item of the previous tile (first item of the group at the start)
    int claim = 0, left = 0;   // next tile of the current claim, tiles left in it
    __device__ bool tile(int, int lane, int &job, int &tx, int &ty)
    {
        if (left == 0) {
            int c = 0;
            if (lane == 0) c = (int)atomicAdd(next, (unsigned)kClaim);
            claim = __shfl_sync(0xffffffffu, c, 0);
            left = kClaim;
        }
        const int tl = claim++;
        --left;
        if (tl >= tiles) return false;
        const int t = t0 + tl;
        for (;;) {
            const int idx = cur + 1 + lane;
            const bool le = idx <= last_item && __ldg(prefix + idx) <= t;
            const unsigned m = __ballot_sync(0xffffffffu, le);   // the prefix grows: a run of lanes
            cur += __popc(m);
            if (m != 0xffffffffu) break;
        }
        job = cur;
        const int local = t - __ldg(prefix + cur);
        const int txs = __ldg(&items[cur].tiles_x);
        ty = local / txs;
        tx = local - ty * txs;
        return true;
    }
    __device__ void job(int j, Job &J) const { J = job_of(items[j]); }
    __device__ unsigned *err() const { return &g_kr_batch_err; }
    __device__ uint64_t first_wait_ns() const { return g_kr_stage_wait_ns; }
};

// Pipelined ragged kernel of kind group G (a 3-channel resize or warp kind): persistent CTAs
// of one producer warp and kPipeConsumers blending threads over the group's tiles.
template <int G>
__global__ void __launch_bounds__(kPipeThreads, 3) ragged_pipe_kernel(uint8_t *ws)
{
    // The next kind's kernel in the stream may start now: the kinds share no data.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    constexpr int KIND = kKinds[G];
    constexpr int OP = KIND & 15, OUTK = (KIND >> 8) & 15;
    static_assert(pipe_kind(KIND), "3-channel resample kinds only");
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ PipeShared<kPipeTW, kPipeTH, kPipeStages> sh;
    const WsHeader *hdr = reinterpret_cast<const WsHeader *>(ws);
    const WorkItem *items = reinterpret_cast<const WorkItem *>(ws + sizeof(WsHeader));
    RaggedPipeTiles P;
    P.next = &reinterpret_cast<WsHeader *>(ws)->next[G];
    P.items = items;
    P.prefix = reinterpret_cast<const int *>(items + hdr->n);
    P.t0 = hdr->first_tile[G];
    P.tiles = hdr->tiles[G];
    P.cur = hdr->first_item[G];
    P.last_item = hdr->first_item[G] + hdr->items[G] - 1;
    pipe_run<OP, OUTK, kPipeTW, kPipeTH, kPipeStages>(P, sh, smem, hdr->stage_bytes[G],
                                                        pipe_unit_bytes<OUTK, kPipeTW>());
}

// Dynamic shared bytes of a pipelined ragged launch with staging slots of `stage` bytes.
static size_t pipe_smem(int kind, int stage)
{
    const int outk = (kind >> 8) & 15;
    const int unit = outk == OUT_U8 ? pipe_unit_bytes<OUT_U8, kPipeTW>()
                     : outk == OUT_U8_GRAY ? pipe_unit_bytes<OUT_U8_GRAY, kPipeTW>()
                     : outk == OUT_F32 ? pipe_unit_bytes<OUT_F32, kPipeTW>()
                                       : pipe_unit_bytes<OUT_F32_GRAY, kPipeTW>();
    return (size_t)kPipeStages * stage + (size_t)2 * (kPipeConsumers / 32) * unit;
}

cudaError_t set_stage_wait_ns_batch(unsigned long long ns)
{
    return cudaMemcpyToSymbol(g_kr_stage_wait_ns, &ns, sizeof(ns));
}

cudaError_t batch_error_flags(unsigned *flags, bool clear)
{
    cudaError_t e = cudaMemcpyFromSymbol(flags, g_kr_batch_err, sizeof(unsigned));
    if (e == cudaSuccess && clear) {
        const unsigned zero = 0;
        e = cudaMemcpyToSymbol(g_kr_batch_err, &zero, sizeof(unsigned));
    }
    return e;
}

// ---------------------------------------------------------------------------
// Tile configurations
// ---------------------------------------------------------------------------
struct TileCfg {
    int tw, th;
    const void *kernels[kGroups];
    int max_smem;
};

template <int TW, int TH> static constexpr int max_region_b()
{
    return 3 * (TH / 2) * round16(TW * 4 + 15) > kRegionBCap ? 3 * (TH / 2) * round16(TW * 4 + 15) : kRegionBCap;
}

#define KR_KERNELS(TW, TH)                                                                                     \
    {(const void *)ragged_kernel<TW, TH, 0>, (const void *)ragged_kernel<TW, TH, 1>,                            \
     (const void *)ragged_kernel<TW, TH, 2>, (const void *)ragged_kernel<TW, TH, 3>,                            \
     (const void *)ragged_kernel<TW, TH, 4>, (const void *)ragged_kernel<TW, TH, 5>,                            \
     (const void *)ragged_kernel<TW, TH, 6>, (const void *)ragged_kernel<TW, TH, 7>,                            \
     (const void *)ragged_kernel<TW, TH, 8>, (const void *)ragged_kernel<TW, TH, 9>,                            \
     (const void *)ragged_kernel<TW, TH, 10>, (const void *)ragged_kernel<TW, TH, 11>,                          \
     (const void *)ragged_kernel<TW, TH, 12>}
// Configuration 0 (64 x 32 tiles) runs the 3-channel resample kinds on the pipelined kernel.
static TileCfg g_cfgs[] = {
    {64, 64,
     {(const void *)ragged_pipe_kernel<0>, (const void *)ragged_pipe_kernel<1>, (const void *)ragged_pipe_kernel<2>,
      (const void *)ragged_pipe_kernel<3>, (const void *)ragged_kernel<64, 64, 4>,
      (const void *)ragged_kernel<64, 64, 5>, (const void *)ragged_pipe_kernel<6>,
      (const void *)ragged_pipe_kernel<7>, (const void *)ragged_pipe_kernel<8>, (const void *)ragged_pipe_kernel<9>,
      (const void *)ragged_kernel<64, 64, 10>, (const void *)ragged_kernel<64, 64, 11>,
      (const void *)ragged_kernel<64, 64, 12>},
     kFootCap + max_region_b<64, 64>()},
    {32, 32, KR_KERNELS(32, 32), kFootCap + max_region_b<32, 32>()},
    {128, 16, KR_KERNELS(128, 16), kFootCap + max_region_b<128, 16>()},
    {64, 16, KR_KERNELS(64, 16), kFootCap + max_region_b<64, 16>()},
};
#undef KR_KERNELS
constexpr int kNumCfgs = sizeof(g_cfgs) / sizeof(g_cfgs[0]);

// Group g of configuration cfg runs on the pipelined kernel.
static bool uses_pipe(int cfg, int g) { return cfg == 0 && pipe_kind(kKinds[g]); }
static int threads_of(int cfg, int g) { return uses_pipe(cfg, g) ? kPipeThreads : kThreads; }

// The output stage of process_tile (out_stage_bytes) for a runtime kind: f32 tiles stage
// one band of th / 2 rows at a time.
static int out_stage_of(int outk, int cin, int tw, int th)
{
    const bool f32 = outk == OUT_F32 || outk == OUT_F32_GRAY;
    const int dC = (outk == OUT_U8_GRAY || outk == OUT_F32_GRAY) ? 1 : cin;
    return f32 ? dC * (th / 2) * round16(tw * 4 + 15) : th * round16(tw * dC + 15);
}

// ---------------------------------------------------------------------------
// Host-side packing
// ---------------------------------------------------------------------------
struct PackInfo {
    int total_tiles = 0;
    size_t smem = 0;        // dynamic shared bytes of the largest group launch
    int opmask = 0;
    double out_px = 0;
    // per kind group (items are stored group by group)
    int first_item[kGroups] = {}, items[kGroups] = {};
    int first_tile[kGroups] = {}, tiles[kGroups] = {};
    size_t gsmem[kGroups] = {};   // dynamic shared bytes the group's launch needs
    int stage[kGroups] = {};      // pipelined groups: bytes of one staging slot
};

// Validate one item and write it as a device work item for tile shape (tw, th); smem gets
// the dynamic shared bytes it needs (see pack_into for smem_cap). pipe: the 3-channel
// resample kinds run on the pipelined kernel, whose staging slot pack_into sizes per group
// from the items' largest raw boxes (foot_budget).
static kr_status build_item(const kr_work_t &w, int tw, int th, int smem_cap, bool pipe, WorkItem &it, size_t &smem)
{
    if (w.src.batch != 1 || w.dst.batch != 1) return KR_ERR_INVALID_ARG;
    std::memset(&it, 0, sizeof(it));
    smem = 0;
    if (w.op == KR_OP_GRAY) {
        GrayDesc g;
        kr_status st = build_gray(&w.src, &w.dst, g);
        if (st != KR_OK) return st;
        it.src = g.src; it.dst = g.dst; it.spitch = g.spitch; it.dpitch = g.dpitch;
        it.H = it.h = g.H; it.W = it.w = g.W;
        it.kind = KIND_GRAY;
    } else if (w.op == KR_OP_RESIZE || w.op == KR_OP_WARP) {
        const int op = w.op == KR_OP_RESIZE ? OP_RESIZE : OP_WARP;
        OpDesc d;
        kr_status st = build_resample(op, &w.src, &w.dst, &w.post, d);
        if (st != KR_OK) return st;
        if (op == OP_WARP)
            for (int k = 0; k < 6; ++k)
                if (!std::isfinite(w.M[k])) return KR_ERR_INVALID_ARG;
        it.src = d.src; it.dst = d.dst; it.spitch = d.spitch; it.dpitch = d.dpitch;
        it.dplane = d.dplane; it.H = d.H; it.W = d.W; it.h = d.h; it.w = d.w; it.chw = d.chw;
        it.kind = kind_of(op, d.cin, d.outk);
        for (int k = 0; k < 6; ++k) it.M[k] = op == OP_WARP ? w.M[k] : 0.f;
        for (int k = 0; k < 3; ++k) { it.scale[k] = d.scale[k]; it.bias[k] = d.bias[k]; }
        const int ob = out_stage_of(d.outk, d.cin, tw, th);
        Budget bud = op == OP_RESIZE ? budget_resize(d.cin, d.H, d.W, d.h, d.w, tw, th, ob)
                                     : budget_warp(d.cin, d.H, d.W, it.M, tw, th, ob);
        it.flags = (op == OP_RESIZE || warp_allows_fast(it.M, d.h, d.w)) ? ITEM_FAST : 0;
        const bool rows16 = ((uintptr_t)d.src & 15) == 0 && (d.spitch & 15) == 0;
        if (rows16) it.flags |= ITEM_ROWS16;
        if (d.replicate) it.flags |= ITEM_REPLICATE;
        if (pipe && d.cin == 3) {
            // raw boxes by bulk row copies (16-byte aligned rows), else taps from global memory
            long long need = 0;
            if (rows16 && bud.cols > 0 && bud.rows > 0 && bud.cols < 1000000 && bud.rows < 1000000)
                need = 16LL * ((15 + bud.cols * 3 + 15) / 16) * bud.rows + 16;
            if (rows16) it.flags |= ITEM_RAW;
            it.foot_budget = (int)std::min<long long>(need, 1 << 30);
            it.region_b = 0;
            it.tiles_x = (it.w + tw - 1) / tw;
            return KR_OK;
        }
        if (d.cin == 3 && rows16 && bud.a > 0 && bud.fits) {
            // bulk row copies and raw taps: region A holds the item's largest box (plus
            // the 16 bytes a last pixel pair may touch), region B only the output tile
            const long long a = 16LL * ((15 + bud.cols * 3 + 15) / 16) * bud.rows + 16;
            if (a <= std::max<long long>(bud.b, kRegionBCap)) {
                it.flags |= ITEM_RAW;
                bud.a = round128((int)a);
                bud.b = round16(ob);
            }
        }
        if ((long long)bud.a + bud.b > smem_cap) {
            const int b_min = round16(ob);
            if (b_min > smem_cap) return KR_ERR_NO_SPACE;   // not even the output stage fits
            if (it.flags & ITEM_RAW) {
                bud.b = b_min;
                bud.a = (smem_cap - b_min) & ~127;
            } else {
                bud.a = 0;   // re-laid staging needs both regions: take the unstaged path
                bud.b = b_min;
            }
        }
        it.foot_budget = bud.a;
        it.region_b = bud.b;
        smem = (size_t)bud.a + bud.b;
    } else {
        return KR_ERR_INVALID_ARG;
    }
    it.tiles_x = (it.w + tw - 1) / tw;
    return KR_OK;
}

// Validate all items and write them as device work items for tile shape (tw, th) into
// out[0..n), grouped by kind (group g in out[first_item[g] ..]), and their first-tile
// indices into prefix[0..n]. Allocates nothing. smem_cap bounds the dynamic shared memory
// of every launch (the residency the caller wants): an item whose boxes need more stages
// only the tiles whose box fits what is left next to its output stage, and its other tiles
// read their taps from global memory.
static kr_status pack_into(const kr_work_t *items, int n, int cfg, int smem_cap, WorkItem *out, int *prefix,
                           PackInfo &P)
{
    P = PackInfo();
    const int tw = g_cfgs[cfg].tw, th = g_cfgs[cfg].th;
    const bool pipe = cfg == 0;
    // pass 1: validate, count the items of each kind
    for (int i = 0; i < n; ++i) {
        WorkItem it;
        size_t sm;
        kr_status st = build_item(items[i], tw, th, smem_cap, pipe, it, sm);
        if (st != KR_OK) return st;
        P.items[group_of(it.kind)]++;
    }
    for (int g = 1; g < kGroups; ++g) P.first_item[g] = P.first_item[g - 1] + P.items[g - 1];
    // pass 2: each item into the next slot of its group
    int fill[kGroups] = {};
    for (int i = 0; i < n; ++i) {
        WorkItem it;
        size_t sm;
        kr_status st = build_item(items[i], tw, th, smem_cap, pipe, it, sm);
        if (st != KR_OK) return st;
        const int g = group_of(it.kind);
        out[P.first_item[g] + fill[g]++] = it;
        if (uses_pipe(cfg, g)) {
            // the slot holds the group's largest raw box, within what the cap leaves next to the
            // unit stages; tiles with larger boxes read their taps from global memory
            const long long cap = ((long long)smem_cap - (long long)pipe_smem(it.kind, 0)) / kPipeStages;
            const int slot = (int)(std::min<long long>(it.foot_budget, std::max(cap, 0LL)) & ~127LL);
            P.stage[g] = std::max(P.stage[g], slot);
            P.gsmem[g] = pipe_smem(it.kind, P.stage[g]);
        } else {
            P.gsmem[g] = std::max(P.gsmem[g], sm);
            P.smem = std::max(P.smem, sm);
        }
        P.opmask |= 1 << items[i].op;
        P.out_px += (double)it.h * it.w;
    }
    long long total = 0;
    for (int g = 0; g < kGroups; ++g) {
        P.first_tile[g] = (int)total;
        for (int j = P.first_item[g]; j < P.first_item[g] + P.items[g]; ++j) {
            prefix[j] = (int)total;
            total += (long long)out[j].tiles_x * ((out[j].h + th - 1) / th);
            if (total > 0x7FFFFFFF) return KR_ERR_INVALID_ARG;
        }
        P.tiles[g] = (int)total - P.first_tile[g];
    }
    prefix[n] = (int)total;
    P.total_tiles = (int)total;
    return KR_OK;
}

// The work list of the submit path, in host memory.
struct Packed {
    std::vector<WorkItem> items;
    std::vector<int> prefix;
    PackInfo info;
};

static kr_status pack_items(const kr_work_t *items, int n, int cfg, int smem_cap, Packed &P)
{
    P.items.resize(n);
    P.prefix.resize(n + 1);
    return pack_into(items, n, cfg, smem_cap, P.items.data(), P.prefix.data(), P.info);
}

// Work-list image: header (with the group tables), items, tile prefix (the layout the
// kernel reads).
static void write_worklist_raw(const WorkItem *items, const int *prefix, int n, const PackInfo &P, uint8_t *dst)
{
    WsHeader h;
    std::memset(&h, 0, sizeof(h));
    h.n = n;
    h.total_tiles = P.total_tiles;
    for (int g = 0; g < kGroups; ++g) {
        h.first_item[g] = P.first_item[g];
        h.items[g] = P.items[g];
        h.first_tile[g] = P.first_tile[g];
        h.tiles[g] = P.tiles[g];
        h.stage_bytes[g] = P.stage[g];
    }
    std::memcpy(dst, &h, sizeof(h));
    std::memcpy(dst + sizeof(h), items, (size_t)n * sizeof(WorkItem));
    std::memcpy(dst + sizeof(h) + (size_t)n * sizeof(WorkItem), prefix, (size_t)(n + 1) * 4);
}

static void write_worklist(const Packed &P, uint8_t *dst)
{
    write_worklist_raw(P.items.data(), P.prefix.data(), (int)P.items.size(), P.info, dst);
}

// ---------------------------------------------------------------------------
// Per-workspace submit contexts: pinned staging ring + graphs.
// ---------------------------------------------------------------------------
constexpr int kSlots = 4;

struct GraphEntry {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t copy = nullptr;
};

// Side streams on which the kernels of further kinds run next to the first one.
constexpr int kSide = 3;

struct Ctx {
    size_t cap = 0;
    uint8_t *slot[kSlots] = {};
    cudaEvent_t done[kSlots] = {};
    int next = 0;
    cudaStream_t side[kSide] = {};
    cudaEvent_t fork = nullptr, join[kSide] = {};
    std::map<std::string, GraphEntry> graphs;   // key: stream|cfg|launch shapes
};

static std::mutex g_mu;
static std::map<void *, Ctx> g_ctx;
static std::map<std::string, std::pair<int, int>> g_tune;   // batch class -> (cfg, ctas/SM)

static void free_ctx(Ctx &c)
{
    for (auto &kv : c.graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    c.graphs.clear();
    for (int i = 0; i < kSlots; ++i) {
        if (c.done[i]) { cudaEventSynchronize(c.done[i]); cudaEventDestroy(c.done[i]); }
        if (c.slot[i]) cudaFreeHost(c.slot[i]);
        c.done[i] = nullptr;
        c.slot[i] = nullptr;
    }
    for (int i = 0; i < kSide; ++i) {
        if (c.side[i]) { cudaStreamSynchronize(c.side[i]); cudaStreamDestroy(c.side[i]); }
        if (c.join[i]) cudaEventDestroy(c.join[i]);
        c.side[i] = nullptr;
        c.join[i] = nullptr;
    }
    if (c.fork) cudaEventDestroy(c.fork);
    c.fork = nullptr;
    c.cap = 0;
}

static cudaError_t ctx_for(void *ws, size_t cap, Ctx *&out)
{
    Ctx &c = g_ctx[ws];
    if (c.cap < cap) {
        free_ctx(c);
        for (int i = 0; i < kSlots; ++i) {
            cudaError_t e = cudaHostAlloc((void **)&c.slot[i], cap, cudaHostAllocDefault);
            if (e != cudaSuccess) { free_ctx(c); return e; }
            e = cudaEventCreateWithFlags(&c.done[i], cudaEventDisableTiming);
            if (e != cudaSuccess) { free_ctx(c); return e; }
        }
        cudaError_t e = cudaEventCreateWithFlags(&c.fork, cudaEventDisableTiming);
        for (int i = 0; i < kSide && e == cudaSuccess; ++i) {
            e = cudaStreamCreateWithFlags(&c.side[i], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.join[i], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) { free_ctx(c); return e; }
        c.cap = cap;
    }
    out = &c;
    return cudaSuccess;
}

static int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// Shared-memory opt-in and residency of the kind-g kernel of configuration cfg.
static cudaError_t prepare_kernel(int cfg, int g, size_t smem, int &occ)
{
    const TileCfg &c = g_cfgs[cfg];
    int max_smem = c.max_smem;
    if (uses_pipe(cfg, g)) {
        // everything the opt-in limit leaves next to the kernel's static shared memory
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa;
        std::memset(&fa, 0, sizeof(fa));
        cudaError_t e = cudaFuncGetAttributes(&fa, c.kernels[g]);
        if (e != cudaSuccess) return e;
        max_smem = (optin - (int)fa.sharedSizeBytes) & ~127;
    }
    cudaError_t e = cudaFuncSetAttribute(c.kernels[g], cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, c.kernels[g], threads_of(cfg, g), smem);
    if (e != cudaSuccess) return e;
    occ = std::max(occ, 1);
    return cudaSuccess;
}

// Launch shape of every kind present: grid (persistent, at most #SM x CTAs per SM) and
// dynamic shared bytes. grid[g] = 0 for absent kinds.
struct Launches {
    int grid[kGroups] = {};
    size_t smem[kGroups] = {};
    int count = 0;
    int min_occ = 1 << 30;   // fewest CTAs per SM among the kinds' kernels
};

static cudaError_t launch_shapes(const PackInfo &I, int cfg, int ctas_per_sm, Launches &L)
{
    L = Launches();
    const int sms = sm_count();
    for (int g = 0; g < kGroups; ++g) {
        if (I.tiles[g] == 0) continue;
        int occ = 1;
        cudaError_t e = prepare_kernel(cfg, g, I.gsmem[g], occ);
        if (e != cudaSuccess) return e;
        L.min_occ = std::min(L.min_occ, occ);
        const int per_sm = ctas_per_sm > 0 ? std::min(ctas_per_sm, occ) : occ;
        L.grid[g] = std::max(1, std::min(sms * per_sm, I.tiles[g]));
        L.smem[g] = I.gsmem[g];
        ++L.count;
    }
    return cudaSuccess;
}

// The kernels of a packed batch on `stream`, the work list already copied: the first kind
// on the stream itself, the others on side streams forked after the copy and joined back,
// so that the kinds run side by side. side == nullptr: all on the stream, one after another.
static cudaError_t launch_kinds(const Launches &L, int cfg, void *ws, cudaStream_t stream, Ctx *side)
{
    cudaError_t e = cudaSuccess;
    void *args[] = {&ws};
    int k = 0;
    if (side && L.count > 1) e = cudaEventRecord(side->fork, stream);
    for (int g = 0; g < kGroups && e == cudaSuccess; ++g) {
        if (!L.grid[g]) continue;
        cudaStream_t s = stream;
        if (side && k > 0) {
            s = side->side[(k - 1) % kSide];
            e = cudaStreamWaitEvent(s, side->fork, 0);
        }
        if (e == cudaSuccess)
            e = cudaLaunchKernel(g_cfgs[cfg].kernels[g], dim3(L.grid[g]), dim3(threads_of(cfg, g)), args, L.smem[g], s);
        ++k;
    }
    if (side && L.count > 1)
        for (int i = 0; i < std::min(kSide, L.count - 1) && e == cudaSuccess; ++i) {
            e = cudaEventRecord(side->join[i], side->side[i]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, side->join[i], 0);
        }
    return e;
}

// Dynamic shared memory per CTA that lets k CTAs of configuration cfg share one SM.
static int smem_cap_for(int cfg, int k)
{
    int dev = 0, per_sm = 0, reserved = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaFuncAttributes fa;
    std::memset(&fa, 0, sizeof(fa));
    cudaFuncGetAttributes(&fa, g_cfgs[cfg].kernels[0]);   // every kind has the same static shared memory
    long long cap = (long long)per_sm / std::max(k, 1) - reserved - (long long)fa.sharedSizeBytes;
    cap = std::min<long long>(cap, g_cfgs[cfg].max_smem);
    return cap > 0 ? (int)(cap & ~127LL) : 0;
}

// Residency the submit path targets when neither the caller nor the tuner chose one.
constexpr int kDefaultCtasPerSm = 4;

static std::string class_key(const Packed &P, int n)
{
    char b[320];
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, dev);
    const int nb = (int)std::floor(std::log2((double)std::max(n, 1)));
    const int pb = (int)std::floor(std::log2(std::max(P.info.out_px, 1.0)));
    std::snprintf(b, sizeof(b), "%s|n2^%d|px2^%d|ops%d", prop.name, nb, pb, P.info.opmask);
    return b;
}

// Enqueue one packed batch: copy the work list, launch the persistent kernel.
static kr_status enqueue(const Packed &P, void *ws, int cfg, int ctas_per_sm, bool use_graph,
                         cudaStream_t stream, const char *where)
{
    const size_t bytes = worklist_bytes((int)P.items.size());
    Launches L;
    cudaError_t e = launch_shapes(P.info, cfg, ctas_per_sm, L);
    if (e != cudaSuccess) { set_last_error(where, e); return KR_ERR_CUDA; }

    std::lock_guard<std::mutex> lk(g_mu);
    Ctx *c = nullptr;
    e = ctx_for(ws, bytes, c);
    if (e != cudaSuccess) { set_last_error(where, e); return KR_ERR_CUDA; }
    const int s = c->next;
    c->next = (c->next + 1) % kSlots;
    e = cudaEventSynchronize(c->done[s]);   // the slot's previous copy has finished
    if (e != cudaSuccess) { set_last_error(where, e); return KR_ERR_CUDA; }
    write_worklist(P, c->slot[s]);

    if (!use_graph) {
        e = cudaMemcpyAsync(ws, c->slot[s], bytes, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = launch_kinds(L, cfg, ws, stream, c);
    } else {
        // graph: the copy, then one kernel node per kind, all depending on the copy only
        std::string key;
        {
            char b[64];
            std::snprintf(b, sizeof(b), "%p|%d", (void *)stream, cfg);
            key = b;
            for (int g = 0; g < kGroups; ++g) {
                std::snprintf(b, sizeof(b), "|%d:%zu", L.grid[g], L.smem[g]);
                key += b;
            }
        }
        GraphEntry &g = c->graphs[key];
        if (!g.exec) {
            e = cudaGraphCreate(&g.graph, 0);
            if (e == cudaSuccess)
                e = cudaGraphAddMemcpyNode1D(&g.copy, g.graph, nullptr, 0, ws, c->slot[s], bytes,
                                             cudaMemcpyHostToDevice);
            void *args[] = {&ws};
            for (int k = 0; k < kGroups && e == cudaSuccess; ++k) {
                if (!L.grid[k]) continue;
                cudaKernelNodeParams kp{};
                kp.func = (void *)g_cfgs[cfg].kernels[k];
                kp.gridDim = dim3(L.grid[k]);
                kp.blockDim = dim3(threads_of(cfg, k));
                kp.sharedMemBytes = (unsigned)L.smem[k];
                kp.kernelParams = args;
                cudaGraphNode_t kn = nullptr;
                e = cudaGraphAddKernelNode(&kn, g.graph, &g.copy, 1, &kp);
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, g.graph, 0);
            if (e != cudaSuccess) {
                if (g.graph) cudaGraphDestroy(g.graph);
                c->graphs.erase(key);
                set_last_error(where, e);
                return KR_ERR_CUDA;
            }
        } else {
            e = cudaGraphExecMemcpyNodeSetParams1D(g.exec, g.copy, ws, c->slot[s], bytes,
                                                   cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess) e = cudaGraphLaunch(g.exec, stream);
    }
    if (e == cudaSuccess) e = cudaEventRecord(c->done[s], stream);
    if (e != cudaSuccess) { set_last_error(where, e); return KR_ERR_CUDA; }
    return KR_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free batch submit: the work list lives in a file-scope device
// array instead of a caller workspace, and is copied there from a file-scope
// host array, so the call allocates no device or host memory.
// ---------------------------------------------------------------------------
constexpr int kNoallocMaxItems = KR_BATCH_NOALLOC_MAX_ITEMS;
constexpr size_t kNoallocBytes = worklist_bytes(kNoallocMaxItems);

// Every device that loads the library holds this array until the process exits.
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoallocBytes];

static std::mutex g_noalloc_mu;                       // guards the host image below
static uint8_t g_noalloc_host[kNoallocBytes];         // packed work list, host side
static WorkItem g_noalloc_items[kNoallocMaxItems];
static int g_noalloc_prefix[kNoallocMaxItems + 1];
constexpr int kMaxDevices = 64;
static void *g_noalloc_dev[kMaxDevices];              // device address of the array, per device

// The device address of g_noalloc_scratch on the current device. The name of the
// array is only a host-side stand-in; its address comes from cudaGetSymbolAddress,
// asked once per device with that device current.
static cudaError_t noalloc_scratch_ptr(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!g_noalloc_dev[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_dev[dev] = p;
    }
    *out = g_noalloc_dev[dev];
    return cudaSuccess;
}

}  // namespace kr

using namespace kr;

extern "C" {

size_t kr_batch_workspace_size(int32_t max_items)
{
    return worklist_bytes(std::max(max_items, 1));
}

int32_t kr_tile_config_count(void) { return kNumCfgs; }

kr_status kr_tile_config_shape(int32_t index, int32_t *tile_w, int32_t *tile_h)
{
    if (index < 0 || index >= kNumCfgs || !tile_w || !tile_h) return KR_ERR_INVALID_ARG;
    *tile_w = g_cfgs[index].tw;
    *tile_h = g_cfgs[index].th;
    return KR_OK;
}

kr_status kr_batch_submit(const kr_work_t *items, int32_t n, void *workspace, size_t ws_bytes,
                          const kr_batch_opts_t *opts, kr_stream_t stream)
{
    if (n < 0 || (n > 0 && (!items || !workspace))) return KR_ERR_INVALID_ARG;
    if (n == 0) return KR_OK;
    if (ws_bytes < worklist_bytes(n)) return KR_ERR_NO_SPACE;
    if ((uintptr_t)workspace & 15) return KR_ERR_INVALID_ARG;
    int cfg = opts ? opts->tile_config : -1;
    int ctas = opts ? opts->ctas_per_sm : 0;
    if (cfg >= kNumCfgs || ctas < 0) return KR_ERR_INVALID_ARG;
    Packed P;
    kr_status st;
    if (cfg < 0) {
        // the cached choice for this batch class, else configuration 0
        const int k0 = ctas ? ctas : kDefaultCtasPerSm;
        if ((st = pack_items(items, n, 0, smem_cap_for(0, k0), P)) != KR_OK) return st;
        const std::string key = class_key(P, n);
        int c = 0, k = k0;
        {
            std::lock_guard<std::mutex> lk(g_mu);
            auto it = g_tune.find(key);
            if (it != g_tune.end()) { c = it->second.first; if (!ctas) k = it->second.second; }
        }
        if (c != 0 || k != k0)
            if ((st = pack_items(items, n, c, smem_cap_for(c, k), P)) != KR_OK) return st;
        cfg = c;
        ctas = k;
    } else {
        if (!ctas) ctas = kDefaultCtasPerSm;
        if ((st = pack_items(items, n, cfg, smem_cap_for(cfg, ctas), P)) != KR_OK)
            return st;
    }
    // every item must fit in shared memory at this tile shape
    if (P.info.smem > (size_t)g_cfgs[cfg].max_smem) return KR_ERR_UNSUPPORTED;
    return enqueue(P, workspace, cfg, ctas, opts && opts->use_graph, (cudaStream_t)stream,
                   "kr_batch_submit");
}

kr_status kr_batch_submit_noalloc(const kr_work_t *items, int32_t n, const kr_batch_opts_t *opts,
                                  kr_stream_t stream)
{
    if (n < 0 || (n > 0 && !items)) return KR_ERR_INVALID_ARG;
    if (n == 0) return KR_OK;
    if (n > kNoallocMaxItems) return KR_ERR_NO_SPACE;
    const int cfg = (opts && opts->tile_config >= 0) ? opts->tile_config : 0;
    const int ctas = opts ? opts->ctas_per_sm : 0;
    if (cfg >= kNumCfgs || ctas < 0) return KR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    // under capture the pageable copy would become a graph node reading g_noalloc_host at
    // every replay, after later calls have rewritten it
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(s, &cap);
    if (ce != cudaSuccess) {
        set_last_error("kr_batch_submit_noalloc", ce);
        return KR_ERR_CUDA;
    }
    if (cap != cudaStreamCaptureStatusNone) return KR_ERR_UNSUPPORTED;

    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    PackInfo P;
    kr_status st = pack_into(items, n, cfg, smem_cap_for(cfg, ctas ? ctas : kDefaultCtasPerSm), g_noalloc_items,
                             g_noalloc_prefix, P);
    if (st != KR_OK) return st;
    if (P.smem > (size_t)g_cfgs[cfg].max_smem) return KR_ERR_UNSUPPORTED;
    Launches L;
    void *ws = nullptr;
    cudaError_t e = launch_shapes(P, cfg, ctas, L);
    if (e == cudaSuccess) e = noalloc_scratch_ptr(&ws);
    if (e != cudaSuccess) {
        set_last_error("kr_batch_submit_noalloc", e);
        return KR_ERR_CUDA;
    }
    const size_t bytes = worklist_bytes(n);
    write_worklist_raw(g_noalloc_items, g_noalloc_prefix, n, P, g_noalloc_host);
    // Pageable source: the call returns once the bytes are out of g_noalloc_host, so the
    // next call may overwrite it. The copy also clears the header's tile counters. The
    // kinds' kernels run one after another on the stream (no side streams here).
    e = cudaMemcpyAsync(ws, g_noalloc_host, bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_kinds(L, cfg, ws, s, nullptr);
    if (e != cudaSuccess) {
        set_last_error("kr_batch_submit_noalloc", e);
        return KR_ERR_CUDA;
    }
    return KR_OK;
}

kr_status kr_autotune_batch(const kr_work_t *items, int32_t n, void *workspace, size_t ws_bytes,
                            kr_stream_t stream, int32_t *best_config, int32_t *best_ctas_per_sm)
{
    if (n < 1 || !items || !workspace) return KR_ERR_INVALID_ARG;
    if (ws_bytes < worklist_bytes(n)) return KR_ERR_NO_SPACE;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return KR_ERR_CUDA;
    float best = 1e30f;
    int bc = 0, bk = 0;
    std::string key;
    kr_status result = KR_OK;
    static const int kCands[] = {1, 2, 3, 4, 6, 8};
    for (int cfg = 0; cfg < kNumCfgs && result == KR_OK; ++cfg) {
        for (int k : kCands) {
            // each residency target packs the batch with its own shared-memory cap
            Packed P;
            kr_status st = pack_items(items, n, cfg, smem_cap_for(cfg, k), P);
            if (st == KR_ERR_NO_SPACE) continue;   // an output stage alone exceeds the cap
            if (st != KR_OK) { result = st; break; }
            if (key.empty()) key = class_key(P, n);   // the class does not depend on cfg or k
            Launches L;
            if (launch_shapes(P.info, cfg, k, L) != cudaSuccess) { result = KR_ERR_CUDA; break; }
            if (L.min_occ < k) continue;   // registers (or the cap's rounding) allow fewer CTAs
            float ms_best = 1e30f;
            for (int rep = 0; rep < 4 && result == KR_OK; ++rep) {
                cudaEventRecord(e0, s);
                st = enqueue(P, workspace, cfg, k, false, s, "kr_autotune_batch");
                cudaEventRecord(e1, s);
                if (st != KR_OK) { result = st; break; }
                if (cudaEventSynchronize(e1) != cudaSuccess) { result = KR_ERR_CUDA; break; }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) ms_best = std::min(ms_best, ms);   // rep 0 warms up
            }
            if (ms_best < best) { best = ms_best; bc = cfg; bk = k; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result != KR_OK) return result;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_tune[key] = {bc, bk};
    }
    if (best_config) *best_config = bc;
    if (best_ctas_per_sm) *best_ctas_per_sm = bk;
    return KR_OK;
}

kr_status kr_autotune_save(const char *path)
{
    if (!path) return KR_ERR_INVALID_ARG;
    FILE *f = std::fopen(path, "w");
    if (!f) return KR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    std::fprintf(f, "{\"entries\": [\n");
    size_t i = 0;
    for (auto &kv : g_tune) {
        std::fprintf(f, "  {\"key\": \"%s\", \"tile_config\": %d, \"ctas_per_sm\": %d}%s\n", kv.first.c_str(),
                     kv.second.first, kv.second.second, ++i < g_tune.size() ? "," : "");
    }
    std::fprintf(f, "]}\n");
    std::fclose(f);
    return KR_OK;
}

kr_status kr_autotune_load(const char *path)
{
    if (!path) return KR_ERR_INVALID_ARG;
    FILE *f = std::fopen(path, "r");
    if (!f) return KR_ERR_INVALID_ARG;
    std::string text;
    char buf[4096];
    size_t r;
    while ((r = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, r);
    std::fclose(f);
    std::map<std::string, std::pair<int, int>> got;
    size_t pos = 0;
    while ((pos = text.find("\"key\": \"", pos)) != std::string::npos) {
        pos += 8;
        const size_t end = text.find('"', pos);
        if (end == std::string::npos) return KR_ERR_INVALID_ARG;
        const std::string key = text.substr(pos, end - pos);
        int cfg = -1, ctas = -1;
        const size_t pc = text.find("\"tile_config\":", end), pk = text.find("\"ctas_per_sm\":", end);
        if (pc == std::string::npos || pk == std::string::npos) return KR_ERR_INVALID_ARG;
        if (std::sscanf(text.c_str() + pc + 14, "%d", &cfg) != 1 ||
            std::sscanf(text.c_str() + pk + 14, "%d", &ctas) != 1)
            return KR_ERR_INVALID_ARG;
        if (cfg < 0 || cfg >= kNumCfgs || ctas < 1) return KR_ERR_INVALID_ARG;
        got[key] = {cfg, ctas};
        pos = end;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &kv : got) g_tune[kv.first] = kv.second;
    return KR_OK;
}

void kr_shutdown(void)
{
    {
        std::lock_guard<std::mutex> lk(g_mu);
        for (auto &kv : g_ctx) free_ctx(kv.second);
        g_ctx.clear();
        g_tune.clear();
    }
    // the allocation-free path looks its array's device address up again on its next call
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    for (int d = 0; d < kMaxDevices; ++d) g_noalloc_dev[d] = nullptr;
}

}  // extern "C"
