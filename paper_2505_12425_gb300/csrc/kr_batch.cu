// Ragged batches: many independent resize / warp / gray items of different
// sizes, matrices and output sizes in ONE persistent launch.
//
//   host:   validate every item -> pack a work list {header, items, tile prefix}
//           into a pinned staging slot -> one async H2D copy into the caller's
//           workspace -> one persistent kernel (optionally both replayed from a
//           CUDA graph);
//   device: #SM x k CTAs pull tile indices from an atomic counter in the
//           workspace header, find the owning item by binary search over the
//           tile prefix, and run the same tile engine as the single-image
//           kernels for that item's (op, channels, output kind).
//
// The tile shape (and CTAs per SM) comes from a small autotuner that times
// every configuration on the batch and caches the winner per batch class.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "kr_device.cuh"
#include "kr_internal.h"

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

struct alignas(16) WsHeader {
    unsigned next;         // tile counter (0 in every freshly copied header)
    int n;                 // items
    int total_tiles;
    int pad[61];
};
static_assert(sizeof(WsHeader) == 256, "header is 256 bytes");

constexpr int kind_of(int op, int cin, int outk) { return op | (cin << 4) | (outk << 8); }
constexpr int KIND_GRAY = 0x1000;
// item flags: the warp map allows the fast path; region A is sized for raw boxes; the
// source rows are 16-byte aligned (bulk row copies)
constexpr int ITEM_FAST = 1, ITEM_RAW = 2, ITEM_ROWS16 = 4;

// Device error flags of the ragged kernel (bit 0: a bounded staging wait ran out).
static __device__ unsigned g_kr_batch_err;

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
    J.tout = nullptr;
    J.zimg = 0;
    J.err = &g_kr_batch_err;
#pragma unroll
    for (int k = 0; k < 6; ++k) J.M[k] = it.M[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        J.scale[k] = it.scale[k];
        J.bias[k] = it.bias[k];
    }
    return J;
}

template <int TW, int TH>
__global__ void __launch_bounds__(kThreads) ragged_kernel(uint8_t *ws)
{
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ TileShared<TW, TH> ts;
    __shared__ int s_tile;
    WsHeader *hdr = reinterpret_cast<WsHeader *>(ws);
    const WorkItem *items = reinterpret_cast<const WorkItem *>(ws + sizeof(WsHeader));
    const int n = hdr->n, total = hdr->total_tiles;
    const int *prefix = reinterpret_cast<const int *>(items + n);
    tile_shared_init(ts);
    for (;;) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(&hdr->next, 1u);
        __syncthreads();
        const int t = s_tile;
        if (t >= total) break;
        int lo = 0, hi = n - 1;   // last item whose first tile is <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(prefix + mid) <= t) lo = mid; else hi = mid - 1;
        }
        const WorkItem &it = items[lo];
        const int local = t - __ldg(prefix + lo);
        const int ty = local / it.tiles_x, tx = local - ty * it.tiles_x;
        if (it.kind == KIND_GRAY) {
            gray_tile<TW, TH>(it, tx, ty);
        } else {
            const Job J = job_of(it);
            switch (it.kind) {
#define KR_CASE(OP, CIN, OUTK) \
    case kind_of(OP, CIN, OUTK): process_tile<OP, CIN, OUTK, TW, TH, true, false>(J, tx, ty, smem, ts); break;
            KR_CASE(OP_RESIZE, 3, OUT_U8)
            KR_CASE(OP_RESIZE, 3, OUT_U8_GRAY)
            KR_CASE(OP_RESIZE, 3, OUT_F32)
            KR_CASE(OP_RESIZE, 3, OUT_F32_GRAY)
            KR_CASE(OP_RESIZE, 1, OUT_U8)
            KR_CASE(OP_RESIZE, 1, OUT_F32)
            KR_CASE(OP_WARP, 3, OUT_U8)
            KR_CASE(OP_WARP, 3, OUT_U8_GRAY)
            KR_CASE(OP_WARP, 3, OUT_F32)
            KR_CASE(OP_WARP, 3, OUT_F32_GRAY)
            KR_CASE(OP_WARP, 1, OUT_U8)
            KR_CASE(OP_WARP, 1, OUT_F32)
#undef KR_CASE
            default: break;
            }
        }
        __syncthreads();   // everyone has read s_tile before thread 0 rewrites it
        // a staging wait ran out twice: copies may still be in flight into this CTA's shared
        // memory, so it takes no further tiles (the others finish the list; error bit set)
        if (!ts.mbar_ok) break;
    }
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
    const void *kernel;
    int max_smem;
};

template <int TW, int TH> static constexpr int max_region_b()
{
    return 3 * (TH / 2) * round16(TW * 4 + 15) > kRegionBCap ? 3 * (TH / 2) * round16(TW * 4 + 15) : kRegionBCap;
}

static TileCfg g_cfgs[] = {
    {64, 32, (const void *)ragged_kernel<64, 32>, kFootCap + max_region_b<64, 32>()},
    {32, 32, (const void *)ragged_kernel<32, 32>, kFootCap + max_region_b<32, 32>()},
    {128, 16, (const void *)ragged_kernel<128, 16>, kFootCap + max_region_b<128, 16>()},
    {64, 16, (const void *)ragged_kernel<64, 16>, kFootCap + max_region_b<64, 16>()},
};
constexpr int kNumCfgs = sizeof(g_cfgs) / sizeof(g_cfgs[0]);

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
    size_t smem = 0;        // dynamic shared bytes the launch needs
    int opmask = 0;
    double out_px = 0;
};

// Validate all items and write them as device work items for tile shape (tw, th) into
// out[0..n) and their first-tile indices into prefix[0..n]. Allocates nothing.
static kr_status pack_into(const kr_work_t *items, int n, int tw, int th, WorkItem *out, int *prefix,
                           PackInfo &P)
{
    P = PackInfo();
    long long total = 0;
    for (int i = 0; i < n; ++i) {
        const kr_work_t &w = items[i];
        if (w.src.batch != 1 || w.dst.batch != 1) return KR_ERR_INVALID_ARG;
        WorkItem &it = out[i];
        std::memset(&it, 0, sizeof(it));
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
            it.foot_budget = bud.a;
            it.region_b = bud.b;
            P.smem = std::max(P.smem, (size_t)bud.a + bud.b);
        } else {
            return KR_ERR_INVALID_ARG;
        }
        P.opmask |= 1 << w.op;
        P.out_px += (double)it.h * it.w;
        it.tiles_x = (it.w + tw - 1) / tw;
        const long long tiles = (long long)it.tiles_x * ((it.h + th - 1) / th);
        prefix[i] = (int)total;
        total += tiles;
        if (total > 0x7FFFFFFF) return KR_ERR_INVALID_ARG;
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

static kr_status pack_items(const kr_work_t *items, int n, int tw, int th, Packed &P)
{
    P.items.resize(n);
    P.prefix.resize(n + 1);
    return pack_into(items, n, tw, th, P.items.data(), P.prefix.data(), P.info);
}

// Work-list image: header, items, tile prefix (the layout the kernel reads).
static void write_worklist_raw(const WorkItem *items, const int *prefix, int n, int total_tiles, uint8_t *dst)
{
    WsHeader h;
    std::memset(&h, 0, sizeof(h));
    h.next = 0;
    h.n = n;
    h.total_tiles = total_tiles;
    std::memcpy(dst, &h, sizeof(h));
    std::memcpy(dst + sizeof(h), items, (size_t)n * sizeof(WorkItem));
    std::memcpy(dst + sizeof(h) + (size_t)n * sizeof(WorkItem), prefix, (size_t)(n + 1) * 4);
}

static void write_worklist(const Packed &P, uint8_t *dst)
{
    write_worklist_raw(P.items.data(), P.prefix.data(), (int)P.items.size(), P.info.total_tiles, dst);
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

struct Ctx {
    size_t cap = 0;
    uint8_t *slot[kSlots] = {};
    cudaEvent_t done[kSlots] = {};
    int next = 0;
    std::map<std::string, GraphEntry> graphs;   // key: stream|cfg|ctas
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

static cudaError_t prepare_cfg(int cfg, size_t smem, int &occ)
{
    const TileCfg &c = g_cfgs[cfg];
    cudaError_t e = cudaFuncSetAttribute(c.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, c.max_smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, c.kernel, kThreads, smem);
    if (e != cudaSuccess) return e;
    occ = std::max(occ, 1);
    return cudaSuccess;
}

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
    int occ = 1;
    cudaError_t e = prepare_cfg(cfg, P.info.smem, occ);
    if (e != cudaSuccess) { set_last_error(where, e); return KR_ERR_CUDA; }
    const int per_sm = ctas_per_sm > 0 ? std::min(ctas_per_sm, occ) : occ;
    const int grid = std::max(1, std::min(sm_count() * per_sm, P.info.total_tiles));

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
        if (e == cudaSuccess) {
            void *args[] = {&ws};
            e = cudaLaunchKernel(g_cfgs[cfg].kernel, dim3(grid), dim3(kThreads), args, P.info.smem, stream);
        }
    } else {
        char key[96];
        std::snprintf(key, sizeof(key), "%p|%d|%d|%zu", (void *)stream, cfg, grid, P.info.smem);
        GraphEntry &g = c->graphs[key];
        if (!g.exec) {
            e = cudaGraphCreate(&g.graph, 0);
            cudaGraphNode_t kn = nullptr;
            if (e == cudaSuccess)
                e = cudaGraphAddMemcpyNode1D(&g.copy, g.graph, nullptr, 0, ws, c->slot[s], bytes,
                                             cudaMemcpyHostToDevice);
            if (e == cudaSuccess) {
                cudaKernelNodeParams kp;
                std::memset(&kp, 0, sizeof(kp));
                void *args[] = {&ws};
                kp.func = (void *)g_cfgs[cfg].kernel;
                kp.gridDim = dim3(grid);
                kp.blockDim = dim3(kThreads);
                kp.sharedMemBytes = (unsigned)P.info.smem;
                kp.kernelParams = args;
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
        if ((st = pack_items(items, n, g_cfgs[0].tw, g_cfgs[0].th, P)) != KR_OK) return st;
        const std::string key = class_key(P, n);
        int c = 0, k = ctas;
        {
            std::lock_guard<std::mutex> lk(g_mu);
            auto it = g_tune.find(key);
            if (it != g_tune.end()) { c = it->second.first; if (!ctas) k = it->second.second; }
        }
        cfg = c;
        ctas = k;
        if (cfg != 0 && (st = pack_items(items, n, g_cfgs[cfg].tw, g_cfgs[cfg].th, P)) != KR_OK) return st;
    } else if ((st = pack_items(items, n, g_cfgs[cfg].tw, g_cfgs[cfg].th, P)) != KR_OK) {
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

    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    PackInfo P;
    kr_status st = pack_into(items, n, g_cfgs[cfg].tw, g_cfgs[cfg].th, g_noalloc_items, g_noalloc_prefix, P);
    if (st != KR_OK) return st;
    if (P.smem > (size_t)g_cfgs[cfg].max_smem) return KR_ERR_UNSUPPORTED;
    int occ = 1;
    void *ws = nullptr;
    cudaError_t e = prepare_cfg(cfg, P.smem, occ);
    if (e == cudaSuccess) e = noalloc_scratch_ptr(&ws);
    if (e != cudaSuccess) {
        set_last_error("kr_batch_submit_noalloc", e);
        return KR_ERR_CUDA;
    }
    const int per_sm = ctas > 0 ? std::min(ctas, occ) : occ;
    const int grid = std::max(1, std::min(sm_count() * per_sm, P.total_tiles));
    const size_t bytes = worklist_bytes(n);
    write_worklist_raw(g_noalloc_items, g_noalloc_prefix, n, P.total_tiles, g_noalloc_host);
    // Pageable source: the call returns once the bytes are out of g_noalloc_host, so the
    // next call may overwrite it. The copy also clears the header's tile counter.
    e = cudaMemcpyAsync(ws, g_noalloc_host, bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        void *args[] = {&ws};
        e = cudaLaunchKernel(g_cfgs[cfg].kernel, dim3(grid), dim3(kThreads), args, P.smem, s);
    }
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
    for (int cfg = 0; cfg < kNumCfgs && result == KR_OK; ++cfg) {
        Packed P;
        kr_status st = pack_items(items, n, g_cfgs[cfg].tw, g_cfgs[cfg].th, P);
        if (st != KR_OK) { result = st; break; }
        if (cfg == 0) key = class_key(P, n);
        if (P.info.smem > (size_t)g_cfgs[cfg].max_smem) continue;
        int occ = 1;
        if (prepare_cfg(cfg, P.info.smem, occ) != cudaSuccess) { result = KR_ERR_CUDA; break; }
        for (int k = 1; k <= occ; ++k) {
            if (k > 2 && k < occ) continue;   // candidates: 1, 2 and the occupancy limit
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
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &kv : g_ctx) free_ctx(kv.second);
    g_ctx.clear();
    g_tune.clear();
}

}  // extern "C"
