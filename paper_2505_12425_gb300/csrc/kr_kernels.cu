// Per-operation kernels: resize / warp over a batch of equally sized images
// (one TW x TH output tile per CTA, blockIdx.z = image) and the standalone
// RGB -> gray streaming kernel.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include <cudaTypedefs.h>

#include "kr_tile.cuh"
#include "kr_internal.h"

namespace kr {

// Tile shape of the per-operation kernels: 64 columns (the 4-pixel quad path) by 64 rows for
// resize and 48 for the warps (measured against 32, 48, 64 and 128 rows: with no output stage,
// taller tiles share the per-tile work of planning and staging among more pixels; the warps'
// boxes, larger for the same tile, keep 8 CTAs per SM at 48 rows).
constexpr int kTW = 64;
template <int OP, int OUTK> constexpr int op_tile_h() { return OP == OP_RESIZE ? 64 : 48; }

// Device error flags of the per-operation kernels (bit 0: a bounded TMA wait ran out).
static __device__ unsigned g_kr_device_err;

// Bound of the first wait for a tile's staged box (0: give up at once); the second wait, for
// copies still in flight, always has the full bound.
static __device__ unsigned long long g_kr_stage_wait_ns = kTmaWaitNs;

// Largest raw box (bytes of 16-byte chunk rows) a 3-channel launch stages.
constexpr long long kRawBoxCap = 56 * 1024;

struct OpParams {
    CUtensorMap tin;    // source map (valid when has_tin)
    int32_t has_tin;
    int32_t direct;     // destination rows are whole 16-byte chunks at 16-byte aligned addresses
    int32_t tin_nc, tin_br;
    const uint8_t *src;
    int64_t spitch, sbatch;
    int32_t H, W;
    uint8_t *dst;
    int64_t dpitch, dplane, dbatch;
    int32_t h, w;
    int32_t chw;
    int32_t foot_budget;
    int32_t region_b;
    int32_t raw_taps;
    int32_t rows16;
    int32_t replicate;
    uint32_t rm[4];   // resize: multiply-high reciprocals of 2w, 4w, 2h, 4h (0: divide)
    uint32_t fast_mask[(kMaxMPerLaunch + 31) / 32];   // warp: images whose map allows the fast path
    float scale[3], bias[3];
    float M[kMaxMPerLaunch][9];   // warp: 6 floats per image; perspective: 9
};

// CTAs per SM the register allocation leaves room for: u8 kinds 8 (32 registers; the
// perspective warp 6, 40), the f32 resize 6 (40), the f32 warps 5 (48: at 40 they spill).
template <int OP, int OUTK> constexpr int resample_min_ctas()
{
    return (OUTK == OUT_F32 || OUTK == OUT_F32_GRAY) ? (OP == OP_RESIZE ? 6 : 5) : (OP == OP_PERSP ? 6 : 8);
}

// ROWS: instantiated for launches whose 3-channel boxes are staged by bulk row copies (no
// tensor map, 16-byte aligned rows); the others do without that code.
template <int OP, int CIN, int OUTK, int TW, int TH, bool ROWS>
__global__ void __launch_bounds__(kThreads, resample_min_ctas<OP, OUTK>()) resample_kernel(const __grid_constant__ OpParams p)
{
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ TileShared<TW, TH> ts;
    const int z = blockIdx.z;
    Job J;
    J.src = p.src + (int64_t)z * p.sbatch;
    J.spitch = p.spitch;
    J.H = p.H;
    J.W = p.W;
    J.dst = p.dst + (int64_t)z * p.dbatch;
    J.dpitch = p.dpitch;
    J.dplane = p.dplane;
    J.h = p.h;
    J.w = p.w;
    J.chw = p.chw;
    J.foot_budget = p.foot_budget;
    J.region_b = p.region_b;
    J.raw_taps = p.raw_taps;
    J.rows16 = p.rows16;
    J.replicate = p.replicate;
    J.allow_fast = OP != OP_RESIZE ? (int)((p.fast_mask[z >> 5] >> (z & 31)) & 1u) : 1;
    J.tin = p.has_tin ? &p.tin : nullptr;
    J.tin_nc = p.tin_nc;
    J.tin_br = p.tin_br;
    J.direct = p.direct;
    J.zimg = z;
    J.err = &g_kr_device_err;
    J.wait_ns = g_kr_stage_wait_ns;
#pragma unroll
    for (int k = 0; k < 4; ++k) J.rm[k] = p.rm[k];
#pragma unroll
    for (int k = 0; k < 9; ++k) J.M[k] = OP != OP_RESIZE ? p.M[z][k] : 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        J.scale[k] = p.scale[k];
        J.bias[k] = p.bias[k];
    }
    process_tile<OP, CIN, OUTK, TW, TH, ROWS, true>(J, blockIdx.x, blockIdx.y, smem, ts);
}

// ---------------------------------------------------------------------------
// Shared-memory budgets
// ---------------------------------------------------------------------------

// clamp: boxes larger than the caps are staged when they fit (warp); else never staged.
// Resize boxes lie inside the image (clipped to W x H); warp boxes are not clipped.
static Budget budget_for(int cin, double cols_d, double rows_d, int H, int W, int out_bytes, bool clamp)
{
    const int cols = clamp ? (int)std::min<double>(cols_d, 1e6) : (int)std::min<double>(cols_d, W);
    const int rows = clamp ? (int)std::min<double>(rows_d, 1e6) : (int)std::min<double>(rows_d, H);
    long long a, raw;
    if (cin == 3) {
        a = (long long)rows * word_row(cols) * 4;
        raw = (long long)rows * raw_row_bytes(cols, 3);
    } else {
        a = (long long)rows * raw_row_bytes(cols, 1) + 16;
        raw = 0;
    }
    Budget b;
    b.cols = cols;
    b.rows = rows;
    if (a <= kFootCap && raw <= kRegionBCap) {
        b.fits = true;
        b.a = round128((int)a);
        b.b = round16((int)std::max<long long>(out_bytes, raw));
    } else if (clamp) {
        // tiles whose box fits these caps are staged, the others take the general path
        b.a = kFootCap;
        b.b = round16(std::max(out_bytes, cin == 3 ? kRegionBCap : 0));
    } else {
        b.a = 0;
        b.b = round16(out_bytes);
    }
    return b;
}

Budget budget_resize(int cin, int H, int W, int h, int w, int tw, int th, int out_bytes)
{
    // Taps of tw consecutive columns span at most (tw - 1) W / w + 2 source columns.
    const double cols = std::ceil((tw - 1) * (double)W / w) + 3;
    const double rows = std::ceil((th - 1) * (double)H / h) + 3;
    return budget_for(cin, cols, rows, H, W, out_bytes, false);
}

Budget budget_warp(int cin, int H, int W, const float *M, int tw, int th, int out_bytes)
{
    // The box of a tile spans at most |m00|(tw-1) + |m01|(th-1) columns plus six
    // (floor, one pixel low margin, three high margin, rounding).
    const double cols = std::ceil(std::fabs(M[0]) * (tw - 1) + std::fabs(M[1]) * (th - 1)) + 6;
    const double rows = std::ceil(std::fabs(M[3]) * (tw - 1) + std::fabs(M[4]) * (th - 1)) + 6;
    if (!(cols < 1e7 && rows < 1e7)) return budget_for(cin, 1e7, 1e7, H, W, out_bytes, true);
    return budget_for(cin, cols, rows, H, W, out_bytes, true);
}

Budget budget_persp(int cin, int H, int W, const float *M, int h, int w, int tw, int th, int out_bytes)
{
    // The box of a tile is the hull of its corners' images (Z > 0 at the corners); its size
    // varies over the output. The bound is taken on a grid of cells of k x k tiles (k keeps
    // the grid near 16 x 16 cells: the launch stays cheap on the host) over the cells whose
    // corners map in front of the camera: a cell's box / k, 15% and six pixels of margin.
    // It only sizes the staging: a tile whose box is larger takes the general path.
    const int tiles_x = (w + tw - 1) / tw, tiles_y = (h + th - 1) / th;
    const int k = std::max(1, (int)std::ceil(std::sqrt((double)tiles_x * tiles_y / 256.0)));
    double cols = 0, rows = 0;
    auto at = [&](double x, double y, double &sx, double &sy) {
        const double xc = x + 0.5, yc = y + 0.5;
        const double Z = M[6] * xc + M[7] * yc + M[8];
        if (!(Z > 0)) return false;
        sx = (M[0] * xc + M[1] * yc + M[2]) / Z - 0.5;
        sy = (M[3] * xc + M[4] * yc + M[5]) / Z - 0.5;
        return std::fabs(sx) < 1048576.0 && std::fabs(sy) < 1048576.0;
    };
    for (int cy = 0; cy < tiles_y; cy += k)
        for (int cx = 0; cx < tiles_x; cx += k) {
            const int x0 = cx * tw, y0 = cy * th;
            const int x1 = std::min(w, (cx + k) * tw) - 1, y1 = std::min(h, (cy + k) * th) - 1;
            const int kx = std::min(k, tiles_x - cx), ky = std::min(k, tiles_y - cy);
            double sx[4], sy[4];
            if (!at(x0, y0, sx[0], sy[0]) || !at(x1, y0, sx[1], sy[1]) || !at(x0, y1, sx[2], sy[2]) ||
                !at(x1, y1, sx[3], sy[3]))
                continue;
            const double bw = std::max(std::max(sx[0], sx[1]), std::max(sx[2], sx[3])) -
                              std::min(std::min(sx[0], sx[1]), std::min(sx[2], sx[3]));
            const double bh = std::max(std::max(sy[0], sy[1]), std::max(sy[2], sy[3])) -
                              std::min(std::min(sy[0], sy[1]), std::min(sy[2], sy[3]));
            // a k x k cell's box over k tiles of each side (the box is linear in the side)
            const double scale = std::max(kx, ky) > 1 ? 1.15 / std::max(kx, ky) : 1.0;
            cols = std::max(cols, std::ceil(bw * scale) + 6);
            rows = std::max(rows, std::ceil(bh * scale) + 6);
        }
    if (cols == 0 || !(cols < 1e7 && rows < 1e7)) return budget_for(cin, 1e7, 1e7, H, W, out_bytes, true);
    return budget_for(cin, cols, rows, H, W, out_bytes, true);
}

bool warp_allows_fast(const float *M, int h, int w)
{
    const double lim = 524288.0;   // 2^19
    for (int r = 0; r < 2; ++r) {
        const float *m = M + 3 * r;
        if (!(std::fabs(m[0]) * (w + 1) < lim && std::fabs(m[1]) * (h + 1) < lim && std::fabs(m[2]) < lim))
            return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// TMA tensor maps: images as {32-bit word, row, (plane,) image} tensors
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Map over n images of `rows` rows of `rowbytes` bytes, with an extra plane dimension when
// planes > 1. Elements are 32-bit words, so a row must be a whole number of words (the map
// then never reads past a row's own bytes). Box: {box_chunks 16-byte chunks, box_rows, 1(, 1)}.
// Returns false (and the caller keeps the non-TMA path) when the layout does not meet TMA's rules.
static bool encode_map(CUtensorMap *m, const void *base, int64_t rowbytes, int rows, int planes, int n,
                       int64_t pitch, int64_t pstride, int64_t bstride, int box_chunks, int box_rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    if ((rowbytes & 3) || rowbytes < 4) return false;
    if (((uintptr_t)base & 15) || (pitch & 15) || pitch < rowbytes) return false;
    // the box's first dimension is at most 256 elements
    if (box_chunks < 1 || box_chunks > 64 || box_rows < 1 || box_rows > 256) return false;
    const int64_t pe = planes > 1 ? pstride : (int64_t)rows * pitch;          // plane extent
    const int64_t be = n > 1 ? bstride : (planes > 1 ? planes * pstride : (int64_t)rows * pitch);
    if (planes > 1 && ((pe & 15) || pe < (int64_t)rows * pitch)) return false;
    if (n > 1 && ((be & 15) || be < (planes > 1 ? planes * pe : (int64_t)rows * pitch))) return false;
    cuuint64_t dims[5];
    cuuint64_t strides[4];
    cuuint32_t box[5], es[5] = {1, 1, 1, 1, 1};
    int rank = 0;
    dims[rank] = (cuuint64_t)(rowbytes / 4); box[rank] = (cuuint32_t)(4 * box_chunks); ++rank;
    dims[rank] = (cuuint64_t)rows; box[rank] = (cuuint32_t)box_rows; strides[rank - 1] = (cuuint64_t)pitch; ++rank;
    if (planes > 1) {
        dims[rank] = (cuuint64_t)planes; box[rank] = 1; strides[rank - 1] = (cuuint64_t)pe; ++rank;
    }
    dims[rank] = (cuuint64_t)n; box[rank] = 1; strides[rank - 1] = (cuuint64_t)((be + 15) & ~(int64_t)15); ++rank;
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, rank, const_cast<void *>(base), dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// ---------------------------------------------------------------------------
// Per-operation launch
// ---------------------------------------------------------------------------
template <int OP, int CIN, int OUTK, int TH>
static cudaError_t launch_th(const OpDesc &d, cudaStream_t stream)
{
    constexpr int TW = kTW;
    auto kern_map = resample_kernel<OP, CIN, OUTK, TW, TH, false>;
    auto kern_rows = resample_kernel<OP, CIN, OUTK, TW, TH, CIN == 3>;
    constexpr int ob = out_stage_bytes<OUTK, CIN, TW, TH>();
    static unsigned attr_done = 0;   // one bit per device ordinal (< 32)
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 32 || !(attr_done & (1u << dev))) {
        const int max_smem = std::max(kFootCap, (int)kRawBoxCap + 128) + std::max(kRegionBCap, ob);
        cudaError_t e = cudaFuncSetAttribute(kern_map, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kern_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
        if (e != cudaSuccess) return e;
        if (dev < 32) __atomic_fetch_or(&attr_done, 1u << dev, __ATOMIC_RELAXED);
    }
    OpParams p;
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
    p.chw = d.chw;
    p.replicate = d.replicate;
    if (OP == OP_RESIZE && d.W < 32768 && d.w < 32768 && d.H < 32768 && d.h < 32768) {
        // the axis tables' divisions by 2w, 4w, 2h, 4h as multiply-high (resize_axis_m)
        const uint32_t den[4] = {2u * d.w, 4u * d.w, 2u * d.h, 4u * d.h};
        for (int k = 0; k < 4; ++k) p.rm[k] = 0xFFFFFFFFu / den[k];
    }
    for (int k = 0; k < 3; ++k) {
        p.scale[k] = d.scale[k];
        p.bias[k] = d.bias[k];
    }
    const int tiles_x = (d.w + TW - 1) / TW, tiles_y = (d.h + TH - 1) / TH;
    const int per_launch = OP != OP_RESIZE ? kMaxMPerLaunch : 65535;
    constexpr int nm = OP == OP_PERSP ? 9 : 6;   // floats per image map
    for (int b0 = 0; b0 < d.batch; b0 += per_launch) {
        const int nb = std::min(per_launch, d.batch - b0);
        Budget bud;
        std::memset(p.fast_mask, 0, sizeof(p.fast_mask));
        // Raw-tap box bound (3 channels): the largest tile box of the launch whose raw rows
        // (16-byte chunks) fit kRawBoxCap; it is independent of the re-laid layout's caps.
        int raw_cols = 0, raw_rows = 0;
        auto raw_bound = [&](const Budget &bi) {
            if (CIN != 3 || bi.cols < 1 || bi.rows < 1 || bi.cols >= 1000000) return;
            const long long raw = 16LL * ((15 + bi.cols * CIN + 15) / 16) * bi.rows + 16;
            if (raw > kRawBoxCap) return;
            raw_cols = std::max(raw_cols, bi.cols);
            raw_rows = std::max(raw_rows, bi.rows);
        };
        if (OP == OP_RESIZE) {
            bud = budget_resize(CIN, d.H, d.W, d.h, d.w, TW, TH, ob);
            raw_bound(bud);
        } else {
            bud.a = 0;
            bud.b = round16(ob);
            for (int i = 0; i < nb; ++i) {
                for (int k = 0; k < nm; ++k) p.M[i][k] = d.M[(size_t)(b0 + i) * nm + k];
                const Budget bi = OP == OP_PERSP ? budget_persp(CIN, d.H, d.W, p.M[i], d.h, d.w, TW, TH, ob)
                                                 : budget_warp(CIN, d.H, d.W, p.M[i], TW, TH, ob);
                bud.a = std::max(bud.a, bi.a);
                bud.b = std::max(bud.b, bi.b);
                if (bi.fits) {   // the TMA box covers every image whose tiles' boxes fit the caps
                    bud.cols = std::max(bud.cols, bi.cols);
                    bud.rows = std::max(bud.rows, bi.rows);
                }
                raw_bound(bi);
                if (warp_allows_fast(p.M[i], d.h, d.w)) p.fast_mask[i >> 5] |= 1u << (i & 31);
            }
        }
        p.src = d.src + (int64_t)b0 * d.sbatch;
        p.dst = d.dst + (int64_t)b0 * d.dbatch;
        p.has_tin = 0;
        p.raw_taps = 0;
        p.rows16 = ((uintptr_t)p.src & 15) == 0 && (d.spitch & 15) == 0 && (nb == 1 || (d.sbatch & 15) == 0);
        if (CIN == 3 && raw_cols > 0) {
            // 3-channel taps straight from the staged rows: region A holds the largest raw box
            // plus the 16 bytes that reading the last pixel pair may touch past it, region B
            // only the output tile; the rows come by one TMA copy per tile when the source
            // takes a map, else by bulk row copies when its rows are 16-byte aligned
            // The box row is padded to 4 mod 8 chunks when that fits: neighbouring staged rows are
            // then 16 banks apart, and the two half-warps of the 4-pixel quad path, which read
            // neighbouring rows, hit disjoint banks for unit-scale maps.
            int nc = (15 + raw_cols * CIN + 15) / 16;
            const int br = raw_rows;
            const int ncp = nc + ((12 - nc % 8) % 8);
            if (ncp <= 64 && 16LL * ncp * br + 16 <= kRawBoxCap) nc = ncp;
            if (encode_map(&p.tin, p.src, (int64_t)d.W * CIN, d.H, 1, nb, d.spitch, 0, d.sbatch, nc, br)) {
                p.has_tin = 1;
                p.tin_nc = nc;
                p.tin_br = br;
            }
            if (p.has_tin || p.rows16) {
                p.raw_taps = 1;
                bud.a = round128(16 * nc * br + 16);
                bud.b = round16(ob);
            }
        } else if (CIN == 1 && bud.a > 0 && bud.cols > 0 && bud.rows > 0) {
            // TMA source map: one box per tile covering the largest source box of the launch
            const int nc = (15 + bud.cols * CIN + 15) / 16, br = bud.rows;
            if ((long long)16 * nc * br <= bud.a - 16 &&
                encode_map(&p.tin, p.src, (int64_t)d.W * CIN, d.H, 1, nb, d.spitch, 0, d.sbatch, nc, br)) {
                p.has_tin = 1;
                p.tin_nc = nc;
                p.tin_br = br;
            }
        }
        p.foot_budget = bud.a;
        p.region_b = bud.b;
        // Destination rows that are whole 16-byte chunks at 16-byte aligned addresses (every row,
        // plane and image) are written straight from registers; region B then only served
        // 3-channel boxes re-laid from raw rows, which launches with raw taps stage by TMA or
        // bulk copies instead (the perspective warp keeps it for its most magnified tiles).
        constexpr int dC = OutTraits<OUTK, CIN>::dC, ES = OutTraits<OUTK, CIN>::esize;
        const bool chw = d.chw != 0;
        const int64_t orowb = chw ? (int64_t)d.w * 4 : (int64_t)d.w * dC * ES;
        p.direct = orowb % 16 == 0 && ((uintptr_t)p.dst & 15) == 0 && (d.dpitch & 15) == 0 && d.dpitch >= orowb &&
                   (!chw || (d.dplane & 15) == 0) && (nb == 1 || (d.dbatch & 15) == 0);
        if (p.direct && OP != OP_PERSP && (CIN == 1 || p.raw_taps)) bud.b = 0;
        p.region_b = bud.b;
        const size_t smem = (size_t)bud.a + bud.b;
        dim3 grid(tiles_x, tiles_y, nb);
        if (p.raw_taps && !p.has_tin)
            kern_rows<<<grid, kThreads, smem, stream>>>(p);
        else
            kern_map<<<grid, kThreads, smem, stream>>>(p);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Tile height of a launch: the kind's height, or 16 rows when the launch has too few tiles to
// fill the GPU for long (small images): a CTA's time grows with its rows plus a fixed part
// (planning and staging, about 24 rows' worth), and a launch takes as many of those as it has
// waves of CTAs (about 8 resident per SM).
template <int OP, int CIN, int OUTK>
static cudaError_t launch_t(const OpDesc &d, cudaStream_t stream)
{
    constexpr int TB = op_tile_h<OP, OUTK>(), TS = 16;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    const long long tiles_x = (d.w + kTW - 1) / kTW, slots = 8LL * sms;
    auto cost = [&](int th) {
        const long long ctas = tiles_x * ((d.h + th - 1) / th) * d.batch;
        return ((ctas + slots - 1) / slots) * (th + 24);
    };
    return cost(TS) < cost(TB) ? launch_th<OP, CIN, OUTK, TS>(d, stream) : launch_th<OP, CIN, OUTK, TB>(d, stream);
}

template <int OP>
static cudaError_t launch_op(const OpDesc &d, cudaStream_t s)
{
    if (d.cin == 3) {
        switch (d.outk) {
        case OUT_U8: return launch_t<OP, 3, OUT_U8>(d, s);
        case OUT_U8_GRAY: return launch_t<OP, 3, OUT_U8_GRAY>(d, s);
        case OUT_F32: return launch_t<OP, 3, OUT_F32>(d, s);
        case OUT_F32_GRAY: return launch_t<OP, 3, OUT_F32_GRAY>(d, s);
        }
    } else {
        switch (d.outk) {
        case OUT_U8: return launch_t<OP, 1, OUT_U8>(d, s);
        case OUT_F32: return launch_t<OP, 1, OUT_F32>(d, s);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_resample(const OpDesc &d, cudaStream_t stream)
{
    if (d.op == OP_RESIZE) return launch_op<OP_RESIZE>(d, stream);
    if (d.op == OP_PERSP) return launch_op<OP_PERSP>(d, stream);
    return launch_op<OP_WARP>(d, stream);
}

// ---------------------------------------------------------------------------
// Standalone RGB -> gray: one thread per 16-pixel chunk of a row (grid: chunks x
// rows x images, no index divisions). Rows whose source and destination start on
// 16-byte boundaries move 48 bytes in through three 128-bit loads and 16 bytes out
// through one 128-bit store, each gray one dp2a on the pixel's word; other rows and
// the ragged tail go pixel by pixel.
// ---------------------------------------------------------------------------
struct GrayParams {
    const uint8_t *src;
    int64_t spitch, sbatch;
    uint8_t *dst;
    int64_t dpitch, dbatch;
    int32_t H, W, chunks_x;
};

// (4899 R + 9617 G + 1868 B + 8192) >> 14 of the pixel in bytes 0..2 of P
__device__ __forceinline__ uint32_t gray_of_word(uint32_t P)
{
    return __dp2a_lo(4899u | (9617u << 16), P, 8192u + 1868u * ((P >> 16) & 255u)) >> 14;
}

__global__ void __launch_bounds__(kThreads) gray_kernel(const __grid_constant__ GrayParams p)
{
    const int cx = blockIdx.x * blockDim.x + threadIdx.x;
    if (cx >= p.chunks_x) return;
    const int y = blockIdx.y;
    const uint8_t *s = p.src + (int64_t)blockIdx.z * p.sbatch + (int64_t)y * p.spitch + (int64_t)cx * 48;
    uint8_t *d = p.dst + (int64_t)blockIdx.z * p.dbatch + (int64_t)y * p.dpitch + (int64_t)cx * 16;
    const int n = min(16, p.W - cx * 16);
    if (n == 16 && (((uintptr_t)s | (uintptr_t)d) & 15) == 0) {
        const uint4 a = __ldg(reinterpret_cast<const uint4 *>(s));
        const uint4 b = __ldg(reinterpret_cast<const uint4 *>(s + 16));
        const uint4 c = __ldg(reinterpret_cast<const uint4 *>(s + 32));
        const uint32_t w[13] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w, 0u};
        uint32_t o[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int bo = 3 * k;   // pixel k: bytes bo .. bo+2
            const uint32_t P = __funnelshift_r(w[bo >> 2], w[(bo >> 2) + 1], 8 * (bo & 3));
            o[k >> 2] |= gray_of_word(P) << (8 * (k & 3));
        }
        *reinterpret_cast<uint4 *>(d) = make_uint4(o[0], o[1], o[2], o[3]);
    } else {
        for (int k = 0; k < n; ++k)
            d[k] = (uint8_t)gray_u8(__ldg(s + 3 * k), __ldg(s + 3 * k + 1), __ldg(s + 3 * k + 2));
    }
}

cudaError_t device_error_flags(unsigned *flags, bool clear)
{
    cudaError_t e = cudaMemcpyFromSymbol(flags, g_kr_device_err, sizeof(unsigned));
    if (e == cudaSuccess && clear) {
        const unsigned zero = 0;
        e = cudaMemcpyToSymbol(g_kr_device_err, &zero, sizeof(unsigned));
    }
    return e;
}

cudaError_t set_stage_wait_ns_ops(unsigned long long ns)
{
    return cudaMemcpyToSymbol(g_kr_stage_wait_ns, &ns, sizeof(ns));
}

cudaError_t launch_gray(const GrayDesc &d, cudaStream_t stream)
{
    GrayParams p;
    p.src = d.src;
    p.spitch = d.spitch;
    p.sbatch = d.sbatch;
    p.dst = d.dst;
    p.dpitch = d.dpitch;
    p.dbatch = d.dbatch;
    p.H = d.H;
    p.W = d.W;
    p.chunks_x = (d.W + 15) / 16;
    const int bx = std::min(kThreads, 32 * ((p.chunks_x + 31) / 32));
    const dim3 grid((p.chunks_x + bx - 1) / bx, d.H, d.batch);
    gray_kernel<<<grid, bx, 0, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace kr
