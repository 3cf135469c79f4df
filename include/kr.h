/*
 * kr.h -- C ABI of the GB300 (sm_103a) image-resampling library.
 *
 * Operators: bilinear resize and affine warp of HWC u8 images, each with an
 * optional fused RGB -> gray and u8 -> f32 normalisation, a standalone
 * RGB -> gray, a ragged batch of such operations in one persistent launch,
 * and a continuous-batching serving loop built on the batch launch.
 *
 * Paper: Kornia-rs (arXiv 2505.12425). Sec. III names the image
 * transformations this library computes (horizontal flip, oversizing,
 * downsizing, RGB to grayscale); Sec. II-A places geometric transforms in
 * kornia-imgproc; Sec. II-B fixes the calling conventions followed here:
 * typed images Image<T, C> (element type + channel count), zero-copy views,
 * caller-owned pre-allocated output buffers and no hidden allocation, and
 * fallible calls that return an error instead of failing silently.
 *
 * Arithmetic (the paper prints none; these are the library's definitions):
 *   resize   sx = (x + 1/2) W / w - 1/2, clamp to the edge;
 *   warp     sx = fmaf(m00, x + 1/2, fmaf(m01, y + 1/2, m02)) - 1/2 (fp32,
 *            round to nearest even), sy likewise with m10, m11, m12; M maps
 *            destination pixels to source pixels; a tap outside the image
 *            reads 0; |sx| or |sy| >= 2^22 (or NaN) gives a 0 sample;
 *   u8       11-bit weights rounded half up, out = (v + 2^21) >> 22, exact;
 *   f32      value p/255 interpolated with fp32 weights, then
 *            (v - mean[c]) / std[c]; within 1e-5 of the exact result;
 *   gray     u8: (4899 R + 9617 G + 1868 B + 8192) >> 14 of the rounded u8
 *            interpolants; f32: 0.299 R + 0.587 G + 0.114 B of the f32
 *            interpolants, normalised with mean[0], std[0].
 *
 * Memory and streams. Every image pointer is a DEVICE address owned by the
 * caller; the library never allocates, frees or retains image memory. All
 * work is enqueued asynchronously on the given stream (NULL = the legacy
 * default stream) and the call returns at once; results are visible after
 * the stream is synchronised. Source and destination must not overlap.
 *
 * Errors. Every argument is validated on the host before anything is
 * enqueued; on a validation error nothing is enqueued and the status says
 * why. KR_ERR_CUDA reports a failed launch or CUDA runtime call; the text of
 * the last such error is returned by kr_last_error(). No call aborts,
 * traps or throws across the ABI.
 */
#ifndef KR_H
#define KR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (cudaStream_t / CUstream); NULL means the legacy default stream. */
typedef struct CUstream_st *kr_stream_t;

typedef enum { KR_U8 = 0, KR_F32 = 1 } kr_dtype;
typedef enum { KR_HWC = 0, KR_CHW = 1 } kr_layout;

typedef enum {
    KR_OK = 0,
    KR_ERR_INVALID_ARG = 1,   /* null pointer, bad size, pitch, dtype, layout or matrix */
    KR_ERR_UNSUPPORTED = 2,   /* a valid combination this library does not implement   */
    KR_ERR_ALIAS = 3,         /* source and destination memory overlap                 */
    KR_ERR_CUDA = 4,          /* a CUDA launch or runtime call failed                  */
    KR_ERR_NO_SPACE = 5,      /* workspace too small / request over the memory budget  */
    KR_ERR_TIMEOUT = 6        /* a bounded wait ran out                                */
} kr_status;

/*
 * An image, or a batch of equally sized images, in device memory
 * (Sec. II-B: Image<T, C> with zero-copy views).
 *
 *   data          address of channel 0 of pixel (0, 0) of image 0;
 *   height, width rows and columns, each >= 1;
 *   channels      1 or 3 (RGB order for 3);
 *   dtype         KR_U8 or KR_F32 (f32 only as a destination);
 *   layout        KR_HWC: pixel (y, x) channel c at data + y*pitch + (x*C + c)*esize;
 *                 KR_CHW (f32 destinations only): at data + c*plane_stride + y*pitch + x*4;
 *   batch         number of images (1 .. 65535); image n starts at data + n*batch_stride;
 *   pitch         bytes between rows, >= width*C*esize (HWC) or width*4 (CHW);
 *   plane_stride  bytes between channel planes (CHW; ignored for HWC);
 *   batch_stride  bytes between images (ignored when batch == 1).
 * A sub-rectangle of a larger image is described by moving `data` and keeping
 * the parent's pitch. f32 images need 4-byte aligned data and strides.
 */
typedef struct {
    void *data;
    int32_t height;
    int32_t width;
    int32_t channels;
    int32_t dtype;
    int32_t layout;
    int32_t batch;
    int64_t pitch;
    int64_t plane_stride;
    int64_t batch_stride;
} kr_image_t;

/* Fused epilogue flags. */
#define KR_GRAY      1u   /* 3-channel source -> 1-channel destination (BT.601)          */
#define KR_NORMALIZE 2u   /* f32 destination: (v - mean[c]) / std[c]; needs dtype KR_F32 */
#define KR_BORDER_REPLICATE 4u /* warps only: taps outside the image read the nearest edge
                                  pixel instead of zero (resize: KR_ERR_INVALID_ARG) */

/*
 * Fused epilogue (Sec. III: RGB to grayscale; u8 -> f32 normalisation).
 * NULL means "none". An f32 destination without KR_NORMALIZE stores v = p/255
 * (mean 0, std 1). std[c] must be finite and nonzero, mean[c] finite.
 */
typedef struct {
    uint32_t flags;
    float mean[3];
    float std[3];
} kr_post_t;

/*
 * Bilinear resize (Sec. III "oversizing, downsizing").
 * src: u8, HWC, C = 1 or 3. dst: same batch as src; its height and width are
 * the output size (Sec. II-B: the caller pre-allocates the output and its size
 * defines the operation). dst channels = src channels, or 1 with KR_GRAY
 * (src C = 3). dst dtype KR_U8 (HWC) or KR_F32 (HWC or CHW).
 * Returns KR_OK once the work is enqueued on `stream`.
 */
kr_status kr_resize_bilinear(const kr_image_t *src, const kr_image_t *dst,
                             const kr_post_t *post, kr_stream_t stream);

/*
 * Affine warp with a 2x3 inverse map (Sec. II-A "geometric transforms";
 * Sec. III "horizontal flip" is the map [-1 0 W; 0 1 0]).
 * M: HOST pointer to batch x 6 floats, row-major [m00 m01 m02 m10 m11 m12]
 * per image, mapping destination pixel centres to source pixel centres. The
 * floats are copied before the call returns. Non-finite entries give
 * KR_ERR_INVALID_ARG. Zero border, tap by tap. dst as for resize.
 */
kr_status kr_warp_affine(const kr_image_t *src, const kr_image_t *dst, const float *M,
                         const kr_post_t *post, kr_stream_t stream);

/*
 * Perspective warp (the projective generalisation of kr_warp_affine; the
 * paper names geometric transforms, Sec. II-A, and prints no convention).
 * M: HOST pointer to batch x 9 floats, row-major 3x3 per image, mapping
 * destination pixel centres to source pixel centres in homogeneous
 * coordinates: X, Y, Z = fmaf(m_r0, x + 0.5, fmaf(m_r1, y + 0.5, m_r2)),
 * q = 1/Z, sx = X q - 0.5, sy = Y q - 0.5 (fp32, round to nearest). Where
 * Z <= 0 the sample is zero; otherwise taps, weights, border, post and dst
 * rules as for kr_warp_affine (with the last row (0, 0, 1) the results equal
 * kr_warp_affine's bit for bit). Non-finite entries give KR_ERR_INVALID_ARG.
 */
kr_status kr_warp_perspective(const kr_image_t *src, const kr_image_t *dst, const float *M,
                              const kr_post_t *post, kr_stream_t stream);

/*
 * RGB -> gray (Sec. III "RGB to grayscale"; Sec. IV-B gray_from_rgb takes an
 * Image<u8,3> and a pre-allocated Image<u8,1> of the same size).
 * src: u8 HWC C = 3. dst: u8 HWC C = 1, same height, width and batch.
 */
kr_status kr_rgb_to_gray(const kr_image_t *src, const kr_image_t *dst, kr_stream_t stream);

/*
 * Nearest-neighbour resize (Sec. IV-A: the Python bindings' "nearest-neighbor
 * resizing"; the paper gives no convention). Half-pixel centres: output pixel
 * (x, y) copies source pixel (((2x + 1) W) div (2w), ((2y + 1) H) div (2h)),
 * the one covering the output pixel's centre. src, dst: u8 HWC, the same
 * channels (1 or 3) and batch; dst's size is the output size. Bit-exact copy of
 * source bytes. Errors as for kr_resize_bilinear; nothing is enqueued on error.
 */
kr_status kr_resize_nearest(const kr_image_t *src, const kr_image_t *dst, kr_stream_t stream);

/*
 * Horizontal flip (Sec. IV-A, one of the geometric transforms of the Rust
 * benchmark): dst(y, x) = src(y, W - 1 - x). src, dst: u8 HWC, the same size,
 * channels (1 or 3) and batch, not overlapping (KR_ERR_ALIAS: no in-place flip).
 */
kr_status kr_flip_horizontal(const kr_image_t *src, const kr_image_t *dst, kr_stream_t stream);

/*
 * Area (antialiased) downscale (a variant of the resize for strong reductions
 * such as 3840x2160 -> 224x224, where 4-tap bilinear aliases; the paper names
 * downsizing, Sec. III, without a convention). Output pixel (x, y) is the
 * mean of the source over [x W/w, (x+1) W/w) x [y H/h, (y+1) H/h), each
 * source pixel weighted by its overlap area (exact integer weights); u8 dst:
 * that mean rounded half up; f32 dst: mean / 255, then the fused normalise.
 * src: u8 HWC C = 1 or 3. dst: same channels and batch (no KR_GRAY),
 * w <= W and h <= H (else KR_ERR_INVALID_ARG). KR_ERR_UNSUPPORTED when two
 * source rows of one output column's footprint exceed 96 KB of shared memory
 * (more than about 16000 source columns per output column with 3 channels,
 * 49000 with 1), reported before anything is enqueued.
 */
kr_status kr_resize_area(const kr_image_t *src, const kr_image_t *dst, const kr_post_t *post, kr_stream_t stream);

/*
 * Sobel gradient magnitude (Sec. V: the robotics example calls
 * imgproc::filter::sobel(&img, &mut out, 3) on an RGB8 image into a Gray8
 * image; the paper gives no formula). ksize must be 3 (KR_ERR_UNSUPPORTED
 * otherwise). src: u8 HWC, C = 1, or C = 3 (first the u8 BT.601 gray of
 * kr_rgb_to_gray). Border: the edge pixel is replicated. With the integer
 * Sobel sums gx, gy of [-1 0 1; -2 0 2; -1 0 1] and its transpose,
 * m = sqrt(gx^2 + gy^2) / 8 (fp32, one rounding of the square root);
 * dst: C = 1, same size and batch, f32 (m) or u8 (floor(m + 1/2), <= 181).
 */
kr_status kr_sobel(const kr_image_t *src, const kr_image_t *dst, int32_t ksize, kr_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Ragged batch: many independent operations in one persistent launch.      */
/* ------------------------------------------------------------------------ */

typedef enum { KR_OP_RESIZE = 0, KR_OP_WARP = 1, KR_OP_GRAY = 2 } kr_op;

/*
 * One item of a ragged batch. src and dst follow the rules of the matching
 * single-image call, with batch == 1. M is used by KR_OP_WARP only; post by
 * KR_OP_RESIZE and KR_OP_WARP.
 */
typedef struct {
    int32_t op;
    kr_image_t src;
    kr_image_t dst;
    float M[6];
    kr_post_t post;
} kr_work_t;

/*
 * Launch options. tile_config: -1 = the choice kr_autotune_batch cached for
 * this batch's shape class, else configuration 0; or an index
 * < kr_tile_config_count(). ctas_per_sm: 0 = the occupancy limit.
 * use_graph: nonzero = replay the launch from a CUDA graph captured once per
 * (stream, workspace, configuration).
 */
typedef struct {
    int32_t tile_config;
    int32_t ctas_per_sm;
    int32_t use_graph;
} kr_batch_opts_t;

/* Device workspace bytes that kr_batch_submit needs for up to max_items items. */
size_t kr_batch_workspace_size(int32_t max_items);

/*
 * Run n work items in one persistent launch (no counterpart in the paper:
 * this is the batching form of the operators above).
 * items: HOST array of n items; it is copied before the call returns.
 * workspace: caller-owned DEVICE buffer of ws_bytes >= kr_batch_workspace_size(n);
 * it holds the device work list and must not be used by another submit that
 * may run concurrently. opts: NULL = defaults (autotuned tile, no graph).
 * Each item's result equals the matching single-image call's bit for bit.
 */
kr_status kr_batch_submit(const kr_work_t *items, int32_t n, void *workspace,
                          size_t ws_bytes, const kr_batch_opts_t *opts, kr_stream_t stream);

/*
 * kr_batch_submit without a workspace and without any allocation.
 *
 * The paper has no counterpart of this call. It exists for callers that cannot
 * allocate device memory at the point where they submit work: real-time loops
 * that forbid allocation on their hot path (an allocation can block or fail at
 * an unpredictable moment), host frameworks whose own allocator owns all device
 * memory, and code that cannot keep a workspace alive between calls. Such a
 * caller passes only the items (their images are the inputs and outputs it
 * already owns); the work list goes into a fixed device array inside this
 * library instead of a workspace.
 *
 * Limits and behaviour:
 *   - at most KR_BATCH_NOALLOC_MAX_ITEMS items per call; more gives
 *     KR_ERR_NO_SPACE with nothing enqueued;
 *   - the array (about 132 KiB) is a file-scope __device__ array: every GPU that
 *     loads the library holds it until the process exits;
 *   - the first call on a device looks up the array's device address for that
 *     device (cudaGetSymbolAddress); make that first call before any stream
 *     capture;
 *   - every call shares the one array and overwrites it (the tile counter is
 *     reset by each call's copy): calls whose work may overlap on the GPU race,
 *     so serialise them (one stream, or events between streams);
 *   - calls no cudaMalloc, cudaFree, cudaHostAlloc or other allocating routine;
 *     the work list is copied from a fixed (pageable) host array with
 *     cudaMemcpyAsync, so the call first waits for the work already on `stream`
 *     to finish (CUDA synchronises a pageable host-to-device copy with its stream)
 *     and returns once that array has been read;
 *   - a call made while `stream` is being captured into a CUDA graph returns
 *     KR_ERR_UNSUPPORTED and enqueues nothing: a captured copy would read the
 *     shared host array again at every replay, after later calls changed it;
 *   - kr_shutdown forgets the looked-up device addresses: call it before a
 *     cudaDeviceReset, after which the next call looks the address up again;
 *   - opts: tile_config < 0 means configuration 0 (no autotune lookup),
 *     ctas_per_sm as for kr_batch_submit, use_graph is ignored.
 * Results equal kr_batch_submit's bit for bit.
 */
#define KR_BATCH_NOALLOC_MAX_ITEMS 1024
kr_status kr_batch_submit_noalloc(const kr_work_t *items, int32_t n, const kr_batch_opts_t *opts,
                                  kr_stream_t stream);

/* Number of tile configurations the batch launch can use, and their shapes. */
int32_t kr_tile_config_count(void);
kr_status kr_tile_config_shape(int32_t index, int32_t *tile_w, int32_t *tile_h);

/*
 * Time every tile configuration x CTA count on these items (the outputs are
 * written several times) and remember the fastest for this batch's shape
 * class. Synchronises `stream`. best_config / best_ctas_per_sm may be NULL.
 */
kr_status kr_autotune_batch(const kr_work_t *items, int32_t n, void *workspace,
                            size_t ws_bytes, kr_stream_t stream,
                            int32_t *best_config, int32_t *best_ctas_per_sm);

/* Save / load the autotune cache as a small JSON text file. */
kr_status kr_autotune_save(const char *path);
kr_status kr_autotune_load(const char *path);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of an open-loop request stream.             */
/* ------------------------------------------------------------------------ */

/*
 * One request (no counterpart in the paper: the serving form of the operators,
 * motivated by Sec. II-B's predictable-latency goal for pre-allocated buffers).
 * op: KR_OP_RESIZE / KR_OP_WARP / KR_OP_GRAY on source image src_index of the
 * pool; output out_h x out_w u8 HWC with 3 channels (1 for gray, which needs the
 * source's size); M: the warp's 2x3 destination -> source map; t_arrival:
 * scheduled arrival in seconds from the start of the run, non-decreasing.
 */
typedef struct {
    int32_t op;
    int32_t src_index;
    int32_t out_h, out_w;
    float M[6];
    double t_arrival;
} kr_request_t;

/*
 * pool / pool_n: device-resident u8 HWC 3-channel source images (batch 1), owned
 * by the caller; out_arena / out_arena_bytes: caller-owned DEVICE memory from
 * which each request's output is carved (256-byte aligned, dense rows);
 * hbm_budget_bytes: at most this many source + output bytes in flight (0 = no
 * limit); max_batch: items per ragged launch; streams: launches in flight (the
 * library creates and destroys these streams and their events); policy: 0 =
 * continuous batching (kr_batch_submit on a free slot with every admitted
 * request), 1 = one launch per request, 2 = size-aware continuous batching (every
 * admitted request of at least direct_px output pixels is launched alone at once,
 * round-robin over the streams as in policy 1; the smaller ones wait for a free
 * slot and share one kr_batch_submit on its stream: large images fill the GPU by
 * themselves, small ones share a launch);
 * workspaces / ws_bytes_each: policies 0 and 2
 * only, `streams` device workspaces of ws_bytes_each >=
 * kr_batch_workspace_size(max_batch) bytes, caller-owned; retain_outputs: 0 =
 * a request's arena space is reused once it completes (the client is taken to
 * consume each output at its completion), 1 = every output keeps its space until
 * the run ends (the arena must then hold all outputs, else KR_ERR_NO_SPACE);
 * direct_px: policy 2's threshold (0 = 2^20 output pixels).
 */
typedef struct {
    const kr_image_t *pool;
    int32_t pool_n;
    void *out_arena;
    size_t out_arena_bytes;
    size_t hbm_budget_bytes;
    int32_t max_batch;
    int32_t streams;
    int32_t policy;
    void *workspaces;
    size_t ws_bytes_each;
    int32_t retain_outputs;
    int64_t direct_px;
} kr_serve_config_t;

/* Per request: admission, launch and observed completion times (seconds from the
 * start of the run, host steady clock) and the output's byte offset in the arena. */
typedef struct {
    double t_admit, t_launch, t_done;
    int64_t out_offset;
    int32_t status;
} kr_serve_result_t;

/*
 * Run the request stream to completion in real time on the calling thread
 * (busy-polling). Requests wait (in arrival order) while admitting them would
 * exceed the budget or the arena; requests that arrive while others run are
 * admitted and launched as soon as a slot frees. Every request is validated
 * before anything runs (KR_ERR_INVALID_ARG / KR_ERR_NO_SPACE, nothing launched).
 * Returns when every request is complete or dropped. Results equal the
 * single-image calls'.
 *
 * Every request ends in one of two states: completed (status KR_OK, t_done set,
 * output in the arena) or dropped (status != KR_OK, t_done = -1, no output).
 *   - a launch that fails drops its requests (status = the launch's status); their
 *     bytes leave the budget, their arena space is freed and the run goes on;
 *   - when recording a launch's completion event fails, the loop waits for that
 *     launch's stream and completes its requests;
 *   - an error reported by the device (an event query) stops the run: it returns
 *     KR_ERR_CUDA and every request not completed is dropped with KR_ERR_CUDA;
 *   - when retained outputs fill the arena so that the next request can never be
 *     admitted, the run returns KR_ERR_NO_SPACE and drops the rest with it.
 * The return value is KR_OK when the run went to the end (dropped requests are
 * reported through their own status).
 */
kr_status kr_serve_run(const kr_request_t *reqs, int32_t n, const kr_serve_config_t *cfg,
                       kr_serve_result_t *results);

/* ------------------------------------------------------------------------ */
/* Misc.                                                                    */
/* ------------------------------------------------------------------------ */

/* Static text for a status code. */
const char *kr_status_string(kr_status status);

/* Text of the last KR_ERR_CUDA in this thread ("" if none). */
const char *kr_last_error(void);

/*
 * Device-side error flags of the single-image and ragged kernels, read
 * synchronously (the current device). Bit 0: a bounded wait for a tile's
 * staging copy (TMA or bulk row copies) ran out (the tile was skipped and its
 * output left unwritten). clear != 0 resets the flags.
 */
#define KR_DEVERR_TMA_TIMEOUT 1u
kr_status kr_device_errors(uint32_t *flags, int32_t clear);

/* Release graphs, pinned staging and caches the library holds. Idempotent. */
void kr_shutdown(void);

/* ------------------------------------------------------------------------ */
/* Test hooks: the failure paths, exercised without faulting a GPU. The     */
/* paper has no counterpart of these.                                       */
/* ------------------------------------------------------------------------ */

/*
 * Bound, in nanoseconds, of the FIRST wait of every tile kernel (single-image and
 * ragged) for its staged source box, on the current device; default 2e9. ns = 0
 * makes that wait give up at once: every staged tile records KR_DEVERR_TMA_TIMEOUT,
 * waits with the full 2 s bound for its copies to land and is abandoned without
 * writing its output (tiles that stage nothing are written as usual). The second
 * wait keeps its bound, so no kernel exits with a copy in flight. Applies to the
 * kernels launched after the call.
 */
kr_status kr_debug_set_stage_wait_ns(uint64_t ns);

/*
 * Make one host-side step of kr_serve_run fail on every period-th time it runs
 * (period 0 = never, the default); process-wide, until changed:
 *   KR_FAULT_SUBMIT  a launch (batch or single request) returns KR_ERR_CUDA;
 *   KR_FAULT_EVENT   recording a launch's completion event fails;
 *   KR_FAULT_ADMIT   an arena allocation fails (as when the arena is full).
 */
#define KR_FAULT_SUBMIT 1
#define KR_FAULT_EVENT 2
#define KR_FAULT_ADMIT 3
kr_status kr_debug_set_fault(int32_t site, int32_t period);

#ifdef __cplusplus
}
#endif

#endif /* KR_H */
