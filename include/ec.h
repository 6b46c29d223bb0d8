/*
 * ec.h -- C ABI of libec, GB300 (sm_103a) sort-last image compositing and
 * run-length pixel coding, after Eilemann, "Parallel Rendering and Large Data
 * Visualization" (arXiv 1902.08755), chapter 5 "Compositing".
 *
 * The thesis states the compositing problem as: N input frames, each with
 * colour (and optionally depth) buffers, a pixel viewport and a region of
 * interest, combined in a given order into one destination frame (3.6, 5.2,
 * 5.3).  Every entry point below is one step of that problem, run by
 * hand-written CUDA kernels on the caller's stream.
 *
 * Conventions
 *  - Coordinates are destination-frame pixels.  A rect {x, y, w, h} covers
 *    x <= px < x+w, y <= py < y+h; w, h >= 0 (0 = empty).
 *  - An image stores the pixels of its pvp ("pixel viewport"): pixel (px, py)
 *    is element (py - pvp.y) * pitch + (px - pvp.x) of its buffers; pitch is in
 *    pixels and >= pvp.w.  Its roi (region of interest, thesis 5.3) is a
 *    sub-rectangle of pvp; outside the roi the image is background (depth mode)
 *    or fully transparent (alpha mode) and is never read.
 *  - Ownership: the caller owns every image, target, stream and gradient
 *    buffer.  libec allocates only what an ec_ctx or ec_batch holds and frees
 *    it in ec_destroy / ec_batch_free.
 *  - Asynchrony: every call enqueues work on stream s and returns at once.  The
 *    return value reports argument validation only (and CUDA launch errors).
 *    Errors found on the device (corrupt stream, wait timeout) are recorded in
 *    the context's device status word, and ec_status_sync reports them.  A
 *    kernel that finds an error stops early and never writes outside the
 *    caller's buffers.
 *  - Pointers are device pointers unless marked "host".  Host arrays are read
 *    before the call returns and may be freed afterwards.
 *  - Vector path: when an image's colour/depth pointers are 16-byte aligned,
 *    pitch * bytes-per-pixel is a multiple of 16 and its pvp.x is offset from
 *    the target's pvp.x by a multiple of 16 bytes of pixels, kernels move 16
 *    bytes per access; otherwise they fall back to per-pixel accesses.  Both
 *    give identical results.
 *  - A context is used from one host thread at a time; calls on one context
 *    that overlap on the device must be on the same stream (they share its
 *    scratch memory and status word).
 */
#ifndef EC_H
#define EC_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EC_OK = 0,
    EC_ERR_INVALID_ARG = 1,  /* bad rect, size, pointer, format or order      */
    EC_ERR_CAPACITY = 2,     /* destination smaller than ec_rle_max_size      */
    EC_ERR_CUDA = 3,         /* a CUDA runtime call failed                    */
    EC_ERR_CORRUPT = 4,      /* malformed run-length stream (device-side)     */
    EC_ERR_UNSUPPORTED = 5,  /* valid but outside this build's limits         */
    EC_ERR_TIMEOUT = 6       /* a bounded device-side wait gave up            */
} ec_status;

typedef struct { int32_t x, y, w, h; } ec_rect;

typedef enum {
    EC_RGBA8 = 0,    /* uint32 per pixel, R in the low byte                    */
    EC_RGBA32F = 1,  /* float[4] per pixel, premultiplied in alpha mode        */
    EC_RGBA16F = 2   /* IEEE half[4] per pixel, premultiplied in alpha mode    */
} ec_format;

typedef void* ec_stream_t; /* a cudaStream_t; NULL = the legacy default stream */

/* One input frame (thesis 3.6: an input frame with colour/depth buffers, a
 * pixel viewport and a region of interest). */
typedef struct {
    ec_rect pvp;        /* rectangle the stored pixels cover                   */
    ec_rect roi;        /* sub-rectangle of pvp holding data                   */
    int32_t pitch;      /* pixels per stored row, >= pvp.w                     */
    int32_t format;     /* ec_format of color                                  */
    const void* color;  /* [pvp.h][pitch] pixels                               */
    const float* depth; /* [pvp.h][pitch] depth, depth mode only (else NULL)   */
} ec_image;

/* The destination frame. */
typedef struct {
    ec_rect pvp;        /* rectangle the output covers                         */
    int32_t pitch;      /* pixels per row, >= pvp.w                            */
    int32_t format;     /* ec_format of color                                  */
    void* color;        /* [pvp.h][pitch] pixels, written in full              */
    float* depth;       /* [pvp.h][pitch] depth out, or NULL                   */
} ec_target;

typedef struct ec_ctx ec_ctx;

/* Limits of this build. */
#define EC_MAX_SOURCES 512          /* images per compositing call            */
#define EC_RLE_CHUNK 4096           /* elements per independently coded chunk */
#define EC_RLE_MAX_ELEMS (1u << 27) /* elements per run-length coded image    */
#define EC_RLE_MAX_JOBS 512         /* images per batched codec call          */

/* Create a context on CUDA device `device`: a device status word and scratch
 * memory for the codec.  *ctx is NULL on failure. */
ec_status ec_create(ec_ctx** ctx, int device);
void ec_destroy(ec_ctx* ctx);

/* Wait for stream s, then return the first device-side error recorded since
 * the last call (EC_OK if none) and clear it. */
ec_status ec_status_sync(ec_ctx* ctx, ec_stream_t s);

/* Self-test of failure detection without a fault: one warp runs the
 * compressor's bounded mbarrier wait (the one kind of wait in libec's kernels)
 * on a barrier that nothing arrives on.  The wait gives up after its try limit
 * (2^20 tries of at most about a microsecond each), records EC_ERR_TIMEOUT in
 * the status word and the kernel returns, leaving the context usable.  Read
 * the result with ec_status_sync. */
ec_status ec_selftest_wait_timeout(ec_ctx* ctx, ec_stream_t s);

/* Human-readable name of a status code (static string). */
const char* ec_status_string(ec_status st);

/* ---------------------------------------------------------------- compositing
 * Depth-sorted sort-last compositing, thesis 5.2.1: every output pixel takes
 * the colour and depth of the input with the smallest depth there.  Inputs may
 * arrive in any order (thesis 3.6, 5.6), so ties go to the lower input index;
 * the cleared background (colour bytes 0, depth 1.0) wins ties at 1.0 and NaN
 * depths never win.  Inputs are read only inside roi_i ∩ out->pvp (thesis 5.3).
 *   in      host array of n images; all share one colour format
 *           (EC_RGBA8 or EC_RGBA32F), depth must be non-NULL.
 *   out     colour (same format) over the whole out->pvp; depth if non-NULL.
 *   winner  device int16 [out->pvp.h][out->pvp.w] (dense), index of the
 *           winning input or -1, or NULL.  Needed by the backward pass.
 *   out_roi host, may be NULL: bounding box of the union of roi_i ∩ out->pvp,
 *           {0,0,0,0} if empty (thesis 5.3, the merged ROI).
 * n == 0 writes the background.  n <= EC_MAX_SOURCES. */
ec_status ec_composite_depth(ec_ctx* ctx, const ec_image* in, int32_t n,
                             const ec_target* out, int16_t* winner,
                             ec_rect* out_roi, ec_stream_t s);

/* Ordered sort-last compositing, thesis 5.2.1 (spatial decomposition, images
 * blended in sorted order): front-to-back Porter-Duff "over" of premultiplied
 * RGBA, C += T * c_k, T *= (1 - a_k), in FP32 arithmetic.
 *   in      host array of n layers, all EC_RGBA32F or all EC_RGBA16F.
 *   order   host array of n distinct layer indices, order[0] in front; NULL
 *           means 0..n-1.
 *   out     same format as the layers, written over the whole out->pvp.
 *   t_final device float [out->pvp.h][out->pvp.w] (dense) remaining
 *           transmittance, or NULL.
 * Outside roi_k a layer is transparent.  n <= EC_MAX_SOURCES. */
ec_status ec_composite_alpha(ec_ctx* ctx, const ec_image* in, const int32_t* order,
                             int32_t n, const ec_target* out, float* t_final,
                             ec_rect* out_roi, ec_stream_t s);

/* Backward pass of ec_composite_alpha for L = sum(grad_out * out): writes
 *   dL/dc_k^{RGB} = g^{RGB} T_k,  dL/da_k = T_k (g^A - R_k),
 *   R_k = sum_{j>k} g.c_j prod_{k<m<j} (1 - a_m)   (reverse "behind" scan),
 * recomputing T_k on chip (no per-layer state is stored by the forward).
 *   out_pvp    the forward's output viewport.
 *   grad_out   device float4 [out_pvp.h][out_pvp.w] (dense), upstream gradient.
 *   grad       host array of n device pointers; grad[i] has layer i's shape
 *              ([pvp_i.h][pitch_i] pixels of grad_format, EC_RGBA32F or
 *              EC_RGBA16F) and is written over pvp_i ∩ out_pvp (0 outside
 *              roi_i); other elements are not written. */
ec_status ec_composite_alpha_backward(ec_ctx* ctx, const ec_image* in,
                                      const int32_t* order, int32_t n, ec_rect out_pvp,
                                      const float* grad_out, void* const* grad,
                                      int32_t grad_format, ec_stream_t s);

/* Forward and backward in one pass, for a loss L = sum(w * out) whose weights
 * w are known before the forward (w = grad_out above).  Reads every layer
 * once; writes out (and t_final if non-NULL) like ec_composite_alpha and the
 * gradients like ec_composite_alpha_backward. */
ec_status ec_composite_alpha_fwd_bwd(ec_ctx* ctx, const ec_image* in,
                                     const int32_t* order, int32_t n,
                                     const ec_target* out, float* t_final,
                                     const float* w, void* const* grad,
                                     int32_t grad_format, ec_rect* out_roi,
                                     ec_stream_t s);

/* Backward pass of ec_composite_depth with EC_RGBA32F colour: an output pixel
 * is a copy of its winner's colour, so grad_i[p] = grad_out[p] where
 * winner[p] == i and 0 elsewhere (no gradient reaches depth).
 *   winner   device int16 [out_pvp.h][out_pvp.w] from the forward.
 *   grad_out device float4 [out_pvp.h][out_pvp.w] (dense).
 *   pvps, pitches  host arrays of n: each input's pvp and pitch.
 *   grad     host array of n device float4 buffers of the inputs' shapes,
 *            written over pvp_i ∩ out_pvp. */
ec_status ec_composite_depth_backward(ec_ctx* ctx, const int16_t* winner,
                                      ec_rect out_pvp, const float* grad_out,
                                      int32_t n, const ec_rect* pvps,
                                      const int32_t* pitches, float* const* grad,
                                      ec_stream_t s);

/* --------------------------------------------------------- batched compositing
 * Many independent composites in one persistent launch.  Thesis 4.2.4 (tile
 * compounds): fixed-size work packages wait in a queue and are pulled until it
 * is empty, which balances uneven work.  A plan cuts every job's destination
 * into tiles (work items), sorts them by estimated cost (largest first),
 * uploads all descriptors once and captures one launch -- a queue-head reset
 * and a grid of resident CTAs that pull items with an atomic counter -- in a
 * CUDA graph; ec_batch_run replays that graph.  Results are bit-identical to
 * calling ec_composite_depth / ec_composite_alpha per job, whatever the tile
 * shapes. */
enum { EC_JOB_DEPTH = 0, EC_JOB_ALPHA = 1 };
#define EC_MAX_BATCH_INPUTS 128     /* inputs per job of a batch              */

typedef struct {
    int32_t mode;           /* EC_JOB_DEPTH or EC_JOB_ALPHA                        */
    int32_t n;              /* inputs, <= EC_MAX_BATCH_INPUTS                      */
    const ec_image* in;     /* host array of n (read while planning)               */
    const int32_t* order;   /* alpha: host array of n or NULL; depth: ignored      */
    ec_target out;          /* destination, as in the single calls                 */
    int16_t* winner;        /* depth: optional winner plane                        */
    float* t_final;         /* alpha: optional transmittance                       */
} ec_job;

/* Tile shapes per job kind, in pixels.  Widths are multiples of the pixels a
 * warp covers in a row: 128 for depth jobs, 32 for RGBA32F and 64 for RGBA16F
 * alpha jobs.  ctas_per_sm = 0 means as many as fit. */
typedef struct {
    int32_t depth_tile_w, depth_tile_h;
    int32_t alpha32_tile_w, alpha32_tile_h;
    int32_t alpha16_tile_w, alpha16_tile_h;
    int32_t ctas_per_sm;
} ec_batch_config;

typedef struct ec_batch ec_batch;

/* Validate the jobs and build a plan.  cfg == NULL autotunes: every candidate
 * tile shape is timed on the jobs themselves (so planning runs the batch, and
 * writes the destinations, several times) and the fastest is kept; the choice
 * is cached per device and job signature for the process (and in the file
 * named by the environment variable EC_AUTOTUNE_CACHE, if set).  The plan
 * refers to the callers' buffers by address: they must stay allocated and in
 * place until ec_batch_free.  Planning allocates device memory and
 * synchronises the device. */
ec_status ec_batch_plan(ec_ctx* ctx, const ec_job* jobs, int32_t njobs,
                        const ec_batch_config* cfg, ec_batch** plan);
/* Enqueue the captured launch on stream s.  Every replay of one plan resets
 * and advances the same device-side queue head, so replays of one plan must
 * not overlap on the GPU: issue them on one stream, or order them with events.
 * Overlapping replays would skip or repeat work items and leave the
 * destinations wrong without any error.  Distinct plans are independent. */
ec_status ec_batch_run(ec_batch* plan, ec_stream_t s);
/* The plan's tile shapes, work-item count and grid size (host pointers, any may be NULL). */
ec_status ec_batch_get_config(const ec_batch* plan, ec_batch_config* cfg, int32_t* n_items,
                              int32_t* grid);
void ec_batch_free(ec_batch* plan);

/* ------------------------------------------------ multi-stage compositing schedules
 * Thesis 5.2.2 (direct send, binary swap, 2-3 swap) and 5.2.3 (streaming
 * sort-last compositing).  The n inputs stand for n rendering resources.  In
 * stages, resources send parts of their partial frames to others; a receiver
 * composites what it holds with what it receives, source by source in index
 * order (depth: ec_composite_depth's merge and tie rule; alpha: front-to-back
 * "over" in the order given).  At the end each resource owns a part of the
 * frame and writes it into out (the stream's last resource owns all of it).
 * A transfer carries only the sender's ROI inside the region sent (thesis
 * 5.3).  The result equals ec_composite_depth of all inputs bit for bit; for
 * alpha it equals ec_composite_alpha up to the rounding of the partials.
 *
 * Geometry (all in out->pvp coordinates; a rectangle R cut into k row bands
 * gives band j the rows [R.y + floor(j R.h / k), R.y + floor((j+1) R.h / k))):
 *   EC_SCHED_STREAM        stage l (l = 0..n-2): resource l sends its whole
 *                          partial frame to l+1, which composites it in front
 *                          of its own image.
 *   EC_SCHED_DIRECT_SEND   one stage: resource i owns row band i of n and
 *                          receives every other resource's pixels there.
 *   EC_SCHED_BINARY_SWAP   n a power of two; stage l pairs u = a + j with
 *                          u + 2^l (a a multiple of 2^(l+1)); their common
 *                          region is halved across its longer side (rows when
 *                          h >= w, the first half floor(len/2)); u keeps the
 *                          first half, u + 2^l the second.
 *   EC_SCHED_TWO_THREE_SWAP  any n: the current units (first the single
 *                          resources) are grouped consecutively in pairs, the
 *                          last group a triple if their count is odd; a
 *                          group's resources, ordered by the first row of the
 *                          region they hold and then by unit, get the frame's
 *                          row bands in that order and receive from every
 *                          group member the part of their band it holds.
 * A receiver's new ROI is the bounding box of the pieces it composites.
 *
 * flags:
 *   EC_SCHED_RLE    transfers are RLE-compressed by the sender and decoded by
 *                   the receiver (depth mode with EC_RGBA8 only: colour mode 2,
 *                   depth mode 1).  Without it transfers are read in place.
 *   EC_SCHED_FUSED  with EC_SCHED_RLE: stages that merge the receiver's own
 *                   image with the pieces of one other unit (every stage of
 *                   the stream and of binary swap) decode inside the
 *                   composite, never writing the decoded pieces.
 */
typedef enum {
    EC_SCHED_STREAM = 0,
    EC_SCHED_DIRECT_SEND = 1,
    EC_SCHED_BINARY_SWAP = 2,
    EC_SCHED_TWO_THREE_SWAP = 3
} ec_sched_algorithm;

#define EC_SCHED_RLE 1u
#define EC_SCHED_FUSED 2u

typedef struct {
    int32_t level;      /* stage of the schedule, from 0                      */
    int32_t sender;     /* resource index (alpha: position in the order)      */
    int32_t receiver;
    int32_t fused;      /* 1 if the receiver decodes it inside the composite   */
    ec_rect piece;      /* pixels carried, out->pvp coordinates                */
} ec_sched_message;

typedef struct ec_schedule ec_schedule;

/* Plan a schedule of n inputs into out.
 *   mode    EC_JOB_DEPTH (inputs and out EC_RGBA8 or EC_RGBA32F with depth;
 *           out->depth required) or EC_JOB_ALPHA (EC_RGBA32F / EC_RGBA16F).
 *   order   alpha: host array of n distinct indices, order[0] in front
 *           (resource i holds input order[i]); NULL means 0..n-1.  Ignored
 *           for depth.
 * The plan allocates one device arena for every intermediate partial, stream
 * and decoded piece, and captures the schedule's launches in a CUDA graph.
 * It refers to the inputs and out by address: they must stay in place until
 * ec_schedule_free.  Partial results depend only on the inputs' ROIs, which
 * are read now.  Errors: EC_ERR_INVALID_ARG (bad geometry, format, flags;
 * binary swap with n not a power of two), EC_ERR_UNSUPPORTED (RLE for alpha
 * or RGBA32F, n > EC_MAX_SOURCES, a composite of more than
 * EC_MAX_BATCH_INPUTS pieces). */
ec_status ec_schedule_plan(ec_ctx* ctx, int32_t mode, int32_t algorithm, const ec_image* in,
                           int32_t n, const int32_t* order, const ec_target* out, uint32_t flags,
                           ec_schedule** plan);
/* Host only, no device work (thesis 5.2.2, 5.2.3): the geometry of the
 * schedule ec_schedule_plan would build for n resources whose data lies in
 * rois[i], all rectangles in the same pixel coordinates as frame (rois are
 * clipped to frame).  Fills msgs (host, cap entries) with the transfers in
 * stage order (fused = 0), *n_levels with the number of stages and, when
 * regions is not NULL, regions[0..n) with the part of frame each resource owns
 * at the end (empty for the senders of a stream).  *n_messages receives the
 * count even when cap is too small (EC_ERR_CAPACITY; msgs then holds the
 * first cap).  Errors: EC_ERR_INVALID_ARG (n < 1, negative sizes, unknown
 * algorithm, binary swap with n not a power of two), EC_ERR_UNSUPPORTED
 * (n > EC_MAX_SOURCES). */
ec_status ec_schedule_geometry(int32_t algorithm, const ec_rect* rois, int32_t n, ec_rect frame,
                               ec_sched_message* msgs, int32_t cap, int32_t* n_messages,
                               int32_t* n_levels, ec_rect* regions);
/* Enqueue the captured schedule on stream s. */
ec_status ec_schedule_run(ec_schedule* plan, ec_stream_t s);
/* Stages, transfers, kernel launches per run and arena bytes (host pointers, any may be NULL). */
ec_status ec_schedule_info(const ec_schedule* plan, int32_t* n_levels, int32_t* n_messages,
                           int32_t* n_launches, uint64_t* arena_bytes);
/* The transfers, in stage order (cap entries of host memory; EC_ERR_CAPACITY if too few). */
ec_status ec_schedule_messages(const ec_schedule* plan, ec_sched_message* msgs, int32_t cap);
/* The schedule's kernel launches, in the order a run enqueues them. */
typedef enum {
    EC_SCHED_LAUNCH_COMPRESS = 0,   /* RLE compress of a stage's transfers          */
    EC_SCHED_LAUNCH_DECOMPRESS = 1, /* decode of the transfers of unfused stages    */
    EC_SCHED_LAUNCH_FUSED = 2,      /* decode-and-merge of the fused stages         */
    EC_SCHED_LAUNCH_COMPOSITE = 3   /* persistent composite of the other stages     */
} ec_sched_launch_kind;
typedef struct {
    int32_t level;
    int32_t kind;       /* ec_sched_launch_kind                                    */
    uint64_t bytes;     /* pixel bytes the launch reads and writes; the RLE
                           streams it reads or writes are not included          */
} ec_sched_launch;
ec_status ec_schedule_launches(const ec_schedule* plan, ec_sched_launch* out, int32_t cap);
/* Enqueue launch i alone on s (ec_schedule_run enqueues all of them, in
 * order, as one graph).  Launches must be enqueued in order, 0 first, each
 * after the previous one completes or on the same stream; for timing. */
ec_status ec_schedule_run_launch(ec_schedule* plan, int32_t i, ec_stream_t s);
/* Wait for s, then copy the colour and depth stream sizes of every transfer of
 * the last run (2 per message, host memory).  EC_ERR_UNSUPPORTED without RLE. */
ec_status ec_schedule_stream_sizes(ec_schedule* plan, uint64_t* sizes, int32_t cap, ec_stream_t s);
void ec_schedule_free(ec_schedule* plan);

/* ------------------------------------------ assembly of the other compound modes
 * Thesis 4.2: sort-first and tile compounds compute complete pixels per source
 * and copy them into place; pixel compounds interleave the destination's
 * pixels over a pixel kernel; subpixel compounds average the samples every
 * source computed for a pixel.  Inputs and output share one colour format
 * (RGBA8, RGBA32F or RGBA16F); depth is neither read nor written.
 *
 * ec_assemble_tiles: the roi of every input, clipped to out->pvp, is copied
 * bit for bit to the same destination pixels, inputs in ascending order (a
 * later input overwrites an earlier one where they overlap).  Output pixels
 * no roi covers are left unchanged.  n <= EC_MAX_SOURCES. */
ec_status ec_assemble_tiles(ec_ctx* ctx, const ec_image* in, int32_t n, const ec_target* out,
                            ec_stream_t s);

/* ec_assemble_pixels: the destination is interleaved over an nx x ny pixel
 * kernel (1 <= nx, ny <= 16).  Input k owns the pixels at offsets
 * (kx[k] + i*nx, ky[k] + j*ny) from out->pvp's origin (0 <= kx[k] < nx,
 * 0 <= ky[k] < ny; host arrays) and stores them densely: its pixel (i, j) is
 * element j*pitch + i of in[k].color, an image of ceil((out.w - kx)/nx) x
 * ceil((out.h - ky)/ny) pixels (in[k].pvp and roi are not used).  Later inputs
 * overwrite earlier ones; pixels no input owns are left unchanged.
 * n <= 256. */
ec_status ec_assemble_pixels(ec_ctx* ctx, const ec_image* in, const int32_t* kx, const int32_t* ky,
                             int32_t n, int32_t nx, int32_t ny, const ec_target* out, ec_stream_t s);

/* ec_average: every pixel of out->pvp becomes the average of the inputs whose
 * roi holds it, channel by channel: RGBA8 (sum + count/2) / count in
 * integers; RGBA32F and RGBA16F the FP32 sum in input order divided by the
 * count, stored in the output type.  Pixels no roi holds become 0.
 * n <= EC_MAX_SOURCES. */
ec_status ec_average(ec_ctx* ctx, const ec_image* in, int32_t n, const ec_target* out, ec_stream_t s);

/* ------------------------------------------------- automatic region of interest
 * Thesis 5.3: instead of the application supplying each frame's ROI, it can be
 * computed by analysing the frame buffer, which also detects holes.
 *
 * ec_detect_roi: for every image, the bounding box of the pixels of its roi
 * (the region searched; roi must lie inside pvp) that hold rendered data, and
 * optionally which tiles of its pvp hold any.  A pixel holds data when
 *   depth != NULL: its depth is below 1.0, the cleared depth (NaN is
 *                  background); only the depth buffer is read;
 *   otherwise:     its colour is not all zero: an RGBA8 word != 0, or one of
 *                  the four float / half channels != +-0 (colour is read).
 * in:        host array of n images (pvp, roi, pitch, format, color, depth;
 *            color may be NULL when depth is given).  Elements must be
 *            naturally aligned; 16-byte aligned buffers with pitch*bytes a
 *            multiple of 16 are read with 16-byte loads.
 * tile:      occupancy tile edge in pixels: 8, 16, 32 or 64.
 * occupancy: NULL, or a host array of n device pointers (entries may be
 *            NULL) to ceil(pvp.h/tile) rows of ceil(pvp.w/tile) bytes; tile
 *            (i, j) covers pvp pixels [j*tile, (j+1)*tile) x [i*tile, (i+1)*tile)
 *            and is written 1 if one of its searched pixels holds data, else 0.
 * d_rois:    device array of n ec_rect, written in destination coordinates;
 *            {0,0,0,0} when no searched pixel holds data.
 * Asynchronous on s; argument errors (bad rectangles, tile, alignment of
 * d_rois to 4 bytes, n > EC_MAX_SOURCES) are returned synchronously.  Uses
 * context scratch: calls on one context must not overlap on the device. */
ec_status ec_detect_roi(ec_ctx* ctx, const ec_image* in, int32_t n, int32_t tile,
                        uint8_t* const* occupancy, ec_rect* d_rois, ec_stream_t s);

/* ------------------------------------------------------------ run-length codec
 * Thesis 5.5.1 (enhanced RLE): the image is coded as four independent byte
 * streams, one per component (mode 1), optionally after regrouping the 32 bits
 * of each element by significance (mode 2, the swizzle preconditioner); the
 * image is cut into independently coded sub-images for parallelism.
 *
 * Container "ECR1" (little-endian):
 *   u32 magic 0x31524345, u16 version 1, u16 mode, u32 w, u32 h,
 *   u32 elem_bytes 4, u32 chunk 4096, u32 n_chunks, u32 n_planes 4  (32 bytes)
 *   u32 end[4 * n_chunks]: exclusive end of stream 4c+p, relative to payload
 *   payload: streams in order chunk-major, plane-minor.
 * Elements are read row-major, q = y*w + x (pitch is storage only); chunk c
 * holds q in [4096c, min(4096(c+1), w*h)); plane p of an element is its byte
 * p (mode 1) or byte p of its swizzled value (mode 2: byte k gathers bits
 * 7-2k..6-2k of components R,G,B,A, R highest).  Each stream is a sequence of
 * tokens: control c < 128 -> the next c+1 bytes are literals; c >= 128 -> the
 * next byte repeats c-127 times.  Runs of >= 3 equal bytes are coded as
 * repeats, maximal spans of shorter runs as literals, at most 128 bytes per
 * token with full tokens first.  Every (image, mode) has exactly one encoding.
 * A decoder accepts any token sequence that yields exactly the chunk's bytes,
 * but rejects a stream longer than len + ceil(len/128) bytes (the all-literal
 * coding of its chunk, the longest the encoder emits).
 *
 * Mode 0 (thesis 5.5.1's basic RLE, 64-bit tokens comparing two pixels at
 * once): each chunk is one stream (header n_planes 1, end table u32
 * end[n_chunks]) over 8-byte units, unit k holding elements 2k (low four
 * bytes) and 2k+1.  Runs of >= 2 equal units are repeat tokens (control
 * 128 + len - 1, then the unit), the other units maximal literal spans
 * (control len - 1, then the units), at most 128 units per token with full
 * tokens first; a chunk of odd length ends with its last element's 4 bytes.
 * The decoder rejects a mode-0 stream longer than 8u + ceil(u/128) (+ 4 for
 * an odd chunk) bytes, u the chunk's units.  ec_rle_max_size bounds all modes.
 */

/* Upper bound on a stream's size: 32 + 16 n_chunks + sum over streams of
 * (len + ceil(len/128)).  0 for negative sizes. */
size_t ec_rle_max_size(int32_t w, int32_t h);

/* Compress w x h uint32 elements at src (row pitch `pitch` elements), mode 0,
 * 1 or 2, into dst
 * (capacity dst_capacity >= ec_rle_max_size(w, h), else EC_ERR_CAPACITY).
 * The stream's size in bytes is written to *d_size (device uint64) when the
 * kernel finishes.  w * h <= EC_RLE_MAX_ELEMS.  Uses the context's scratch
 * memory. */
ec_status ec_rle_compress(ec_ctx* ctx, const void* src, int32_t w, int32_t h,
                          int32_t pitch, uint32_t mode, void* dst, size_t dst_capacity,
                          uint64_t* d_size, ec_stream_t s);

/* Decompress a stream of src_size bytes (src 4-byte aligned) into dst (w x h
 * elements, row pitch `pitch`).  The header must name the same w and h.  Malformed input records
 * EC_ERR_CORRUPT in the status word; the kernel never reads past src_size nor
 * writes outside the w x h elements of dst. */
ec_status ec_rle_decompress(ec_ctx* ctx, const void* src, size_t src_size, void* dst,
                            int32_t w, int32_t h, int32_t pitch, ec_stream_t s);

/* Several images in one launch (the codec's data decomposition spans them). */
typedef struct {
    const void* src;     /* compress: elements; decompress: stream             */
    void* dst;           /* compress: stream; decompress: elements             */
    size_t capacity;     /* compress: dst capacity; decompress: src size       */
    uint64_t* d_size;    /* compress: device uint64 receiving the size         */
    int32_t w, h, pitch; /* image size and row pitch in elements               */
    uint32_t mode;       /* compress: 1 or 2; ignored by decompress            */
} ec_rle_job;

ec_status ec_rle_compress_batch(ec_ctx* ctx, const ec_rle_job* jobs, int32_t njobs,
                                ec_stream_t s);
ec_status ec_rle_decompress_batch(ec_ctx* ctx, const ec_rle_job* jobs, int32_t njobs,
                                  ec_stream_t s);

/* ------------------------------------------------------ lossy YUV compressor
 * Thesis 5.5.3: a colour space conversion with chroma subsampling before the
 * RLE codec (which then codes the Y, U and V channels), inverted after it.
 * Full-range BT.601 in 8-bit fixed point, divisions rounding down:
 *   Y = (77 R + 150 G + 29 B + 128) / 256
 *   U = min(255, 128 + (-43 R - 85 G + 128 B + 128) / 256)
 *   V = min(255, 128 + (128 R - 107 G - 21 B + 128) / 256)
 * Each 2x2 block keeps its four Y and the means of its pixels' U, V and alpha,
 * rounded half up, over the pixels the image has.  Decoding gives each pixel
 * its block's U, V, alpha:
 *   R = Y + (359 (V-128) + 128) / 256,  G = Y - (88 (U-128) + 183 (V-128) + 128) / 256,
 *   B = Y + (454 (U-128) + 128) / 256,  clamped to [0, 255].
 * Packed image: 2 * ceil(h/2) rows of ceil(w/2) uint32 words (row pitch
 * dst_pitch / src_pitch words): rows [0, ceil(h/2)) luma words, byte k the Y
 * of pixel (2bx + (k & 1), 2by + (k >> 1)) or 0 where the image has none;
 * then chroma words, bytes U, V, A, 0.  Code it with mode 1.
 * RGBA8 images are w x h uint32 with row pitch `pitch`; all pointers device,
 * 4-byte aligned; asynchronous on s. */
ec_status ec_yuv_encode(ec_ctx* ctx, const void* src, int32_t w, int32_t h, int32_t pitch, void* dst,
                        int32_t dst_pitch, ec_stream_t s);
ec_status ec_yuv_decode(ec_ctx* ctx, const void* src, int32_t src_pitch, int32_t w, int32_t h, void* dst,
                        int32_t pitch, ec_stream_t s);

/* Several images in one launch. */
typedef struct {
    const void* src;       /* encode: RGBA8 image; decode: packed image             */
    void* dst;             /* encode: packed image; decode: RGBA8 image             */
    int32_t w, h;          /* frame size in pixels                                  */
    int32_t pitch;         /* row pitch of the RGBA8 image, elements                */
    int32_t packed_pitch;  /* row pitch of the packed image, words (>= ceil(w/2))   */
} ec_yuv_job;
ec_status ec_yuv_encode_batch(ec_ctx* ctx, const ec_yuv_job* jobs, int32_t njobs, ec_stream_t s);
ec_status ec_yuv_decode_batch(ec_ctx* ctx, const ec_yuv_job* jobs, int32_t njobs, ec_stream_t s);

/* ------------------------------------------------ allocation-free compressor
 * The thesis has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory.  ec_rle_compress takes its scratch
 * memory (a record per chunk, a pool for the coded chunks, counters) from an
 * ec_ctx, which allocates it with cudaMalloc.  Code that must not allocate once it runs -- a frame loop
 * that reserved all of its memory at start-up, code whose device memory is
 * owned by another framework's pool, or code that cannot absorb the implicit
 * device synchronisation cudaMalloc/cudaFree may cause -- can call this
 * variant instead: it allocates nothing and needs no context.
 *
 * Its scratch is a fixed array of EC_RLE_NOALLOC_SCRATCH_BYTES compiled into
 * libec; every GPU that loads the library holds one copy until the process
 * exits.  Images of more than EC_RLE_NOALLOC_MAX_CHUNKS chunks (4096 elements
 * each, 33,554,432 elements in all, enough for one 7680x4320 frame) are
 * refused with EC_ERR_UNSUPPORTED.  The first call on a device looks up the
 * array's device address with that device current; make that first call
 * before any stream capture.  All calls share the one array and it keeps the
 * last call's contents (each call clears what it needs with a memset on s), so
 * calls that overlap on the GPU -- on different streams or from several host
 * threads -- race; serialise them.
 *
 * Arguments are those of ec_rle_compress without the context, on the current
 * device, plus d_status: a device uint32 that the caller zeroes and that
 * receives the first device-side error (EC_ERR_TIMEOUT if a bounded wait gave
 * up), since there is no context status word.  The stream written is byte for
 * byte the one ec_rle_compress writes. */
#define EC_RLE_NOALLOC_MAX_CHUNKS 8192
#define EC_RLE_NOALLOC_SCRATCH_BYTES (16 + 532 * EC_RLE_NOALLOC_MAX_CHUNKS)
ec_status ec_rle_compress_noalloc(const void* src, int32_t w, int32_t h, int32_t pitch,
                                  uint32_t mode, void* dst, size_t dst_capacity,
                                  uint64_t* d_size, uint32_t* d_status, ec_stream_t s);

#ifdef __cplusplus
}
#endif
#endif
