/*
 * ec_oracle.h -- plain, slow, single-threaded CPU oracle for sort-last image
 * compositing and the run-length pixel codec of Eilemann, "Parallel Rendering
 * and Large Data Visualization" (arXiv 1902.08755).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.  Only
 * the test suite, the smoke check and the CPU-baseline leg of the benchmark
 * may load it; the product path never does.  It shares no header, helper,
 * table or constant with the CUDA library: every definition below is written
 * out again here from the thesis text.
 *
 * Conventions (all coordinates are destination-frame pixel coordinates):
 *   rect {x, y, w, h}: pixels x <= px < x+w, y <= py < y+h; w, h >= 0.
 *   pvp  ("pixel viewport"): the rectangle a stored image covers.  Its pixel
 *        (px, py) lives at element (py - pvp.y) * pitch + (px - pvp.x).
 *   roi  ("region of interest", thesis 5.3): the sub-rectangle of pvp that
 *        holds rendered data.  Outside it a source is background (depth mode)
 *        or fully transparent (alpha mode) and is never read.
 *
 * Return codes: ORC_OK = 0, ORC_EINVAL = 1 (bad argument), ORC_ECAP = 2
 * (capacity too small), ORC_ECORRUPT = 4 (malformed stream).
 */
#ifndef EC_ORACLE_H
#define EC_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ECAP = 2, ORC_ECORRUPT = 4 };

typedef struct { int32_t x, y, w, h; } orc_rect;

/* One partial image for depth-sorted compositing (thesis 5.2.1).  color holds color_bytes bytes per pixel (4 = RGBA8,
 * 8 = RGBA16F, 16 = RGBA32F); the merge copies them bit for bit. */
typedef struct {
    orc_rect pvp, roi;
    int32_t pitch;            /* elements per stored row, >= pvp.w          */
    const void* color;        /* [pvp.h][pitch] pixels                       */
    const float* depth;       /* [pvp.h][pitch] depth values                 */
} orc_depth_src;

/* One premultiplied RGBA layer for spatial, ordered compositing (thesis
 * 5.2.1). */
typedef struct {
    orc_rect pvp, roi;
    int32_t pitch;            /* pixels per stored row, >= pvp.w             */
    const void* color;        /* [pvp.h][pitch] RGBA, fp32 or fp16 storage   */
} orc_layer;

enum { ORC_F32 = 1, ORC_F16 = 2 };

/* Depth-test merge.  Background is depth 1.0, colour all-zero bytes, winner -1.
 * Sources are scanned in ascending index; a source replaces the current best
 * only when its depth is strictly smaller, so ties go to the lower index and
 * to the background, and NaN never wins.  out_depth and winner may be NULL.
 * out_roi (may be NULL) receives the bounding box of all roi_i clipped to
 * out_pvp, or {0,0,0,0} when that union is empty. */
int orc_composite_depth(const orc_depth_src* src, int32_t n, int32_t color_bytes,
                        orc_rect out_pvp, int32_t out_pitch, void* out_color,
                        float* out_depth, int16_t* winner, orc_rect* out_roi);

/* Ordered front-to-back "over" of premultiplied RGBA, in double precision.
 * order[k] names the layer composited k-th (order[0] is in front); NULL means
 * 0..n-1.  out is [out_pvp.h][out_pvp.w][4] doubles, t_final (may be NULL) is
 * the remaining transmittance [out_pvp.h][out_pvp.w]. */
int orc_composite_alpha(const orc_layer* layers, int32_t n, int32_t fmt,
                        const int32_t* order, orc_rect out_pvp, double* out,
                        double* t_final, orc_rect* out_roi);

/* Gradient of L = sum(g * out) with respect to every layer's premultiplied
 * colour (RGB) and alpha.  g is [out_pvp.h][out_pvp.w][4].  grad[i] is a
 * [pvp_i.h][pitch_i][4] double array; the pixels of pvp_i inside out_pvp are
 * written (zero outside roi_i), all other elements are left untouched. */
int orc_composite_alpha_backward(const orc_layer* layers, int32_t n, int32_t fmt,
                                 const int32_t* order, orc_rect out_pvp,
                                 const double* g, double* const* grad);

/* Gradient of a depth composite with RGBA32F colour: the output colour of a
 * pixel is a copy of the winner's colour, so the upstream gradient g
 * ([out_pvp.h][out_pvp.w][4] floats) flows to the winning source only:
 * grad_i[p] = (winner[p] == i) ? g[p] : 0.  grad[i] is [pvps[i].h][pitch[i]][4]
 * floats, written over pvp_i inside out_pvp; other elements are untouched. */
int orc_composite_depth_backward(const int16_t* winner, orc_rect out_pvp,
                                 const float* g, int32_t n, const orc_rect* pvps,
                                 const int32_t* pitches, float* const* grad);

/* ---- assembly of the other compound modes (thesis 4.2) -------------------
 * Tile assembly (sort-first and tile compounds): the roi of every source,
 * clipped to out_pvp, is copied bit for bit (bpp = 4, 8 or 16 bytes per pixel)
 * to the same destination pixels, sources in ascending order, so a later one
 * overwrites an earlier one where they overlap.  Output pixels no roi covers
 * are left unchanged. */
int orc_assemble_tiles(const orc_layer* src, int32_t n, int32_t bpp, orc_rect out_pvp,
                       int32_t out_pitch, void* out);

/* Pixel compound: the destination is interleaved over an nx x ny pixel
 * kernel.  Source k owns the pixels at offsets (kx[k] + i*nx, ky[k] + j*ny)
 * from the out_pvp origin, 0 <= kx[k] < nx, 0 <= ky[k] < ny, and stores them
 * densely: its element j*pitch[k] + i is destination offset (kx[k] + i*nx,
 * ky[k] + j*ny), for i < ceil((out_pvp.w - kx[k]) / nx) and
 * j < ceil((out_pvp.h - ky[k]) / ny).  Pixels are copied bit for bit, sources
 * in ascending order; destination pixels no source owns are left unchanged. */
int orc_assemble_pixels(const void* const* src, const int32_t* pitch, const int32_t* kx,
                        const int32_t* ky, int32_t n, int32_t nx, int32_t ny, int32_t bpp,
                        orc_rect out_pvp, int32_t out_pitch, void* out);

/* Subpixel compound: every output pixel is the average of the sources whose
 * roi holds it, channel by channel.  format 0 (RGBA8): per 8-bit channel the
 * integer (sum + count/2) / count, written to out as uint32 pixels; ORC_F32 /
 * ORC_F16 sources: the exact average, written to out as doubles (4 per pixel).
 * Pixels no roi holds become 0.  out is [out_pvp.h][out_pitch] pixels. */
int orc_average(const orc_layer* src, int32_t n, int32_t format, orc_rect out_pvp,
                int32_t out_pitch, void* out);

/* ---- automatic region of interest (thesis 5.3) ---------------------------
 * The ROI found by scanning a frame buffer instead of being supplied by the
 * application: the bounding box of the pixels that hold rendered data, plus a
 * grid of tiles telling which tiles hold any (holes are the empty tiles).
 * A pixel holds data when
 *   depth != NULL:          its depth is below 1.0, the cleared background
 *                           depth (a NaN depth is background);
 *   else colour format 0 (RGBA8):    its 32-bit word is not 0;
 *        format 1 (RGBA32F):         one of its four floats is not 0 (-0 is 0);
 *        format 2 (RGBA16F, bits):   one of its four halves is not +-0.
 * Only pixels of search (clipped to pvp) are examined.  *roi receives the
 * bounding box in destination coordinates, {0,0,0,0} when no pixel holds
 * data.  occ, when not NULL, receives ceil(pvp.h/tile) rows of
 * ceil(pvp.w/tile) bytes: tile (i, j) covers pvp pixels [j*tile, (j+1)*tile)
 * x [i*tile, (i+1)*tile) and is 1 iff one of its examined pixels holds data. */
int orc_detect_roi(orc_rect pvp, orc_rect search, int32_t pitch, int32_t format,
                   const void* color, const float* depth, int32_t tile, uint8_t* occ,
                   orc_rect* roi);

/* ---- run-length codec (thesis 5.5.1), container "ECR1" ------------------
 * The image is w*h four-byte elements read row-major (pitch ignored in the
 * logical order).  Mode 1 splits each element into its four bytes (one stream
 * per component); mode 2 first regroups the 32 bits by significance (the
 * swizzle preconditioner).  The element sequence is cut into chunks of 4096
 * elements, each chunk's four byte streams are run-length coded on their
 * own, and the streams are stored chunk-major with an offset table.  Mode 0
 * (basic RLE) codes each chunk as one stream of 8-byte units (element pairs),
 * an odd chunk's last element as 4 raw bytes at its end; its header says one
 * plane and its table has one entry per chunk. */
size_t  orc_rle_max_size(int32_t w, int32_t h);
uint32_t orc_swizzle(uint32_t v);
uint32_t orc_unswizzle(uint32_t v);
/* Returns the stream size in bytes, or -(error code). */
int64_t orc_rle_compress(const uint32_t* src, int32_t w, int32_t h, int32_t pitch,
                         uint32_t mode, uint8_t* dst, size_t capacity);
int     orc_rle_decompress(const uint8_t* src, size_t size, uint32_t* dst,
                           int32_t w, int32_t h, int32_t pitch);

/* ---- lossy YUV compressor (thesis 5.5.3) --------------------------------
 * Full-range BT.601 in 8-bit fixed point, chroma and alpha averaged over 2x2
 * blocks.  Packed image: ceil(w/2) words per row, ceil(h/2) rows of luma words
 * then ceil(h/2) rows of chroma words (U, V, A, 0). */
int     orc_yuv_encode(const uint32_t* src, int32_t w, int32_t h, int32_t pitch, uint32_t* dst);
int     orc_yuv_decode(const uint32_t* src, int32_t w, int32_t h, uint32_t* dst, int32_t pitch);

#ifdef __cplusplus
}
#endif
#endif
