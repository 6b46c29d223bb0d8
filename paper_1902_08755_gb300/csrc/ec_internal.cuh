// ec_internal.cuh -- internal definitions shared by libec's translation units.
//
// Host-side argument validation turns every input into flat descriptors whose
// coordinates are relative to the destination's pvp origin; the kernels never
// see ec_image directly.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ec.h"

// Makes a device current for the duration of a call, then restores the
// caller's device.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

struct ec_ctx {
    int device = 0;
    uint32_t* d_status = nullptr;   // first device-side error (0 = none)
    void* scratch = nullptr;        // codec scratch: counters, chunk records, pool
    size_t scratch_bytes = 0;
    void* roi_scratch = nullptr;    // ROI detection: per-image box accumulators + done counter
    size_t roi_scratch_bytes = 0;
    int sm_count = 0;
};

namespace ec {

// Per-source descriptor (48 bytes).  Coordinates are relative to the output
// viewport origin; [x0,x1) x [y0,y1) is roi ∩ out.pvp, (ox, oy) the stored
// pvp origin, so pixel (x, y) is element (y - oy) * pitch + (x - ox).
struct SrcDesc {
    int32_t x0, y0, x1, y1;
    int32_t ox, oy;
    int32_t pitch;
    int32_t vec;           // 1 if this source may be read with 16-byte accesses
    const void* color;
    const float* depth;
};
static_assert(sizeof(SrcDesc) == 48, "descriptor layout");

// Source lists travel as kernel parameters (no staging copy, capturable in a
// CUDA graph).  Three capacities keep small calls' parameter blocks small.
template <int N>
struct SrcList {
    int32_t n;
    int32_t pad[3];
    SrcDesc s[N];
};
static_assert(sizeof(SrcList<512>) < 32764 - 256, "kernel parameter limit");

// Destination descriptor.
struct DstDesc {
    int32_t W, H;          // out.pvp size
    int32_t pitch;         // pixels
    int32_t vec;           // 16-byte stores allowed
    void* color;
    float* depth;          // may be null
    int16_t* winner;       // may be null, dense [H][W]
    float* tfinal;         // may be null, dense [H][W]
};

// Device status word: the first error wins.
__device__ __forceinline__ void set_status(uint32_t* st, uint32_t code)
{
    atomicCAS(st, 0u, code);
}

// Streaming (evict-first) 16-byte global loads and stores: every input pixel
// is read once per launch.
__device__ __forceinline__ uint4 ld_stream(const uint4* p) { return __ldcs(p); }
__device__ __forceinline__ float4 ld_stream(const float4* p) { return __ldcs(p); }
__device__ __forceinline__ void st_stream(uint4* p, uint4 v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(float4* p, float4 v) { __stcs(p, v); }

inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Per-layer descriptor of the backward passes (64 bytes), in compositing
// order.  [x0,x1) x [y0,y1) is roi ∩ out.pvp, [gx0,gx1) x [gy0,gy1) is
// pvp ∩ out.pvp (where gradients are written), both relative to out.pvp.
constexpr int kMaxBwdLayers = 256;
struct BwdDesc {
    int32_t x0, y0, x1, y1;
    int32_t gx0, gy0, gx1, gy1;
    int32_t ox, oy;
    int32_t pitch;
    int16_t cls;           // alignment of the colour data in bytes (16, 8, 4 or 2)
    int16_t gvec;          // gradient stores may be one vector per pixel
    const void* color;
    void* grad;
};
static_assert(sizeof(BwdDesc) == 64, "backward descriptor layout");

template <int N>
struct BwdList {
    int32_t n;
    int32_t pad[3];
    BwdDesc d[N];
};
static_assert(sizeof(BwdList<kMaxBwdLayers>) < 32764 - 256, "kernel parameter limit");

// ---- batched compositing ----------------------------------------------------
// One job = one full composite; mode 0 depth RGBA8, 1 depth RGBA32F, 2 alpha
// RGBA32F, 3 alpha RGBA16F.  Its n inputs are srcs[first, first + n), in
// compositing order.  A work item is one output tile (tx, ty) of one job.
struct BatchJob {
    int32_t mode;
    int32_t n;
    int32_t first;
    int32_t pad;
    DstDesc D;
};
static_assert(sizeof(BatchJob) == 64, "batch job layout");

struct BatchItem {
    int32_t job;
    int16_t tx, ty;
};

struct BatchShape {
    int32_t tw[4], th[4];   // tile width / height in pixels, per mode
};

int batch_warp_px(int mode);
int batch_ctas_per_sm();
cudaError_t launch_batch(const BatchJob* jobs, const SrcDesc* srcs, const BatchItem* items,
                         int n_items, uint32_t* head, const BatchShape& shape, int grid,
                         cudaStream_t s);

// ---- launchers (defined in the kernel translation units) -------------------

cudaError_t launch_alpha_bwd(const BwdDesc* d, int n, bool f16, bool g16, bool fused,
                             const DstDesc& dst, const float* g, cudaStream_t s);
cudaError_t launch_depth_bwd(const BwdDesc* d, int n, int W, int H, const int16_t* winner,
                             const float* g, cudaStream_t s);
cudaError_t launch_depth(const SrcDesc* src, int n, int color_bytes, const DstDesc& dst,
                         cudaStream_t s);
cudaError_t launch_alpha_fwd(const SrcDesc* src, int n, bool f16, const DstDesc& dst,
                             cudaStream_t s);

struct RleJobDesc {
    const uint32_t* src;   // compress: elements; decompress: stream bytes (as u8)
    void* dst;
    uint64_t* d_size;
    uint64_t capacity;     // decompress: source size in bytes
    int32_t w, h, pitch;
    uint32_t mode;
    uint32_t n_chunks;     // ceil(w*h / 4096)
    uint32_t first_unit;   // first global work unit of this job
    uint32_t vec;          // 16-byte element loads/stores allowed
    uint32_t pad;
};
static_assert(sizeof(RleJobDesc) == 64, "rle job layout");

// At most kRleJobsPerLaunch jobs travel in one launch's parameters; larger
// batches are split into several launches.
constexpr int kRleJobsPerLaunch = 256;

template <int N>
struct RleJobList {
    int32_t n;
    uint32_t total_units;
    int32_t pad[2];
    RleJobDesc j[N];
};
static_assert(sizeof(RleJobList<kRleJobsPerLaunch>) < 32764 - 256, "kernel parameter limit");

// Scratch of a compress launch of `units` work units: a ticket, a counter and a
// pool cursor, a 16-byte record and a 4-byte list entry per unit (modes 1, 2;
// mode 0 uses 8 bytes per unit of them), then a pool for the coded chunks,
// pool_per_unit bytes per unit.  A
// chunk that finds the pool full is coded a second time when placed, so any
// pool size gives the same stream.
size_t rle_compress_scratch_bytes(uint32_t units, size_t pool_per_unit);
constexpr size_t kRlePoolPerUnit = 512;

cudaError_t launch_rle_compress(const RleJobDesc* jobs, int n, uint32_t total_units,
                                void* scratch, size_t scratch_bytes, uint32_t* status, cudaStream_t s);
cudaError_t launch_rle_decompress(const RleJobDesc* jobs, int n, uint32_t total_units,
                                  uint32_t* status, cudaStream_t s);

// ---- assembly of the other compound modes ------------------------------------

cudaError_t launch_assemble_tiles(const SrcDesc* src, int n, int bpp, const DstDesc& D, cudaStream_t s);
// fmt: 0 RGBA8, 1 RGBA32F, 2 RGBA16F
cudaError_t launch_average(const SrcDesc* src, int n, int fmt, const DstDesc& D, cudaStream_t s);

// Pixel compound source: densely stored interleaved pixels.
struct PixSrc {
    const void* color;
    int32_t pitch;
    int32_t pad;
};
static_assert(sizeof(PixSrc) == 16, "pixel source layout");
constexpr int kPixMaxSources = 256, kPixMaxKernel = 16;   // kernel edge <= 16 pixels

template <int N>
struct PixList {
    int32_t n, nx, ny, pad;
    PixSrc s[N];
    int16_t owner[kPixMaxKernel * kPixMaxKernel];   // source owning offset (x % nx, y % ny), or -1
};

cudaError_t launch_assemble_pixels(const PixSrc* src, const int16_t* owner, int n, int nx, int ny, int bpp,
                                   const DstDesc& D, cudaStream_t s);

// ---- automatic region of interest -------------------------------------------

// One image of an ROI detection launch (64 bytes).  The image is scanned in
// kRoiBlkW x kRoiBlkH blocks aligned to its pvp origin; [x0,x1) x [y0,y1) are
// the searched pixels relative to that origin.
struct RoiDesc {
    int32_t x0, y0, x1, y1;
    int32_t ox, oy;            // pvp origin in destination coordinates
    int32_t pitch;
    int32_t gw, gh;            // occupancy grid (tiles)
    int32_t bw;                // blocks along x
    uint32_t first_block;      // first CTA of this image (within its kind's launch)
    int16_t idx;               // image index within the call (accumulators, output)
    int16_t vec;               // 16-byte loads allowed
    const void* data;          // depth or colour, pvp pixel (0, 0)
    uint8_t* occ;              // occupancy grid or null
};
static_assert(sizeof(RoiDesc) == 64, "roi descriptor layout");

constexpr int kRoiPerLaunch = 256;
constexpr int kRoiBlkW = 64, kRoiBlkH = 128;    // pixels one CTA scans

template <int N>
struct RoiList {
    int32_t n;
    uint32_t blocks;           // CTAs with work (the launch may have one more)
    int32_t tile;
    int32_t pad;
    RoiDesc d[N];
};

// Images of one call: kinds[i] is 0 depth, 1 RGBA8, 2 RGBA32F, 3 RGBA16F;
// nblocks[i] the image's blocks.  scratch holds 4 box accumulators per image,
// 16-byte aligned; they must be zero on entry and are zero again on exit.
cudaError_t launch_detect_roi(RoiDesc* d, const int* kinds, const uint32_t* nblocks, int n, int tile,
                              uint32_t* scratch, ec_rect* out, cudaStream_t s);

// ---- fused decode-and-composite (stages of multi-stage schedules) ---------
// One receiver's binary depth merge: a plain local input and RLE-coded pieces
// of one other unit, all in frame coordinates.  Buffers are [rows][pitch]
// uint32 colour + float depth; element [0][0] sits at frame (ox, oy) / (lx, ly).
struct FusedStage {
    uint32_t* oc;
    float* od;
    const uint32_t* lc;
    const float* ld;
    int32_t opitch, ox, oy;
    int32_t lpitch, lx, ly;
    int32_t r0x, r0y, r1x, r1y;   // local ROI [r0, r1); empty if r0x >= r1x
    int32_t front;                // 1: the pieces are in front of the local input
    int32_t ovec, lvec;           // 16-byte aligned bases and pitches (multiples of 4)
    int32_t pad;
};
static_assert(sizeof(FusedStage) == 88, "fused stage layout");

// A work unit.  With streams (cs, ds non-null) it is chunk `chunk` (4096
// elements, row-major) of a coded piece, which it decodes and merges; without,
// it is rows [chunk, chunk + nrows) of a part of the output no piece covers,
// where it writes the local input (or the background).
struct FusedUnit {
    const uint8_t* cs;
    const uint8_t* ds;
    const uint64_t* csize;        // stream sizes written by the compressor
    const uint64_t* dsize;
    int32_t stage;
    int32_t x, y, w, h;
    uint32_t chunk;
    int32_t nrows;
    uint32_t cap;                 // bytes allocated to each stream (>= its size)
};
static_assert(sizeof(FusedUnit) == 64, "fused unit layout");

}  // namespace ec

// Validate a codec job and turn it into a descriptor (first_unit left 0).
ec_status rle_job_desc(const ec_rle_job& j, bool compress, ec::RleJobDesc* d);

namespace ec {

// A bounded mbarrier wait (the compressor's) on a barrier that nothing
// arrives on; it gives up and records EC_ERR_TIMEOUT.
cudaError_t launch_selftest_wait(uint32_t* status, cudaStream_t s);

cudaError_t launch_fused_depth(const FusedStage* stages, const FusedUnit* units, int n_units,
                               uint32_t* status, cudaStream_t s);

// One image of a YUV launch: encode reads src (RGBA8, row pitch `pitch`) and
// writes the packed dst (row pitch dpitch); decode reads the packed src (row
// pitch dpitch) and writes RGBA8 dst (row pitch `pitch`).
struct YuvJob {
    const uint32_t* src;
    uint32_t* dst;
    int32_t w, h, pitch, dpitch;
    uint32_t first;      // first CTA tile of this image
    uint32_t tiles_x;    // CTA tiles per row of blocks
    int32_t vec;         // bits: RGBA8 side 8-byte (1) / 16-byte (2) accesses, packed side 8-byte (4)
    int32_t pad;
};
static_assert(sizeof(YuvJob) == 48, "yuv job layout");

constexpr int kYuvJobsPerLaunch = 128;

template <int N>
struct YuvJobList {
    int32_t n;
    int32_t pad[3];
    YuvJob j[N];
};

// jobs: at most kYuvJobsPerLaunch; first/tiles_x are filled in here.
cudaError_t launch_yuv(YuvJob* jobs, int n, bool encode, cudaStream_t s);

// Enqueue a batch plan's persistent launch directly (no graph), for callers
// that capture their own graph.
cudaError_t batch_enqueue(const ec_batch* b, cudaStream_t s);

}  // namespace ec
