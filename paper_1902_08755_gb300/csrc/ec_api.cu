// ec_api.cu -- the C ABI of libec (see include/ec.h): contexts, argument
// validation and descriptor building on the host, then kernel launches.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ec_internal.cuh"

using namespace ec;

namespace {

// Makes ctx->device current for the duration of a call, then restores the
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

bool rect_ok(const ec_rect& r)
{
    return r.w >= 0 && r.h >= 0 && (int64_t)r.x + r.w <= INT32_MAX && (int64_t)r.y + r.h <= INT32_MAX;
}

bool rect_empty(const ec_rect& r) { return r.w <= 0 || r.h <= 0; }

bool rect_inside(const ec_rect& in, const ec_rect& out)
{
    if (rect_empty(in)) return true;
    return in.x >= out.x && in.y >= out.y && (int64_t)in.x + in.w <= (int64_t)out.x + out.w &&
           (int64_t)in.y + in.h <= (int64_t)out.y + out.h;
}

ec_rect intersect(const ec_rect& a, const ec_rect& b)
{
    const int64_t x0 = std::max(a.x, b.x), y0 = std::max(a.y, b.y);
    const int64_t x1 = std::min((int64_t)a.x + a.w, (int64_t)b.x + b.w);
    const int64_t y1 = std::min((int64_t)a.y + a.h, (int64_t)b.y + b.h);
    if (x1 <= x0 || y1 <= y0) return ec_rect{0, 0, 0, 0};
    return ec_rect{(int32_t)x0, (int32_t)y0, (int32_t)(x1 - x0), (int32_t)(y1 - y0)};
}

// Bounding box of the union of the clipped ROIs (thesis 5.3, merged ROI).
ec_rect merged_roi(const ec_image* in, int n, const ec_rect& pvp)
{
    bool have = false;
    int64_t x0 = 0, y0 = 0, x1 = 0, y1 = 0;
    for (int i = 0; i < n; ++i) {
        const ec_rect c = intersect(in[i].roi, pvp);
        if (rect_empty(c)) continue;
        if (!have) { x0 = c.x; y0 = c.y; x1 = (int64_t)c.x + c.w; y1 = (int64_t)c.y + c.h; have = true; }
        else {
            x0 = std::min<int64_t>(x0, c.x); y0 = std::min<int64_t>(y0, c.y);
            x1 = std::max<int64_t>(x1, (int64_t)c.x + c.w); y1 = std::max<int64_t>(y1, (int64_t)c.y + c.h);
        }
    }
    if (!have) return ec_rect{0, 0, 0, 0};
    return ec_rect{(int32_t)x0, (int32_t)y0, (int32_t)(x1 - x0), (int32_t)(y1 - y0)};
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int mod_pos(int64_t a, int m) { return (int)(((a % m) + m) % m); }

int bytes_per_px(int fmt)
{
    switch (fmt) {
    case EC_RGBA8: return 4;
    case EC_RGBA32F: return 16;
    case EC_RGBA16F: return 8;
    default: return 0;
    }
}

// Validate one input image and build its descriptor relative to out_pvp.
// group = pixels per 16-byte vector access of this path.
ec_status make_desc(const ec_image& im, const ec_rect& out_pvp, int group, bool need_depth,
                    SrcDesc* d)
{
    if (!rect_ok(im.pvp) || !rect_ok(im.roi) || im.pitch < im.pvp.w || im.pitch < 0)
        return EC_ERR_INVALID_ARG;
    if (!rect_inside(im.roi, im.pvp)) return EC_ERR_INVALID_ARG;
    const ec_rect c = intersect(im.roi, out_pvp);
    memset(d, 0, sizeof(*d));
    if (!rect_empty(c)) {
        if (!im.color || (need_depth && !im.depth)) return EC_ERR_INVALID_ARG;
        d->x0 = c.x - out_pvp.x;
        d->y0 = c.y - out_pvp.y;
        d->x1 = d->x0 + c.w;
        d->y1 = d->y0 + c.h;
    }
    const int64_t ox = (int64_t)im.pvp.x - out_pvp.x, oy = (int64_t)im.pvp.y - out_pvp.y;
    if (ox < INT32_MIN || ox > INT32_MAX || oy < INT32_MIN || oy > INT32_MAX) return EC_ERR_INVALID_ARG;
    d->ox = (int32_t)ox;
    d->oy = (int32_t)oy;
    d->pitch = im.pitch;
    d->color = im.color;
    d->depth = im.depth;
    d->vec = aligned16(im.color) && (!need_depth || aligned16(im.depth)) && im.pitch % group == 0 &&
             mod_pos(ox, group) == 0;
    return EC_OK;
}

ec_status check_target(const ec_target* out, int fmt_a, int fmt_b)
{
    if (!out || !rect_ok(out->pvp) || out->pitch < out->pvp.w) return EC_ERR_INVALID_ARG;
    if (out->format != fmt_a && out->format != fmt_b) return EC_ERR_INVALID_ARG;
    if (!rect_empty(out->pvp) && !out->color) return EC_ERR_INVALID_ARG;
    return EC_OK;
}

ec_status cuda_status(cudaError_t e) { return e == cudaSuccess ? EC_OK : EC_ERR_CUDA; }

uint32_t rle_units(uint64_t n) { return (uint32_t)std::max<uint64_t>(1, (n + EC_RLE_CHUNK - 1) / EC_RLE_CHUNK); }

ec_status ensure_scratch(ec_ctx* ctx, size_t bytes)
{
    if (ctx->scratch_bytes >= bytes) return EC_OK;
    // growing synchronises with the device (cudaFree); contexts start with
    // room for 65536 chunks (256 Mi elements), so this is rare
    if (ctx->scratch) cudaFree(ctx->scratch);
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
    if (cudaMalloc(&ctx->scratch, bytes) != cudaSuccess) return EC_ERR_CUDA;
    ctx->scratch_bytes = bytes;
    return EC_OK;
}

}  // namespace

extern "C" {

const char* ec_status_string(ec_status st)
{
    switch (st) {
    case EC_OK: return "EC_OK";
    case EC_ERR_INVALID_ARG: return "EC_ERR_INVALID_ARG";
    case EC_ERR_CAPACITY: return "EC_ERR_CAPACITY";
    case EC_ERR_CUDA: return "EC_ERR_CUDA";
    case EC_ERR_CORRUPT: return "EC_ERR_CORRUPT";
    case EC_ERR_UNSUPPORTED: return "EC_ERR_UNSUPPORTED";
    case EC_ERR_TIMEOUT: return "EC_ERR_TIMEOUT";
    }
    return "EC_ERR_UNKNOWN";
}

ec_status ec_create(ec_ctx** out, int device)
{
    if (!out) return EC_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return EC_ERR_INVALID_ARG;
    DeviceGuard g(device);
    if (!g.ok) return EC_ERR_CUDA;
    ec_ctx* ctx = new ec_ctx;
    ctx->device = device;
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc(&ctx->d_status, sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(ctx->d_status, 0, sizeof(uint32_t)) != cudaSuccess ||
        ensure_scratch(ctx, 16 + 8 * 65536) != EC_OK) {
        ec_destroy(ctx);
        return EC_ERR_CUDA;
    }
    *out = ctx;
    return EC_OK;
}

void ec_destroy(ec_ctx* ctx)
{
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->scratch) cudaFree(ctx->scratch);
    delete ctx;
}

ec_status ec_status_sync(ec_ctx* ctx, ec_stream_t s)
{
    if (!ctx) return EC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (cudaStreamSynchronize((cudaStream_t)s) != cudaSuccess) return EC_ERR_CUDA;
    uint32_t v = 0;
    if (cudaMemcpy(&v, ctx->d_status, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return EC_ERR_CUDA;
    if (v && cudaMemset(ctx->d_status, 0, sizeof(uint32_t)) != cudaSuccess) return EC_ERR_CUDA;
    return (ec_status)v;
}

ec_status ec_composite_depth(ec_ctx* ctx, const ec_image* in, int32_t n, const ec_target* out,
                             int16_t* winner, ec_rect* out_roi, ec_stream_t s)
{
    if (!ctx || n < 0 || (n > 0 && !in)) return EC_ERR_INVALID_ARG;
    if (n > EC_MAX_SOURCES) return EC_ERR_UNSUPPORTED;
    ec_status st = check_target(out, EC_RGBA8, EC_RGBA32F);
    if (st != EC_OK) return st;
    std::vector<SrcDesc> d((size_t)std::max(n, 1));
    for (int i = 0; i < n; ++i) {
        if (in[i].format != out->format) return EC_ERR_INVALID_ARG;
        if ((st = make_desc(in[i], out->pvp, 4, true, &d[i])) != EC_OK) return st;
    }
    DstDesc D;
    D.W = out->pvp.w;
    D.H = out->pvp.h;
    D.pitch = out->pitch;
    D.color = out->color;
    D.depth = out->depth;
    D.winner = winner;
    D.tfinal = nullptr;
    D.vec = aligned16(out->color) && (!out->depth || aligned16(out->depth)) && out->pitch % 4 == 0;
    if (out_roi) *out_roi = merged_roi(in, n, out->pvp);
    DeviceGuard g(ctx->device);
    if (!g.ok) return EC_ERR_CUDA;
    return cuda_status(launch_depth(d.data(), n, bytes_per_px(out->format), D, (cudaStream_t)s));
}

static ec_status alpha_descs(const ec_image* in, const int32_t* order, int32_t n, int fmt,
                             const ec_rect& pvp, std::vector<SrcDesc>& d)
{
    if (n < 0 || (n > 0 && !in)) return EC_ERR_INVALID_ARG;
    if (n > EC_MAX_SOURCES) return EC_ERR_UNSUPPORTED;
    if (fmt != EC_RGBA32F && fmt != EC_RGBA16F) return EC_ERR_INVALID_ARG;
    d.assign((size_t)std::max(n, 1), SrcDesc{});
    std::vector<char> seen((size_t)std::max(n, 1), 0);
    const int group = fmt == EC_RGBA16F ? 2 : 1;
    for (int k = 0; k < n; ++k) {
        const int i = order ? order[k] : k;
        if (i < 0 || i >= n || seen[i]) return EC_ERR_INVALID_ARG;
        seen[i] = 1;
        if (in[i].format != fmt) return EC_ERR_INVALID_ARG;
        const ec_status st = make_desc(in[i], pvp, group, false, &d[k]);
        if (st != EC_OK) return st;
    }
    return EC_OK;
}

ec_status ec_composite_alpha(ec_ctx* ctx, const ec_image* in, const int32_t* order, int32_t n,
                             const ec_target* out, float* t_final, ec_rect* out_roi, ec_stream_t s)
{
    if (!ctx) return EC_ERR_INVALID_ARG;
    ec_status st = check_target(out, EC_RGBA32F, EC_RGBA16F);
    if (st != EC_OK) return st;
    std::vector<SrcDesc> d;
    if ((st = alpha_descs(in, order, n, out->format, out->pvp, d)) != EC_OK) return st;
    const bool f16 = out->format == EC_RGBA16F;
    DstDesc D;
    D.W = out->pvp.w;
    D.H = out->pvp.h;
    D.pitch = out->pitch;
    D.color = out->color;
    D.depth = nullptr;
    D.winner = nullptr;
    D.tfinal = t_final;
    D.vec = aligned16(out->color) && (!f16 || out->pitch % 2 == 0);
    if (out_roi) *out_roi = merged_roi(in, n, out->pvp);
    DeviceGuard g(ctx->device);
    if (!g.ok) return EC_ERR_CUDA;
    return cuda_status(launch_alpha_fwd(d.data(), n, f16, D, (cudaStream_t)s));
}

size_t ec_rle_max_size(int32_t w, int32_t h)
{
    if (w < 0 || h < 0) return 0;
    const uint64_t n = (uint64_t)w * (uint64_t)h;
    const uint64_t full = n / EC_RLE_CHUNK, rem = n % EC_RLE_CHUNK;
    const uint64_t nc = full + (rem ? 1 : 0);
    uint64_t size = 32 + 16 * nc + full * 4 * (EC_RLE_CHUNK + EC_RLE_CHUNK / 128);
    if (rem) size += 4 * (rem + (rem + 127) / 128);
    return (size_t)size;
}

static ec_status rle_job_desc(const ec_rle_job& j, bool compress, RleJobDesc* d)
{
    if (j.w < 0 || j.h < 0 || j.pitch < j.w) return EC_ERR_INVALID_ARG;
    const uint64_t n = (uint64_t)j.w * (uint64_t)j.h;
    if (n > EC_RLE_MAX_ELEMS) return EC_ERR_UNSUPPORTED;
    if ((compress && !j.dst) || (n > 0 && (!j.src || !j.dst))) return EC_ERR_INVALID_ARG;
    memset(d, 0, sizeof(*d));
    d->src = reinterpret_cast<const uint32_t*>(j.src);
    d->dst = j.dst;
    d->w = j.w;
    d->h = j.h;
    d->pitch = j.pitch;
    d->n_chunks = (uint32_t)((n + EC_RLE_CHUNK - 1) / EC_RLE_CHUNK);
    if (compress) {
        if (j.mode != 1 && j.mode != 2) return EC_ERR_INVALID_ARG;
        if (!j.d_size || (reinterpret_cast<uintptr_t>(j.d_size) & 7u)) return EC_ERR_INVALID_ARG;
        if (j.capacity < ec_rle_max_size(j.w, j.h)) return EC_ERR_CAPACITY;
        if (n > 0 && (reinterpret_cast<uintptr_t>(j.src) & 3u)) return EC_ERR_INVALID_ARG;
        d->mode = j.mode;
        d->d_size = j.d_size;
        d->vec = aligned16(j.src) && j.w % 4 == 0 && j.pitch % 4 == 0;
    } else {
        if (!j.src) return EC_ERR_INVALID_ARG;
        if (n > 0 && (reinterpret_cast<uintptr_t>(j.dst) & 3u)) return EC_ERR_INVALID_ARG;
        d->capacity = j.capacity;
        d->vec = aligned16(j.dst) && j.w % 4 == 0 && j.pitch % 4 == 0;
    }
    return EC_OK;
}

static ec_status rle_batch(ec_ctx* ctx, const ec_rle_job* jobs, int32_t njobs, bool compress,
                           ec_stream_t s)
{
    if (!ctx || njobs < 0 || (njobs > 0 && !jobs)) return EC_ERR_INVALID_ARG;
    if (njobs > EC_RLE_MAX_JOBS) return EC_ERR_UNSUPPORTED;
    std::vector<RleJobDesc> d((size_t)std::max(njobs, 1));
    for (int i = 0; i < njobs; ++i) {
        const ec_status st = rle_job_desc(jobs[i], compress, &d[i]);
        if (st != EC_OK) return st;
    }
    DeviceGuard g(ctx->device);
    if (!g.ok) return EC_ERR_CUDA;
    for (int b = 0; b < njobs; b += kRleJobsPerLaunch) {
        const int cnt = std::min(kRleJobsPerLaunch, njobs - b);
        uint32_t units = 0;
        for (int i = 0; i < cnt; ++i) {
            d[b + i].first_unit = units;
            units += rle_units((uint64_t)d[b + i].w * (uint64_t)d[b + i].h);
        }
        cudaError_t e;
        if (compress) {
            const ec_status st = ensure_scratch(ctx, 16 + 8ull * units);
            if (st != EC_OK) return st;
            e = launch_rle_compress(&d[b], cnt, units, ctx->scratch, ctx->d_status, (cudaStream_t)s);
        } else {
            e = launch_rle_decompress(&d[b], cnt, units, ctx->d_status, (cudaStream_t)s);
        }
        if (e != cudaSuccess) return EC_ERR_CUDA;
    }
    return EC_OK;
}

ec_status ec_rle_compress_batch(ec_ctx* ctx, const ec_rle_job* jobs, int32_t njobs, ec_stream_t s)
{
    return rle_batch(ctx, jobs, njobs, true, s);
}

ec_status ec_rle_decompress_batch(ec_ctx* ctx, const ec_rle_job* jobs, int32_t njobs, ec_stream_t s)
{
    return rle_batch(ctx, jobs, njobs, false, s);
}

ec_status ec_rle_compress(ec_ctx* ctx, const void* src, int32_t w, int32_t h, int32_t pitch,
                          uint32_t mode, void* dst, size_t dst_capacity, uint64_t* d_size,
                          ec_stream_t s)
{
    ec_rle_job j;
    j.src = src;
    j.dst = dst;
    j.capacity = dst_capacity;
    j.d_size = d_size;
    j.w = w;
    j.h = h;
    j.pitch = pitch;
    j.mode = mode;
    return rle_batch(ctx, &j, 1, true, s);
}

ec_status ec_rle_decompress(ec_ctx* ctx, const void* src, size_t src_size, void* dst, int32_t w,
                            int32_t h, int32_t pitch, ec_stream_t s)
{
    ec_rle_job j;
    j.src = src;
    j.dst = dst;
    j.capacity = src_size;
    j.d_size = nullptr;
    j.w = w;
    j.h = h;
    j.pitch = pitch;
    j.mode = 0;
    return rle_batch(ctx, &j, 1, false, s);
}

}  // extern "C"

static_assert(sizeof(ec_image) == 56 && sizeof(ec_target) == 40 && sizeof(ec_rle_job) == 48,
              "ABI struct layouts are mirrored by the Python binding");

// ------------------------------------------------------------- backward ----

namespace {

bool aligned(const void* p, int a) { return (reinterpret_cast<uintptr_t>(p) % (uintptr_t)a) == 0; }

int align_class(const void* p, int px_bytes)
{
    for (int a = px_bytes; a >= 2; a >>= 1)
        if (aligned(p, a)) return a;
    return 1;
}

// Descriptor of one layer for a backward pass (roi/pvp clipped to out_pvp).
ec_status make_bwd_desc(const ec_rect& pvp, const ec_rect& roi, int32_t pitch, const void* color,
                        void* grad, int px_bytes, int grad_px_bytes, const ec_rect& out_pvp,
                        BwdDesc* d)
{
    if (!rect_ok(pvp) || !rect_ok(roi) || pitch < pvp.w || !rect_inside(roi, pvp)) return EC_ERR_INVALID_ARG;
    memset(d, 0, sizeof(*d));
    const ec_rect c = intersect(roi, out_pvp), g = intersect(pvp, out_pvp);
    if (!rect_empty(c)) {
        if (!color) return EC_ERR_INVALID_ARG;
        d->x0 = c.x - out_pvp.x; d->y0 = c.y - out_pvp.y; d->x1 = d->x0 + c.w; d->y1 = d->y0 + c.h;
    }
    if (!rect_empty(g)) {
        if (!grad || !aligned(grad, 2)) return EC_ERR_INVALID_ARG;
        d->gx0 = g.x - out_pvp.x; d->gy0 = g.y - out_pvp.y; d->gx1 = d->gx0 + g.w; d->gy1 = d->gy0 + g.h;
    }
    const int64_t ox = (int64_t)pvp.x - out_pvp.x, oy = (int64_t)pvp.y - out_pvp.y;
    if (ox < INT32_MIN || ox > INT32_MAX || oy < INT32_MIN || oy > INT32_MAX) return EC_ERR_INVALID_ARG;
    d->ox = (int32_t)ox;
    d->oy = (int32_t)oy;
    d->pitch = pitch;
    d->cls = (int16_t)(color ? align_class(color, px_bytes) : px_bytes);
    if (color && d->cls < 2) return EC_ERR_INVALID_ARG;
    d->gvec = (int16_t)(grad ? aligned(grad, grad_px_bytes) : 0);
    d->color = color;
    d->grad = grad;
    return EC_OK;
}

ec_status alpha_bwd_common(ec_ctx* ctx, const ec_image* in, const int32_t* order, int32_t n,
                           const ec_rect& out_pvp, const float* g, void* const* grad,
                           int32_t grad_format, std::vector<BwdDesc>& d, bool* f16, bool* g16)
{
    if (!ctx || n < 0 || (n > 0 && (!in || !grad))) return EC_ERR_INVALID_ARG;
    if (n > kMaxBwdLayers) return EC_ERR_UNSUPPORTED;
    if (!rect_ok(out_pvp)) return EC_ERR_INVALID_ARG;
    if (!rect_empty(out_pvp) && (!g || !aligned(g, 16))) return EC_ERR_INVALID_ARG;
    if (grad_format != EC_RGBA32F && grad_format != EC_RGBA16F) return EC_ERR_INVALID_ARG;
    const int fmt = n > 0 ? in[0].format : EC_RGBA32F;
    if (fmt != EC_RGBA32F && fmt != EC_RGBA16F) return EC_ERR_INVALID_ARG;
    *f16 = fmt == EC_RGBA16F;
    *g16 = grad_format == EC_RGBA16F;
    d.assign((size_t)std::max(n, 1), BwdDesc{});
    std::vector<char> seen((size_t)std::max(n, 1), 0);
    for (int k = 0; k < n; ++k) {
        const int i = order ? order[k] : k;
        if (i < 0 || i >= n || seen[i]) return EC_ERR_INVALID_ARG;
        seen[i] = 1;
        if (in[i].format != fmt) return EC_ERR_INVALID_ARG;
        const ec_status st = make_bwd_desc(in[i].pvp, in[i].roi, in[i].pitch, in[i].color, grad[i],
                                           bytes_per_px(fmt), bytes_per_px(grad_format), out_pvp, &d[k]);
        if (st != EC_OK) return st;
    }
    return EC_OK;
}

}  // namespace

extern "C" {

ec_status ec_composite_alpha_backward(ec_ctx* ctx, const ec_image* in, const int32_t* order,
                                      int32_t n, ec_rect out_pvp, const float* grad_out,
                                      void* const* grad, int32_t grad_format, ec_stream_t s)
{
    std::vector<BwdDesc> d;
    bool f16 = false, g16 = false;
    ec_status st = alpha_bwd_common(ctx, in, order, n, out_pvp, grad_out, grad, grad_format, d, &f16, &g16);
    if (st != EC_OK) return st;
    DstDesc D{};
    D.W = out_pvp.w;
    D.H = out_pvp.h;
    DeviceGuard g(ctx->device);
    if (!g.ok) return EC_ERR_CUDA;
    return cuda_status(launch_alpha_bwd(d.data(), n, f16, g16, false, D, grad_out, (cudaStream_t)s));
}

ec_status ec_composite_alpha_fwd_bwd(ec_ctx* ctx, const ec_image* in, const int32_t* order,
                                     int32_t n, const ec_target* out, float* t_final, const float* w,
                                     void* const* grad, int32_t grad_format, ec_rect* out_roi,
                                     ec_stream_t s)
{
    ec_status st = check_target(out, EC_RGBA32F, EC_RGBA16F);
    if (st != EC_OK) return st;
    if (n > 0 && in && in[0].format != out->format) return EC_ERR_INVALID_ARG;
    std::vector<BwdDesc> d;
    bool f16 = false, g16 = false;
    st = alpha_bwd_common(ctx, in, order, n, out->pvp, w, grad, grad_format, d, &f16, &g16);
    if (st != EC_OK) return st;
    if (n == 0) f16 = out->format == EC_RGBA16F;
    DstDesc D{};
    D.W = out->pvp.w;
    D.H = out->pvp.h;
    D.pitch = out->pitch;
    D.color = out->color;
    D.tfinal = t_final;
    D.vec = aligned(out->color, f16 ? 8 : 16);
    if (out_roi) *out_roi = merged_roi(in, n, out->pvp);
    DeviceGuard g(ctx->device);
    if (!g.ok) return EC_ERR_CUDA;
    return cuda_status(launch_alpha_bwd(d.data(), n, f16, g16, true, D, w, (cudaStream_t)s));
}

ec_status ec_composite_depth_backward(ec_ctx* ctx, const int16_t* winner, ec_rect out_pvp,
                                      const float* grad_out, int32_t n, const ec_rect* pvps,
                                      const int32_t* pitches, float* const* grad, ec_stream_t s)
{
    if (!ctx || n < 0 || (n > 0 && (!pvps || !pitches || !grad)) || !rect_ok(out_pvp)) return EC_ERR_INVALID_ARG;
    if (n > kMaxBwdLayers) return EC_ERR_UNSUPPORTED;
    if (!rect_empty(out_pvp) && (!winner || !grad_out || !aligned(grad_out, 16))) return EC_ERR_INVALID_ARG;
    std::vector<BwdDesc> d((size_t)std::max(n, 1));
    for (int i = 0; i < n; ++i) {
        const ec_status st = make_bwd_desc(pvps[i], ec_rect{pvps[i].x, pvps[i].y, 0, 0}, pitches[i], nullptr,
                                           grad[i], 16, 16, out_pvp, &d[i]);
        if (st != EC_OK) return st;
        if (grad[i] && !aligned(grad[i], 4)) return EC_ERR_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    if (!g.ok) return EC_ERR_CUDA;
    return cuda_status(launch_depth_bwd(d.data(), n, out_pvp.w, out_pvp.h, winner, grad_out, (cudaStream_t)s));
}

}  // extern "C"
