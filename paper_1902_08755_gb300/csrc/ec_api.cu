// ec_api.cu -- the C ABI of libec (see include/ec.h): contexts, argument
// validation and descriptor building on the host, then kernel launches.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ec_internal.cuh"

using namespace ec;

namespace {

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

ec_status ensure_roi_scratch(ec_ctx* ctx, size_t bytes)
{
    if (ctx->roi_scratch_bytes >= bytes) return EC_OK;
    if (ctx->roi_scratch) cudaFree(ctx->roi_scratch);
    ctx->roi_scratch = nullptr;
    ctx->roi_scratch_bytes = 0;
    bytes = std::max<size_t>(bytes, 16 * 1024);
    if (cudaMalloc(&ctx->roi_scratch, bytes) != cudaSuccess) return EC_ERR_CUDA;
    // the accumulators start at zero; every launch leaves them zero
    if (cudaMemset(ctx->roi_scratch, 0, bytes) != cudaSuccess) return EC_ERR_CUDA;
    ctx->roi_scratch_bytes = bytes;
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
        ensure_scratch(ctx, rle_compress_scratch_bytes(1024, kRlePoolPerUnit)) != EC_OK) {
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
    if (ctx->roi_scratch) cudaFree(ctx->roi_scratch);
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

// Target of an assembly call: any colour format, 4-byte aligned pixels.
static ec_status check_assembly_target(const ec_target* out)
{
    if (!out || bytes_per_px(out->format) == 0) return EC_ERR_INVALID_ARG;
    const ec_status st = check_target(out, out->format, out->format);
    if (st != EC_OK) return st;
    if (!rect_empty(out->pvp) && (reinterpret_cast<uintptr_t>(out->color) & 3u)) return EC_ERR_INVALID_ARG;
    return EC_OK;
}

// Inputs of an assembly call: same colour format as the target, descriptors
// relative to out->pvp.
static ec_status assembly_descs(const ec_image* in, int32_t n, const ec_target* out, std::vector<SrcDesc>& d)
{
    const int bpp = bytes_per_px(out->format);
    d.assign((size_t)std::max(n, 1), SrcDesc{});
    for (int i = 0; i < n; ++i) {
        if (in[i].format != out->format) return EC_ERR_INVALID_ARG;
        const ec_status st = make_desc(in[i], out->pvp, 16 / bpp, false, &d[i]);
        if (st != EC_OK) return st;
        if (d[i].x1 > d[i].x0 && (reinterpret_cast<uintptr_t>(in[i].color) & 3u)) return EC_ERR_INVALID_ARG;
    }
    return EC_OK;
}

static DstDesc assembly_target(const ec_target* out)
{
    const int bpp = bytes_per_px(out->format);
    DstDesc D;
    memset(&D, 0, sizeof(D));
    D.W = out->pvp.w;
    D.H = out->pvp.h;
    D.pitch = out->pitch;
    D.vec = aligned16(out->color) && ((int64_t)out->pitch * bpp) % 16 == 0;
    D.color = out->color;
    return D;
}

ec_status ec_assemble_tiles(ec_ctx* ctx, const ec_image* in, int32_t n, const ec_target* out, ec_stream_t s)
{
    if (!ctx || n < 0 || (n > 0 && !in)) return EC_ERR_INVALID_ARG;
    if (n > EC_MAX_SOURCES) return EC_ERR_UNSUPPORTED;
    ec_status st = check_assembly_target(out);
    if (st != EC_OK) return st;
    std::vector<SrcDesc> d;
    st = assembly_descs(in, n, out, d);
    if (st != EC_OK) return st;
    DeviceGuard g(ctx->device);
    if (!g.ok) return EC_ERR_CUDA;
    return cuda_status(launch_assemble_tiles(d.data(), n, bytes_per_px(out->format), assembly_target(out),
                                             (cudaStream_t)s));
}

ec_status ec_average(ec_ctx* ctx, const ec_image* in, int32_t n, const ec_target* out, ec_stream_t s)
{
    if (!ctx || n < 0 || (n > 0 && !in)) return EC_ERR_INVALID_ARG;
    if (n > EC_MAX_SOURCES) return EC_ERR_UNSUPPORTED;
    ec_status st = check_assembly_target(out);
    if (st != EC_OK) return st;
    std::vector<SrcDesc> d;
    st = assembly_descs(in, n, out, d);
    if (st != EC_OK) return st;
    const int fmt = out->format == EC_RGBA8 ? 0 : out->format == EC_RGBA32F ? 1 : 2;
    DeviceGuard g(ctx->device);
    if (!g.ok) return EC_ERR_CUDA;
    return cuda_status(launch_average(d.data(), n, fmt, assembly_target(out), (cudaStream_t)s));
}

ec_status ec_assemble_pixels(ec_ctx* ctx, const ec_image* in, const int32_t* kx, const int32_t* ky,
                             int32_t n, int32_t nx, int32_t ny, const ec_target* out, ec_stream_t s)
{
    if (!ctx || n < 0 || (n > 0 && (!in || !kx || !ky))) return EC_ERR_INVALID_ARG;
    if (nx < 1 || ny < 1 || nx > kPixMaxKernel || ny > kPixMaxKernel) return EC_ERR_INVALID_ARG;
    if (n > kPixMaxSources) return EC_ERR_UNSUPPORTED;
    ec_status st = check_assembly_target(out);
    if (st != EC_OK) return st;
    std::vector<PixSrc> src((size_t)std::max(n, 1));
    std::vector<int16_t> owner((size_t)nx * ny, (int16_t)-1);
    for (int k = 0; k < n; ++k) {
        if (in[k].format != out->format || kx[k] < 0 || kx[k] >= nx || ky[k] < 0 || ky[k] >= ny)
            return EC_ERR_INVALID_ARG;
        const int64_t w = out->pvp.w > kx[k] ? (out->pvp.w - kx[k] + nx - 1) / nx : 0;
        const int64_t h = out->pvp.h > ky[k] ? (out->pvp.h - ky[k] + ny - 1) / ny : 0;
        if (in[k].pitch < w || (w > 0 && h > 0 && (!in[k].color || (reinterpret_cast<uintptr_t>(in[k].color) & 3u))))
            return EC_ERR_INVALID_ARG;
        src[k].color = in[k].color;
        src[k].pitch = in[k].pitch;
        src[k].pad = 0;
        owner[(size_t)ky[k] * nx + kx[k]] = (int16_t)k;    // later inputs overwrite earlier ones
    }
    DeviceGuard g(ctx->device);
    if (!g.ok) return EC_ERR_CUDA;
    return cuda_status(launch_assemble_pixels(src.data(), owner.data(), n, nx, ny, bytes_per_px(out->format),
                                              assembly_target(out), (cudaStream_t)s));
}

ec_status ec_detect_roi(ec_ctx* ctx, const ec_image* in, int32_t n, int32_t tile,
                        uint8_t* const* occupancy, ec_rect* d_rois, ec_stream_t s)
{
    if (!ctx || n < 0 || (n > 0 && (!in || !d_rois))) return EC_ERR_INVALID_ARG;
    if (tile != 8 && tile != 16 && tile != 32 && tile != 64) return EC_ERR_INVALID_ARG;
    if (n > EC_MAX_SOURCES) return EC_ERR_UNSUPPORTED;
    if (reinterpret_cast<uintptr_t>(d_rois) & 3u) return EC_ERR_INVALID_ARG;
    std::vector<RoiDesc> d((size_t)std::max(n, 1));
    std::vector<uint64_t> nblocks((size_t)std::max(n, 1));
    std::vector<int> kinds((size_t)std::max(n, 1));
    for (int i = 0; i < n; ++i) {
        const ec_image& im = in[i];
        if (!rect_ok(im.pvp) || !rect_ok(im.roi) || im.pitch < im.pvp.w || im.pitch < 0 ||
            !rect_inside(im.roi, im.pvp))
            return EC_ERR_INVALID_ARG;
        int kind;
        if (im.depth) kind = 0;
        else if (im.format == EC_RGBA8) kind = 1;
        else if (im.format == EC_RGBA32F) kind = 2;
        else if (im.format == EC_RGBA16F) kind = 3;
        else return EC_ERR_INVALID_ARG;
        const void* data = im.depth ? static_cast<const void*>(im.depth) : im.color;
        const bool search = !rect_empty(im.roi);
        const uintptr_t align = kind == 3 ? 2u : 4u;
        if (search && (!data || (reinterpret_cast<uintptr_t>(data) & (align - 1)))) return EC_ERR_INVALID_ARG;
        const int bpp = kind == 2 ? 16 : kind == 3 ? 8 : 4;
        RoiDesc& r = d[i];
        memset(&r, 0, sizeof(r));
        if (search) {
            r.x0 = im.roi.x - im.pvp.x;
            r.y0 = im.roi.y - im.pvp.y;
            r.x1 = r.x0 + im.roi.w;
            r.y1 = r.y0 + im.roi.h;
        }
        r.ox = im.pvp.x;
        r.oy = im.pvp.y;
        r.pitch = im.pitch;
        r.gw = (im.pvp.w + tile - 1) / tile;
        r.gh = (im.pvp.h + tile - 1) / tile;
        r.bw = (im.pvp.w + kRoiBlkW - 1) / kRoiBlkW;
        nblocks[i] = (uint64_t)r.bw * (uint64_t)((im.pvp.h + kRoiBlkH - 1) / kRoiBlkH);
        kinds[i] = kind;
        r.vec = (int16_t)(aligned16(data) && ((int64_t)im.pitch * bpp) % 16 == 0);
        r.data = data;
        r.occ = occupancy ? occupancy[i] : nullptr;
    }
    DeviceGuard g(ctx->device);
    if (!g.ok) return EC_ERR_CUDA;
    for (int b = 0; b < n; b += kRoiPerLaunch) {
        const int cnt = std::min(kRoiPerLaunch, n - b);
        uint64_t blocks = 0;
        std::vector<uint32_t> nb((size_t)cnt);
        for (int i = 0; i < cnt; ++i) {
            d[b + i].idx = (int16_t)i;
            nb[i] = (uint32_t)nblocks[b + i];
            blocks += nblocks[b + i];
        }
        if (blocks >= (1ull << 31)) return EC_ERR_UNSUPPORTED;
        const ec_status st = ensure_roi_scratch(ctx, 4ull * cnt * sizeof(uint32_t));
        if (st != EC_OK) return st;
        const cudaError_t e = launch_detect_roi(&d[b], &kinds[b], nb.data(), cnt, tile,
                                                reinterpret_cast<uint32_t*>(ctx->roi_scratch), d_rois + b,
                                                (cudaStream_t)s);
        if (e != cudaSuccess) return EC_ERR_CUDA;
    }
    return EC_OK;
}

static ec_status yuv_batch(ec_ctx* ctx, const ec_yuv_job* jobs, int32_t njobs, bool encode, ec_stream_t s)
{
    if (!ctx || njobs < 0 || (njobs > 0 && !jobs)) return EC_ERR_INVALID_ARG;
    std::vector<YuvJob> d;
    for (int i = 0; i < njobs; ++i) {
        const ec_yuv_job& j = jobs[i];
        if (j.w < 0 || j.h < 0 || j.pitch < j.w || j.packed_pitch < (j.w + 1) / 2) return EC_ERR_INVALID_ARG;
        if ((int64_t)j.w * j.h == 0) continue;
        if (!j.src || !j.dst || (reinterpret_cast<uintptr_t>(j.src) & 3u) || (reinterpret_cast<uintptr_t>(j.dst) & 3u))
            return EC_ERR_INVALID_ARG;
        YuvJob y;
        memset(&y, 0, sizeof(y));
        y.src = static_cast<const uint32_t*>(j.src);
        y.dst = static_cast<uint32_t*>(j.dst);
        y.w = j.w;
        y.h = j.h;
        y.pitch = j.pitch;
        y.dpitch = j.packed_pitch;
        const uintptr_t rgba = reinterpret_cast<uintptr_t>(encode ? j.src : j.dst);
        const uintptr_t packed = reinterpret_cast<uintptr_t>(encode ? j.dst : j.src);
        y.vec = ((rgba & 7u) == 0 && j.pitch % 2 == 0 ? 1 : 0) |          // 8-byte RGBA pairs
                ((rgba & 15u) == 0 && j.pitch % 4 == 0 ? 2 : 0) |         // 16-byte RGBA quads
                ((packed & 7u) == 0 && j.packed_pitch % 2 == 0 ? 4 : 0);  // 8-byte packed word pairs
        d.push_back(y);
    }
    DeviceGuard g(ctx->device);
    if (!g.ok) return EC_ERR_CUDA;
    for (size_t b = 0; b < d.size(); b += kYuvJobsPerLaunch) {
        const int cnt = (int)std::min<size_t>(kYuvJobsPerLaunch, d.size() - b);
        if (launch_yuv(&d[b], cnt, encode, (cudaStream_t)s) != cudaSuccess) return EC_ERR_CUDA;
    }
    return EC_OK;
}

ec_status ec_yuv_encode_batch(ec_ctx* ctx, const ec_yuv_job* jobs, int32_t njobs, ec_stream_t s)
{
    return yuv_batch(ctx, jobs, njobs, true, s);
}

ec_status ec_yuv_decode_batch(ec_ctx* ctx, const ec_yuv_job* jobs, int32_t njobs, ec_stream_t s)
{
    return yuv_batch(ctx, jobs, njobs, false, s);
}

ec_status ec_yuv_encode(ec_ctx* ctx, const void* src, int32_t w, int32_t h, int32_t pitch, void* dst,
                        int32_t dst_pitch, ec_stream_t s)
{
    const ec_yuv_job j{src, dst, w, h, pitch, dst_pitch};
    return yuv_batch(ctx, &j, 1, true, s);
}

ec_status ec_yuv_decode(ec_ctx* ctx, const void* src, int32_t src_pitch, int32_t w, int32_t h, void* dst,
                        int32_t pitch, ec_stream_t s)
{
    const ec_yuv_job j{src, dst, w, h, pitch, src_pitch};
    return yuv_batch(ctx, &j, 1, false, s);
}

ec_status ec_selftest_wait_timeout(ec_ctx* ctx, ec_stream_t s)
{
    if (!ctx) return EC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return EC_ERR_CUDA;
    return cuda_status(launch_selftest_wait(ctx->d_status, (cudaStream_t)s));
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

}  // extern "C"

ec_status rle_job_desc(const ec_rle_job& j, bool compress, RleJobDesc* d)
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
        if (j.mode > 2) return EC_ERR_INVALID_ARG;
        if (!j.d_size || (reinterpret_cast<uintptr_t>(j.d_size) & 7u)) return EC_ERR_INVALID_ARG;
        if (j.capacity < ec_rle_max_size(j.w, j.h)) return EC_ERR_CAPACITY;
        if (n > 0 && (reinterpret_cast<uintptr_t>(j.src) & 3u)) return EC_ERR_INVALID_ARG;
        d->mode = j.mode;
        d->d_size = j.d_size;
        // 16-byte reads: rows of whole 16-byte groups, or one contiguous run
        // of a multiple of 4 elements
        d->vec = aligned16(j.src) && ((j.w % 4 == 0 && j.pitch % 4 == 0) || (j.pitch == j.w && n % 4 == 0));
    } else {
        if (!j.src || (reinterpret_cast<uintptr_t>(j.src) & 3u)) return EC_ERR_INVALID_ARG;
        if (n > 0 && (reinterpret_cast<uintptr_t>(j.dst) & 3u)) return EC_ERR_INVALID_ARG;
        d->capacity = j.capacity;
        d->vec = aligned16(j.dst) && j.w % 4 == 0 && j.pitch % 4 == 0;
    }
    return EC_OK;
}

extern "C" {

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
    // one compress launch codes one mode family: the four-plane modes first,
    // then basic RLE (mode 0)
    if (compress)
        std::stable_partition(d.begin(), d.begin() + njobs, [](const RleJobDesc& x) { return x.mode != 0; });
    for (int b = 0; b < njobs;) {
        int cnt = std::min(kRleJobsPerLaunch, njobs - b);
        if (compress)
            for (int i = 1; i < cnt; ++i)
                if ((d[b + i].mode == 0) != (d[b].mode == 0)) { cnt = i; break; }
        uint32_t units = 0;
        for (int i = 0; i < cnt; ++i) {
            d[b + i].first_unit = units;
            units += rle_units((uint64_t)d[b + i].w * (uint64_t)d[b + i].h);
        }
        cudaError_t e;
        if (compress) {
            const ec_status st = ensure_scratch(ctx, rle_compress_scratch_bytes(units, kRlePoolPerUnit));
            if (st != EC_OK) return st;
            e = launch_rle_compress(&d[b], cnt, units, ctx->scratch, ctx->scratch_bytes, ctx->d_status,
                                    (cudaStream_t)s);
        } else {
            e = launch_rle_decompress(&d[b], cnt, units, ctx->d_status, (cudaStream_t)s);
        }
        if (e != cudaSuccess) return EC_ERR_CUDA;
        b += cnt;
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

static_assert(sizeof(ec_image) == 56 && sizeof(ec_target) == 40 && sizeof(ec_rle_job) == 48 &&
                  sizeof(ec_job) == 80 && sizeof(ec_batch_config) == 28,
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

// -------------------------------------------------------------- batching ----

#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>

struct ec_batch {
    ec_ctx* ctx = nullptr;
    std::vector<BatchJob> jobs;
    std::vector<SrcDesc> srcs;
    BatchJob* d_jobs = nullptr;
    SrcDesc* d_srcs = nullptr;
    BatchItem* d_items = nullptr;
    uint32_t* d_head = nullptr;
    size_t items_cap = 0;
    int n_items = 0;
    BatchShape shape{};
    int grid = 0;
    int ctas_per_sm = 0;
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

std::mutex g_tune_lock;
std::map<std::string, BatchShape> g_tune_cache;

int job_kind(const BatchJob& j) { return j.mode; }

// Work items for one tile shape, sorted by estimated bytes moved, largest first.
std::vector<BatchItem> make_items(const ec_batch& b, const BatchShape& sh)
{
    struct Costed { double cost; int idx; BatchItem it; };
    std::vector<Costed> v;
    for (size_t j = 0; j < b.jobs.size(); ++j) {
        const BatchJob& J = b.jobs[j];
        const int m = job_kind(J);
        const int TW = sh.tw[m], TH = sh.th[m];
        const int bpp = m == 0 ? 8 : (m == 1 ? 20 : (m == 2 ? 16 : 8));
        const int tx = ceil_div(J.D.W, TW), ty = ceil_div(J.D.H, TH);
        for (int y = 0; y < ty; ++y)
            for (int x = 0; x < tx; ++x) {
                const int x0 = x * TW, y0 = y * TH;
                const int x1 = std::min(x0 + TW, J.D.W), y1 = std::min(y0 + TH, J.D.H);
                double cost = (double)(x1 - x0) * (y1 - y0) * bpp;           // output
                for (int i = 0; i < J.n; ++i) {
                    const SrcDesc& s = b.srcs[J.first + i];
                    const int64_t w = std::min(x1, s.x1) - std::max(x0, s.x0);
                    const int64_t h = std::min(y1, s.y1) - std::max(y0, s.y0);
                    if (w > 0 && h > 0) cost += (double)w * h * bpp;
                }
                BatchItem it;
                it.job = (int32_t)j;
                it.tx = (int16_t)x;
                it.ty = (int16_t)y;
                v.push_back({cost, (int)v.size(), it});
            }
    }
    std::stable_sort(v.begin(), v.end(), [](const Costed& a, const Costed& c) { return a.cost > c.cost; });
    std::vector<BatchItem> out(v.size());
    for (size_t i = 0; i < v.size(); ++i) out[i] = v[i].it;
    return out;
}

ec_status upload_items(ec_batch& b, const BatchShape& sh)
{
    const std::vector<BatchItem> items = make_items(b, sh);
    if (items.size() > b.items_cap) {
        if (b.d_items) cudaFree(b.d_items);
        b.d_items = nullptr;
        if (cudaMalloc(&b.d_items, std::max<size_t>(items.size(), 1) * sizeof(BatchItem)) != cudaSuccess)
            return EC_ERR_CUDA;
        b.items_cap = items.size();
    }
    if (!items.empty() &&
        cudaMemcpy(b.d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice) != cudaSuccess)
        return EC_ERR_CUDA;
    b.n_items = (int)items.size();
    b.shape = sh;
    return EC_OK;
}

ec_status capture(ec_batch& b)
{
    if (b.exec) { cudaGraphExecDestroy(b.exec); b.exec = nullptr; }
    if (b.graph) { cudaGraphDestroy(b.graph); b.graph = nullptr; }
    if (cudaStreamBeginCapture(b.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return EC_ERR_CUDA;
    const cudaError_t e = launch_batch(b.d_jobs, b.d_srcs, b.d_items, b.n_items, b.d_head, b.shape, b.grid, b.stream);
    const cudaError_t e2 = cudaStreamEndCapture(b.stream, &b.graph);
    if (e != cudaSuccess || e2 != cudaSuccess) return EC_ERR_CUDA;
    if (cudaGraphInstantiate(&b.exec, b.graph, 0) != cudaSuccess) return EC_ERR_CUDA;
    return EC_OK;
}

// Mean device time of a few direct launches (after one warm-up).
float time_shape(ec_batch& b, const BatchShape& sh)
{
    if (upload_items(b, sh) != EC_OK) return 1e30f;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int r = 0; r < 4; ++r) {
        cudaEventRecord(e0, b.stream);
        launch_batch(b.d_jobs, b.d_srcs, b.d_items, b.n_items, b.d_head, b.shape, b.grid, b.stream);
        cudaEventRecord(e1, b.stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

std::string signature(const ec_batch& b, int device)
{
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, device);
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](int64_t v) { h ^= (uint64_t)v; h *= 1099511628211ull; };
    mix(b.ctas_per_sm);
    for (const BatchJob& J : b.jobs) {
        mix(J.mode); mix(J.n); mix(J.D.W); mix(J.D.H);
        for (int i = 0; i < J.n; ++i) {
            const SrcDesc& s = b.srcs[J.first + i];
            mix(s.x1 - s.x0); mix(s.y1 - s.y0);
        }
    }
    char buf[64];
    snprintf(buf, sizeof(buf), "%016llx", (unsigned long long)h);
    // the key is one whitespace-free token: device names contain spaces
    std::string name(prop.name);
    for (char& ch : name)
        if (!isalnum((unsigned char)ch) && ch != '-' && ch != '.') ch = '_';
    return name + "/" + std::to_string(prop.multiProcessorCount) + "/" + buf;
}

bool shape_ok(const BatchShape& sh)
{
    for (int m = 0; m < 4; ++m) {
        const int wpx = batch_warp_px(m);
        if (sh.tw[m] <= 0 || sh.th[m] <= 0 || sh.tw[m] % wpx || sh.tw[m] > 32768 || sh.th[m] > 32768)
            return false;
    }
    return true;
}

bool cache_lookup(const std::string& sig, BatchShape* sh)
{
    std::lock_guard<std::mutex> lk(g_tune_lock);
    auto it = g_tune_cache.find(sig);
    if (it != g_tune_cache.end()) { *sh = it->second; return true; }
    const char* path = getenv("EC_AUTOTUNE_CACHE");
    if (!path) return false;
    FILE* f = fopen(path, "r");
    if (!f) return false;
    // one entry per line: key, then four tile widths and heights; lines that
    // do not parse, or whose shape the kernel cannot run, are skipped (the
    // batch is then autotuned and a fresh entry appended)
    char line[512], key[256];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        BatchShape s{};
        if (sscanf(line, "%255s %d %d %d %d %d %d %d %d", key, &s.tw[0], &s.th[0], &s.tw[1], &s.th[1],
                   &s.tw[2], &s.th[2], &s.tw[3], &s.th[3]) != 9)
            continue;
        if (sig == key && shape_ok(s)) { *sh = s; found = true; }
    }
    fclose(f);
    if (found) g_tune_cache[sig] = *sh;
    return found;
}

void cache_store(const std::string& sig, const BatchShape& sh)
{
    std::lock_guard<std::mutex> lk(g_tune_lock);
    g_tune_cache[sig] = sh;
    const char* path = getenv("EC_AUTOTUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %d %d %d %d %d %d\n", sig.c_str(), sh.tw[0], sh.th[0], sh.tw[1], sh.th[1],
            sh.tw[2], sh.th[2], sh.tw[3], sh.th[3]);
    fclose(f);
}

// Coordinate-descent search: depth shapes with the alpha shapes fixed, then
// each alpha format in turn.
BatchShape autotune(ec_batch& b)
{
    BatchShape best{{128, 128, 32, 64}, {8, 8, 8, 8}};
    bool has[4] = {false, false, false, false};
    for (const BatchJob& J : b.jobs) has[J.mode] = true;
    float t_best = time_shape(b, best);
    auto try_mode = [&](std::initializer_list<int> modes, std::initializer_list<int> widths) {
        for (int w : widths)
            for (int h : {4, 8, 16, 32}) {
                BatchShape c = best;
                for (int m : modes) { c.tw[m] = w; c.th[m] = h; }
                if (!shape_ok(c)) continue;
                const float t = time_shape(b, c);
                if (t < t_best) { t_best = t; best = c; }
            }
    };
    if (has[0] || has[1]) try_mode({0, 1}, {128, 256});
    if (has[2]) try_mode({2}, {32, 64, 128});
    if (has[3]) try_mode({3}, {64, 128});
    return best;
}

}  // namespace

extern "C" {

ec_status ec_batch_plan(ec_ctx* ctx, const ec_job* jobs, int32_t njobs, const ec_batch_config* cfg,
                        ec_batch** plan)
{
    if (!ctx || !plan || njobs < 0 || (njobs > 0 && !jobs)) return EC_ERR_INVALID_ARG;
    *plan = nullptr;
    ec_batch* b = new ec_batch;
    b->ctx = ctx;
    ec_status st = EC_OK;
    for (int j = 0; j < njobs && st == EC_OK; ++j) {
        const ec_job& job = jobs[j];
        if (job.n < 0 || (job.n > 0 && !job.in)) { st = EC_ERR_INVALID_ARG; break; }
        if (job.n > EC_MAX_BATCH_INPUTS) { st = EC_ERR_UNSUPPORTED; break; }
        BatchJob J{};
        J.n = job.n;
        J.first = (int32_t)b->srcs.size();
        const ec_target* out = &job.out;
        std::vector<SrcDesc> d;
        if (job.mode == EC_JOB_DEPTH) {
            if ((st = check_target(out, EC_RGBA8, EC_RGBA32F)) != EC_OK) break;
            d.resize((size_t)std::max(job.n, 1));
            for (int i = 0; i < job.n && st == EC_OK; ++i) {
                if (job.in[i].format != out->format) st = EC_ERR_INVALID_ARG;
                else st = make_desc(job.in[i], out->pvp, 4, true, &d[i]);
            }
            J.mode = out->format == EC_RGBA8 ? 0 : 1;
            J.D.vec = aligned16(out->color) && (!out->depth || aligned16(out->depth)) && out->pitch % 4 == 0;
            J.D.winner = job.winner;
            J.D.depth = out->depth;
        } else if (job.mode == EC_JOB_ALPHA) {
            if ((st = check_target(out, EC_RGBA32F, EC_RGBA16F)) != EC_OK) break;
            st = alpha_descs(job.in, job.order, job.n, out->format, out->pvp, d);
            const bool f16 = out->format == EC_RGBA16F;
            J.mode = f16 ? 3 : 2;
            J.D.vec = aligned16(out->color) && (!f16 || out->pitch % 2 == 0);
            J.D.tfinal = job.t_final;
        } else {
            st = EC_ERR_INVALID_ARG;
        }
        if (st != EC_OK) break;
        J.D.W = out->pvp.w;
        J.D.H = out->pvp.h;
        J.D.pitch = out->pitch;
        J.D.color = out->color;
        for (int i = 0; i < job.n; ++i) b->srcs.push_back(d[i]);
        b->jobs.push_back(J);
    }
    if (st != EC_OK) { delete b; return st; }

    DeviceGuard g(ctx->device);
    if (!g.ok) { delete b; return EC_ERR_CUDA; }
    auto fail = [&](ec_status e) { ec_batch_free(b); return e; };
    // the autotuner runs the batch on the plan's own stream: inputs written
    // by earlier work on any stream must be complete
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(EC_ERR_CUDA);
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(EC_ERR_CUDA);
    if (cudaMalloc(&b->d_jobs, std::max<size_t>(b->jobs.size(), 1) * sizeof(BatchJob)) != cudaSuccess ||
        cudaMalloc(&b->d_srcs, std::max<size_t>(b->srcs.size(), 1) * sizeof(SrcDesc)) != cudaSuccess ||
        cudaMalloc(&b->d_head, sizeof(uint32_t)) != cudaSuccess)
        return fail(EC_ERR_CUDA);
    if ((!b->jobs.empty() && cudaMemcpy(b->d_jobs, b->jobs.data(), b->jobs.size() * sizeof(BatchJob), cudaMemcpyHostToDevice) != cudaSuccess) ||
        (!b->srcs.empty() && cudaMemcpy(b->d_srcs, b->srcs.data(), b->srcs.size() * sizeof(SrcDesc), cudaMemcpyHostToDevice) != cudaSuccess))
        return fail(EC_ERR_CUDA);
    b->ctas_per_sm = (cfg && cfg->ctas_per_sm > 0) ? cfg->ctas_per_sm : batch_ctas_per_sm();
    b->grid = std::max(1, ctx->sm_count * b->ctas_per_sm);

    BatchShape sh;
    if (cfg) {
        sh = BatchShape{{cfg->depth_tile_w, cfg->depth_tile_w, cfg->alpha32_tile_w, cfg->alpha16_tile_w},
                        {cfg->depth_tile_h, cfg->depth_tile_h, cfg->alpha32_tile_h, cfg->alpha16_tile_h}};
        if (!shape_ok(sh)) return fail(EC_ERR_INVALID_ARG);
    } else {
        const std::string sig = signature(*b, ctx->device);
        if (!cache_lookup(sig, &sh)) {
            sh = autotune(*b);
            cache_store(sig, sh);
        }
    }
    if ((st = upload_items(*b, sh)) != EC_OK) return fail(st);
    if ((st = capture(*b)) != EC_OK) return fail(st);
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return fail(EC_ERR_CUDA);
    *plan = b;
    return EC_OK;
}

}  // extern "C"

cudaError_t ec::batch_enqueue(const ec_batch* b, cudaStream_t s)
{
    return launch_batch(b->d_jobs, b->d_srcs, b->d_items, b->n_items, b->d_head, b->shape, b->grid, s);
}

extern "C" {

ec_status ec_batch_run(ec_batch* b, ec_stream_t s)
{
    if (!b || !b->exec) return EC_ERR_INVALID_ARG;
    DeviceGuard g(b->ctx->device);
    if (!g.ok) return EC_ERR_CUDA;
    return cudaGraphLaunch(b->exec, (cudaStream_t)s) == cudaSuccess ? EC_OK : EC_ERR_CUDA;
}

ec_status ec_batch_get_config(const ec_batch* b, ec_batch_config* cfg, int32_t* n_items, int32_t* grid)
{
    if (!b) return EC_ERR_INVALID_ARG;
    if (cfg) {
        cfg->depth_tile_w = b->shape.tw[0];
        cfg->depth_tile_h = b->shape.th[0];
        cfg->alpha32_tile_w = b->shape.tw[2];
        cfg->alpha32_tile_h = b->shape.th[2];
        cfg->alpha16_tile_w = b->shape.tw[3];
        cfg->alpha16_tile_h = b->shape.th[3];
        cfg->ctas_per_sm = b->ctas_per_sm;
    }
    if (n_items) *n_items = b->n_items;
    if (grid) *grid = b->grid;
    return EC_OK;
}

void ec_batch_free(ec_batch* b)
{
    if (!b) return;
    DeviceGuard g(b->ctx->device);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->stream) cudaStreamDestroy(b->stream);
    if (b->d_jobs) cudaFree(b->d_jobs);
    if (b->d_srcs) cudaFree(b->d_srcs);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_head) cudaFree(b->d_head);
    delete b;
}

}  // extern "C"
