// ec_schedule.cu -- multi-stage compositing schedules on one GPU.
//
// Thesis 5.2.2 (direct send, binary swap and its extension 2-3 swap) and
// 5.2.3 (streaming sort-last compositing): n rendering resources exchange
// parts of their partial frames in stages; at every stage each resource
// composites what it holds with what it receives, in source-index order;
// finally each resource owns a part of the frame (the stream's last resource
// owns all of it).  Transfers carry only the sender's ROI inside the region
// sent (thesis 5.3) and, with EC_SCHED_RLE, travel RLE-compressed
// (thesis 5.5.1).
//
// Here the resources are buffers in one GPU's memory.  A plan fixes the
// geometry from the inputs' ROIs (regions, pieces, partial ROIs), lays every
// intermediate buffer and stream out in one device arena, and captures the
// whole schedule in a CUDA graph; a run replays it.  Each level of the
// schedule becomes at most four launches:
//   1. one compress launch for all of the level's transfers (colour mode 2,
//      depth mode 1);
//   2. a decompress launch for the transfers of stages that are not fused;
//   3. one fused decode-and-composite launch (k_fused_depth) for the stages
//      that merge one plain local input with the coded pieces of one other
//      unit (every stage of binary swap and of the stream);
//   4. one persistent batch launch (k_batch) compositing every other stage
//      from its pieces in order.
// Stages of the last level write straight into the destination's regions.
//
// Planning (the thesis prints no algorithm for the splits; these readings): regions
// are rectangles of out->pvp; a rectangle is cut into k row bands at rows
// floor(j h / k); binary swap halves a region across its longer side (rows
// when h >= w, the first half floor(len/2)), the lower resource of a pair
// keeping the first half; 2-3 swap groups the current units consecutively in
// pairs (a triple last when their count is odd), orders a group's resources
// by the first row of their region and then by unit, and deals them the
// frame's row bands in that order.  A receiver's pieces are the
// intersections of every group member's region and ROI with its new region,
// composited unit by unit in index order; its new ROI is their bounding box.
#include "ec_internal.cuh"

#include <algorithm>
#include <cstring>
#include <vector>

namespace {

using ec::FusedStage;
using ec::FusedUnit;
using ec::RleJobDesc;

constexpr ec_rect kEmpty{0, 0, 0, 0};

bool is_empty(const ec_rect& r) { return r.w <= 0 || r.h <= 0; }

ec_rect isect(const ec_rect& a, const ec_rect& b)
{
    const int64_t x0 = std::max(a.x, b.x), y0 = std::max(a.y, b.y);
    const int64_t x1 = std::min((int64_t)a.x + a.w, (int64_t)b.x + b.w);
    const int64_t y1 = std::min((int64_t)a.y + a.h, (int64_t)b.y + b.h);
    if (x1 <= x0 || y1 <= y0) return kEmpty;
    return ec_rect{(int32_t)x0, (int32_t)y0, (int32_t)(x1 - x0), (int32_t)(y1 - y0)};
}

ec_rect bound(const ec_rect& a, const ec_rect& b)
{
    if (is_empty(a)) return b;
    if (is_empty(b)) return a;
    const int64_t x0 = std::min(a.x, b.x), y0 = std::min(a.y, b.y);
    const int64_t x1 = std::max((int64_t)a.x + a.w, (int64_t)b.x + b.w);
    const int64_t y1 = std::max((int64_t)a.y + a.h, (int64_t)b.y + b.h);
    return ec_rect{(int32_t)x0, (int32_t)y0, (int32_t)(x1 - x0), (int32_t)(y1 - y0)};
}

std::vector<ec_rect> row_bands(const ec_rect& R, int k)
{
    std::vector<ec_rect> v;
    for (int j = 0; j < k; ++j) {
        const int32_t a = R.y + (int32_t)(((int64_t)j * R.h) / k);
        const int32_t b = R.y + (int32_t)(((int64_t)(j + 1) * R.h) / k);
        v.push_back(ec_rect{R.x, a, R.w, b - a});
    }
    return v;
}

void halve(const ec_rect& R, ec_rect* first, ec_rect* second)
{
    if (R.h >= R.w) {
        const int32_t m = R.h / 2;
        *first = ec_rect{R.x, R.y, R.w, m};
        *second = ec_rect{R.x, R.y + m, R.w, R.h - m};
    } else {
        const int32_t m = R.w / 2;
        *first = ec_rect{R.x, R.y, m, R.h};
        *second = ec_rect{R.x + m, R.y, R.w - m, R.h};
    }
}

// Parts of O that none of the holes cover, as rectangles (row sweep).
std::vector<ec_rect> subtract(const ec_rect& O, const std::vector<ec_rect>& holes_in)
{
    std::vector<ec_rect> holes;
    for (const ec_rect& h : holes_in) {
        const ec_rect c = isect(h, O);
        if (!is_empty(c)) holes.push_back(c);
    }
    std::vector<int32_t> ys{O.y, O.y + O.h};
    for (const ec_rect& h : holes) { ys.push_back(h.y); ys.push_back(h.y + h.h); }
    std::sort(ys.begin(), ys.end());
    ys.erase(std::unique(ys.begin(), ys.end()), ys.end());
    std::vector<ec_rect> out;
    for (size_t i = 0; i + 1 < ys.size(); ++i) {
        const int32_t y0 = ys[i], y1 = ys[i + 1];
        if (y0 < O.y || y1 > O.y + O.h || y1 <= y0) continue;
        std::vector<std::pair<int32_t, int32_t>> xs;
        for (const ec_rect& h : holes)
            if (h.y <= y0 && h.y + h.h >= y1) xs.push_back({h.x, h.x + h.w});
        std::sort(xs.begin(), xs.end());
        int32_t x = O.x;
        auto emit = [&](int32_t a, int32_t b) {
            if (b <= a) return;
            // extend a rectangle of the previous band with the same columns
            for (ec_rect& r : out)
                if (r.x == a && r.w == b - a && r.y + r.h == y0) { r.h += y1 - y0; return; }
            out.push_back(ec_rect{a, y0, b - a, y1 - y0});
        };
        for (const auto& iv : xs) {
            emit(x, iv.first);
            x = std::max(x, iv.second);
        }
        emit(x, O.x + O.w);
    }
    return out;
}

// ---------------------------------------------------------------- planner

struct Piece {
    int sender;
    int unit;      // unit of the sender within the group
    ec_rect r;
};

struct Stage {
    int receiver = 0;
    ec_rect region = kEmpty;
    int n_units = 0, own_unit = 0;
    std::vector<Piece> pieces;     // compositing order
    ec_rect roi = kEmpty;
};

struct Planner {
    int n = 0;
    ec_rect frame = kEmpty;
    std::vector<ec_rect> region, roi;
    std::vector<std::vector<Stage>> levels;

    using Group = std::vector<std::vector<int>>;   // units of nodes

    void level(const std::vector<Group>& groups, const std::vector<ec_rect>& nr)
    {
        std::vector<Stage> lv;
        for (const Group& g : groups)
            for (size_t ui = 0; ui < g.size(); ++ui)
                for (int r : g[ui]) {
                    Stage st;
                    st.receiver = r;
                    st.region = nr[r];
                    st.n_units = (int)g.size();
                    st.own_unit = (int)ui;
                    for (size_t uj = 0; uj < g.size(); ++uj)
                        for (int m : g[uj]) {
                            const ec_rect p = isect(isect(region[m], nr[r]), roi[m]);
                            if (is_empty(p)) continue;
                            st.pieces.push_back(Piece{m, (int)uj, p});
                            st.roi = bound(st.roi, p);
                        }
                    lv.push_back(st);
                }
        for (const Stage& st : lv) {
            region[st.receiver] = st.region;
            roi[st.receiver] = st.roi;
        }
        levels.push_back(std::move(lv));
    }

    ec_status plan(int algo)
    {
        region.assign(n, frame);
        std::vector<ec_rect> nr(n, kEmpty);
        switch (algo) {
        case EC_SCHED_STREAM:
            for (int l = 0; l + 1 < n; ++l) {
                nr[l] = kEmpty;
                nr[l + 1] = frame;
                level({Group{{l}, {l + 1}}}, nr);
            }
            return EC_OK;
        case EC_SCHED_DIRECT_SEND: {
            if (n == 1) return EC_OK;
            const std::vector<ec_rect> b = row_bands(frame, n);
            Group g;
            for (int i = 0; i < n; ++i) {
                g.push_back({i});
                nr[i] = b[i];
            }
            level({g}, nr);
            return EC_OK;
        }
        case EC_SCHED_BINARY_SWAP:
            if (n & (n - 1)) return EC_ERR_INVALID_ARG;
            for (int s = 1; s < n; s *= 2) {
                std::vector<Group> groups;
                for (int a = 0; a < n; a += 2 * s) {
                    Group g(2);
                    for (int j = 0; j < s; ++j) {
                        g[0].push_back(a + j);
                        g[1].push_back(a + s + j);
                        halve(region[a + j], &nr[a + j], &nr[a + s + j]);
                    }
                    groups.push_back(g);
                }
                level(groups, nr);
            }
            return EC_OK;
        case EC_SCHED_TWO_THREE_SWAP: {
            std::vector<std::vector<int>> units;
            for (int i = 0; i < n; ++i) units.push_back({i});
            while (units.size() > 1) {
                const size_t k = units.size();
                std::vector<size_t> sizes(k / 2, 2);
                if (k % 2) sizes.back() = 3;
                std::vector<Group> groups;
                std::vector<std::vector<int>> merged;
                size_t at = 0;
                for (size_t sz : sizes) {
                    Group g(units.begin() + at, units.begin() + at + sz);
                    at += sz;
                    struct Key { int32_t y; int unit, pos, node; };
                    std::vector<Key> keys;
                    for (size_t ui = 0; ui < g.size(); ++ui)
                        for (size_t p = 0; p < g[ui].size(); ++p)
                            keys.push_back(Key{region[g[ui][p]].y, (int)ui, (int)p, g[ui][p]});
                    std::sort(keys.begin(), keys.end(), [](const Key& a, const Key& b) {
                        if (a.y != b.y) return a.y < b.y;
                        if (a.unit != b.unit) return a.unit < b.unit;
                        return a.pos < b.pos;
                    });
                    const std::vector<ec_rect> b = row_bands(frame, (int)keys.size());
                    std::vector<int> members;
                    for (size_t i = 0; i < keys.size(); ++i) {
                        nr[keys[i].node] = b[i];
                        members.push_back(keys[i].node);
                    }
                    std::sort(members.begin(), members.end());
                    groups.push_back(g);
                    merged.push_back(members);
                }
                level(groups, nr);
                units = merged;
            }
            return EC_OK;
        }
        default:
            return EC_ERR_INVALID_ARG;
        }
    }
};

// ------------------------------------------------------------- executor

// A buffer of pixels: absolute pointers, or offsets into the plan's arena.
struct Buf {
    bool arena = false;
    const char* c = nullptr;
    const char* d = nullptr;
    size_t c_off = 0, d_off = 0;
    int32_t pitch = 0, ox = 0, oy = 0;   // element [0][0] is frame pixel (ox, oy)

    char* color(char* base) const { return arena ? base + c_off : const_cast<char*>(c); }
    char* depth(char* base) const { return arena ? base + d_off : const_cast<char*>(d); }
};

struct Xfer {
    int sender = 0, receiver = 0;
    ec_rect piece = kEmpty;
    Buf src;                                   // the sender's buffer
    size_t cs_off = 0, ds_off = 0, cap = 0, sz_off = 0;   // streams and their two sizes
    bool fused = false;
    Buf raw;                                   // decoded piece (stages not fused)
};

struct StageRec {
    Stage st;
    bool fused = false;
    Buf local;                    // the receiver's buffer before the level
    Buf out;
    ec_rect out_rect = kEmpty;
    std::vector<int> xfer;        // per piece: transfer index, or -1 for the local piece
};

struct LevelRec {
    std::vector<Xfer> xfers;
    std::vector<StageRec> stages;
    size_t fst_off = 0, fun_off = 0;
    int n_fused_units = 0;
};

int32_t round4(int32_t v) { return (v + 3) & ~3; }
uint64_t chunks(const ec_rect& r) { return ((uint64_t)r.w * r.h + EC_RLE_CHUNK - 1) / EC_RLE_CHUNK; }

// Fill units take whole rows, about one chunk's worth of pixels each.
int32_t fill_rows(const ec_rect& r) { return std::max<int32_t>(1, EC_RLE_CHUNK / std::max<int32_t>(r.w, 1)); }
uint64_t fill_units(const ec_rect& r) { return ((uint64_t)r.h + fill_rows(r) - 1) / fill_rows(r); }

struct Arena {
    size_t top = 0;
    size_t take(size_t bytes)
    {
        const size_t o = top;
        top += (bytes + 255) & ~size_t(255);
        return o;
    }
};

int bytes_per_pixel(int fmt) { return fmt == EC_RGBA32F ? 16 : (fmt == EC_RGBA16F ? 8 : 4); }

ec_status check_image(const ec_image& im, int fmt, bool need_depth)
{
    if (im.format != fmt || im.pvp.w < 0 || im.pvp.h < 0 || im.roi.w < 0 || im.roi.h < 0 || im.pitch < im.pvp.w)
        return EC_ERR_INVALID_ARG;
    if (!is_empty(isect(im.roi, im.pvp)) && (!im.color || (need_depth && !im.depth))) return EC_ERR_INVALID_ARG;
    return EC_OK;
}

// The image of piece p read from buffer b.
ec_image piece_image(const Buf& b, char* base, const ec_rect& p, int fmt, int bpp, bool depth)
{
    ec_image im;
    im.pvp = p;
    im.roi = p;
    im.pitch = b.pitch;
    im.format = fmt;
    const size_t e = (size_t)(p.y - b.oy) * b.pitch + (p.x - b.ox);
    im.color = b.color(base) + e * bpp;
    im.depth = depth ? reinterpret_cast<const float*>(b.depth(base)) + e : nullptr;
    return im;
}

ec_target buf_target(const Buf& b, char* base, const ec_rect& r, int fmt, int bpp, bool depth)
{
    ec_target t;
    t.pvp = r;
    t.pitch = b.pitch;
    t.format = fmt;
    const size_t e = (size_t)(r.y - b.oy) * b.pitch + (r.x - b.ox);
    t.color = b.color(base) + e * bpp;
    t.depth = depth ? reinterpret_cast<float*>(b.depth(base)) + e : nullptr;
    return t;
}

}  // namespace

// One kernel launch of a schedule: the graph is captured from these, and
// ec_schedule_run_launch enqueues one alone.
struct SchedLaunch {
    int kind = 0;                        // EC_SCHED_LAUNCH_*
    int level = 0;
    std::vector<ec::RleJobDesc> jobs;    // codec launches
    uint32_t units = 0;
    const ec::FusedStage* stages = nullptr;
    const ec::FusedUnit* funits = nullptr;
    int n_units = 0;
    ec_batch* batch = nullptr;
    uint64_t bytes = 0;                  // pixel bytes read and written (streams not counted)
};

struct ec_schedule {
    ec_ctx* ctx = nullptr;
    std::vector<SchedLaunch> launches;
    void* scratch = nullptr;             // the compressor's scratch, inside the arena
    size_t scratch_bytes = 0;
    int mode = 0, algo = 0, n = 0, fmt = 0;
    uint32_t flags = 0;
    char* arena = nullptr;
    size_t arena_bytes = 0;
    std::vector<ec_sched_message> msgs;
    std::vector<size_t> size_offs;        // per message: offset of its two stream sizes
    std::vector<ec_batch*> batches;
    int n_levels = 0, n_launches = 0;
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

cudaError_t enqueue(ec_schedule* S, const SchedLaunch& r, cudaStream_t s)
{
    switch (r.kind) {
    case EC_SCHED_LAUNCH_COMPRESS:
        return ec::launch_rle_compress(r.jobs.data(), (int)r.jobs.size(), r.units, S->scratch, S->scratch_bytes,
                                       S->ctx->d_status, s);
    case EC_SCHED_LAUNCH_DECOMPRESS:
        return ec::launch_rle_decompress(r.jobs.data(), (int)r.jobs.size(), r.units, S->ctx->d_status, s);
    case EC_SCHED_LAUNCH_FUSED:
        return ec::launch_fused_depth(r.stages, r.funits, r.n_units, S->ctx->d_status, s);
    default:
        return ec::batch_enqueue(r.batch, s);
    }
}

}  // namespace

extern "C" {

ec_status ec_schedule_plan(ec_ctx* ctx, int32_t mode, int32_t algorithm, const ec_image* in, int32_t n,
                           const int32_t* order, const ec_target* out, uint32_t flags, ec_schedule** plan)
{
    if (!ctx || !plan || !out || n < 1 || !in) return EC_ERR_INVALID_ARG;
    *plan = nullptr;
    if (n > EC_MAX_SOURCES) return EC_ERR_UNSUPPORTED;
    if (flags & ~(uint32_t)(EC_SCHED_RLE | EC_SCHED_FUSED)) return EC_ERR_INVALID_ARG;
    const bool depth = mode == EC_JOB_DEPTH;
    if (!depth && mode != EC_JOB_ALPHA) return EC_ERR_INVALID_ARG;
    const bool rle = (flags & EC_SCHED_RLE) != 0;
    const bool fuse = rle && (flags & EC_SCHED_FUSED) != 0;
    const int fmt = out->format;
    if (depth) {
        if (fmt != EC_RGBA8 && fmt != EC_RGBA32F) return EC_ERR_INVALID_ARG;
        if (!out->depth) return EC_ERR_INVALID_ARG;
        if (rle && fmt != EC_RGBA8) return EC_ERR_UNSUPPORTED;     // the codec carries 4-byte pixels
    } else {
        if (fmt != EC_RGBA32F && fmt != EC_RGBA16F) return EC_ERR_INVALID_ARG;
        if (rle) return EC_ERR_UNSUPPORTED;                         // alpha partials travel raw
    }
    if (!out->color || out->pvp.w < 0 || out->pvp.h < 0 || out->pitch < out->pvp.w) return EC_ERR_INVALID_ARG;
    const int bpp = bytes_per_pixel(fmt);

    // resource i holds input order[i] (alpha, front to back) or input i (depth)
    std::vector<int> src(n);
    if (!depth && order) {
        std::vector<char> seen(n, 0);
        for (int i = 0; i < n; ++i) {
            if (order[i] < 0 || order[i] >= n || seen[order[i]]) return EC_ERR_INVALID_ARG;
            seen[order[i]] = 1;
            src[i] = order[i];
        }
    } else {
        for (int i = 0; i < n; ++i) src[i] = i;
    }
    for (int i = 0; i < n; ++i) {
        const ec_status st = check_image(in[i], fmt, depth);
        if (st != EC_OK) return st;
    }

    Planner P;
    P.n = n;
    P.frame = out->pvp;
    for (int i = 0; i < n; ++i) P.roi.push_back(isect(isect(in[src[i]].roi, in[src[i]].pvp), out->pvp));
    {
        const ec_status st = P.plan(algorithm);
        if (st != EC_OK) return st;
    }

    ec_schedule* S = new ec_schedule;
    S->ctx = ctx;
    S->mode = mode;
    S->algo = algorithm;
    S->n = n;
    S->fmt = fmt;
    S->flags = flags;
    S->n_levels = (int)P.levels.size();
    auto fail = [&](ec_status e) { ec_schedule_free(S); return e; };

    // ---- phase 1: buffers, streams and stage kinds, as arena offsets
    Arena A;
    std::vector<Buf> node(n);
    for (int i = 0; i < n; ++i) {
        const ec_image& im = in[src[i]];
        node[i].c = reinterpret_cast<const char*>(im.color);
        node[i].d = reinterpret_cast<const char*>(im.depth);
        node[i].pitch = im.pitch;
        node[i].ox = im.pvp.x;
        node[i].oy = im.pvp.y;
    }
    Buf target;
    target.c = reinterpret_cast<const char*>(out->color);
    target.d = reinterpret_cast<const char*>(out->depth);
    target.pitch = out->pitch;
    target.ox = out->pvp.x;
    target.oy = out->pvp.y;

    std::vector<LevelRec> L(P.levels.size());
    uint64_t max_units = 0;
    for (size_t li = 0; li < P.levels.size(); ++li) {
        const bool last = li + 1 == P.levels.size();
        LevelRec& lr = L[li];
        std::vector<Buf> next = node;
        uint64_t level_units = 0;
        for (const Stage& st : P.levels[li]) {
            StageRec sr;
            sr.st = st;
            const int r = st.receiver;
            sr.local = node[r];
            sr.out_rect = last ? st.region : st.roi;
            bool own_only = true;
            for (const Piece& p : st.pieces)
                if (p.unit == st.own_unit && p.sender != r) own_only = false;
            sr.fused = fuse && st.n_units == 2 && own_only;
            if (!sr.fused && st.pieces.size() > EC_MAX_BATCH_INPUTS) return fail(EC_ERR_UNSUPPORTED);
            for (const Piece& p : st.pieces) {
                if (p.sender == r) { sr.xfer.push_back(-1); continue; }
                Xfer x;
                x.sender = p.sender;
                x.receiver = r;
                x.piece = p.r;
                x.src = node[p.sender];
                x.fused = sr.fused;
                if (rle) {
                    if ((uint64_t)p.r.w * p.r.h > EC_RLE_MAX_ELEMS) return fail(EC_ERR_UNSUPPORTED);
                    x.cap = ec_rle_max_size(p.r.w, p.r.h);
                    x.cs_off = A.take(x.cap);
                    x.ds_off = A.take(x.cap);
                    x.sz_off = A.take(16);
                    level_units += 2 * chunks(p.r);
                    if (!sr.fused) {
                        x.raw.arena = true;
                        x.raw.pitch = round4(p.r.w);
                        x.raw.ox = p.r.x;
                        x.raw.oy = p.r.y;
                        x.raw.c_off = A.take((size_t)x.raw.pitch * p.r.h * 4);
                        x.raw.d_off = A.take((size_t)x.raw.pitch * p.r.h * 4);
                    }
                } else {
                    x.raw = x.src;                   // zero-copy: read the sender's buffer
                }
                sr.xfer.push_back((int)lr.xfers.size());
                lr.xfers.push_back(x);
            }
            if (!is_empty(sr.out_rect)) {
                if (last) {
                    sr.out = target;
                } else {
                    // the buffer starts at a frame column that is a multiple of 4, so
                    // that four pixels from such a column are one 16-byte access
                    Buf b;
                    b.arena = true;
                    b.ox = sr.out_rect.x & ~3;
                    b.oy = sr.out_rect.y;
                    b.pitch = round4(sr.out_rect.x + sr.out_rect.w - b.ox);
                    b.c_off = A.take((size_t)b.pitch * sr.out_rect.h * bpp);
                    if (depth) b.d_off = A.take((size_t)b.pitch * sr.out_rect.h * 4);
                    sr.out = b;
                }
            }
            next[r] = sr.out;
            lr.stages.push_back(std::move(sr));
        }
        max_units = std::max(max_units, level_units);
        node = next;
        // fused stage and unit tables
        size_t ns = 0, nu = 0;
        for (const StageRec& sr : lr.stages) {
            if (!sr.fused || is_empty(sr.out_rect)) continue;
            ++ns;
            std::vector<ec_rect> holes;
            for (size_t k = 0; k < sr.st.pieces.size(); ++k)
                if (sr.xfer[k] >= 0) {
                    holes.push_back(sr.st.pieces[k].r);
                    nu += chunks(sr.st.pieces[k].r);
                }
            for (const ec_rect& f : subtract(sr.out_rect, holes)) nu += fill_units(f);
        }
        if (nu > (size_t)INT32_MAX) return fail(EC_ERR_UNSUPPORTED);
        lr.n_fused_units = (int)nu;
        lr.fst_off = A.take(std::max<size_t>(ns, 1) * sizeof(FusedStage));
        lr.fun_off = A.take(std::max<size_t>(nu, 1) * sizeof(FusedUnit));
    }
    const size_t scratch_bytes = ec::rle_compress_scratch_bytes((uint32_t)std::max<uint64_t>(max_units, 1),
                                                                ec::kRlePoolPerUnit);
    const size_t scratch_off = A.take(scratch_bytes);

    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(EC_ERR_CUDA);
    S->arena_bytes = std::max<size_t>(A.top, 256);
    if (cudaMalloc(&S->arena, S->arena_bytes) != cudaSuccess) return fail(EC_ERR_CUDA);
    char* base = S->arena;
    if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(EC_ERR_CUDA);

    // ---- phase 2: descriptors
    std::vector<std::vector<RleJobDesc>> cjobs(L.size()), djobs(L.size());
    std::vector<std::vector<FusedStage>> fst(L.size());
    std::vector<std::vector<FusedUnit>> fun(L.size());
    std::vector<ec_batch*> level_batch(L.size() + 1, nullptr);
    ec_batch_config bcfg{128, 8, 32, 8, 64, 8, 0};
    for (size_t li = 0; li < L.size(); ++li) {
        LevelRec& lr = L[li];
        for (const Xfer& x : lr.xfers) {
            ec_sched_message m;
            m.level = (int32_t)li;
            m.sender = x.sender;
            m.receiver = x.receiver;
            m.fused = x.fused ? 1 : 0;
            m.piece = x.piece;
            S->msgs.push_back(m);
            S->size_offs.push_back(rle ? x.sz_off : SIZE_MAX);
            if (!rle) continue;
            const size_t e = (size_t)(x.piece.y - x.src.oy) * x.src.pitch + (x.piece.x - x.src.ox);
            for (int k = 0; k < 2; ++k) {
                ec_rle_job j;
                j.src = (k ? x.src.depth(base) : x.src.color(base)) + 4 * e;
                j.dst = base + (k ? x.ds_off : x.cs_off);
                j.capacity = x.cap;
                j.d_size = reinterpret_cast<uint64_t*>(base + x.sz_off) + k;
                j.w = x.piece.w;
                j.h = x.piece.h;
                j.pitch = x.src.pitch;
                j.mode = k ? 1u : 2u;
                RleJobDesc d;
                ec_status st = rle_job_desc(j, true, &d);
                if (st != EC_OK) return fail(st);
                cjobs[li].push_back(d);
                if (!x.fused) {
                    ec_rle_job u;
                    u.src = j.dst;
                    u.dst = k ? x.raw.depth(base) : x.raw.color(base);
                    u.capacity = x.cap;
                    u.d_size = nullptr;
                    u.w = x.piece.w;
                    u.h = x.piece.h;
                    u.pitch = x.raw.pitch;
                    u.mode = 0;
                    if ((st = rle_job_desc(u, false, &d)) != EC_OK) return fail(st);
                    djobs[li].push_back(d);
                }
            }
        }
        std::vector<ec_job> jobs;
        std::vector<std::vector<ec_image>> jimgs;
        jimgs.reserve(lr.stages.size());
        for (const StageRec& sr : lr.stages) {
            if (is_empty(sr.out_rect)) continue;
            if (sr.fused) {
                FusedStage fs;
                memset(&fs, 0, sizeof(fs));
                fs.oc = reinterpret_cast<uint32_t*>(sr.out.color(base));
                fs.od = reinterpret_cast<float*>(sr.out.depth(base));
                fs.opitch = sr.out.pitch;
                fs.ox = sr.out.ox;
                fs.oy = sr.out.oy;
                fs.ovec = aligned16(fs.oc) && aligned16(fs.od) && fs.opitch % 4 == 0;
                fs.lc = reinterpret_cast<const uint32_t*>(sr.local.color(base));
                fs.ld = reinterpret_cast<const float*>(sr.local.depth(base));
                fs.lpitch = sr.local.pitch;
                fs.lx = sr.local.ox;
                fs.ly = sr.local.oy;
                fs.lvec = aligned16(fs.lc) && aligned16(fs.ld) && fs.lpitch % 4 == 0;
                int other = -1;
                std::vector<ec_rect> holes;
                for (size_t k = 0; k < sr.st.pieces.size(); ++k) {
                    const Piece& p = sr.st.pieces[k];
                    if (sr.xfer[k] < 0) {
                        fs.r0x = p.r.x;
                        fs.r0y = p.r.y;
                        fs.r1x = p.r.x + p.r.w;
                        fs.r1y = p.r.y + p.r.h;
                    } else {
                        other = p.unit;
                        holes.push_back(p.r);
                    }
                }
                fs.front = other >= 0 && other < sr.st.own_unit ? 1 : 0;
                const int si = (int)fst[li].size();
                fst[li].push_back(fs);
                for (size_t k = 0; k < sr.st.pieces.size(); ++k) {
                    if (sr.xfer[k] < 0) continue;
                    const Xfer& x = lr.xfers[sr.xfer[k]];
                    for (uint64_t c = 0; c < chunks(x.piece); ++c) {
                        FusedUnit u;
                        memset(&u, 0, sizeof(u));
                        u.cs = reinterpret_cast<const uint8_t*>(base + x.cs_off);
                        u.ds = reinterpret_cast<const uint8_t*>(base + x.ds_off);
                        u.csize = reinterpret_cast<const uint64_t*>(base + x.sz_off);
                        u.dsize = u.csize + 1;
                        u.cap = (uint32_t)x.cap;
                        u.stage = si;
                        u.x = x.piece.x;
                        u.y = x.piece.y;
                        u.w = x.piece.w;
                        u.h = x.piece.h;
                        u.chunk = (uint32_t)c;
                        fun[li].push_back(u);
                    }
                }
                for (const ec_rect& f : subtract(sr.out_rect, holes))
                    for (int32_t r0 = 0; r0 < f.h; r0 += fill_rows(f)) {
                        FusedUnit u;
                        memset(&u, 0, sizeof(u));
                        u.stage = si;
                        u.x = f.x;
                        u.y = f.y;
                        u.w = f.w;
                        u.h = f.h;
                        u.chunk = (uint32_t)r0;
                        u.nrows = std::min(fill_rows(f), f.h - r0);
                        fun[li].push_back(u);
                    }
                continue;
            }
            std::vector<ec_image> im;
            for (size_t k = 0; k < sr.st.pieces.size(); ++k) {
                const ec_rect& p = sr.st.pieces[k].r;
                const Buf& b = sr.xfer[k] < 0 ? sr.local : lr.xfers[sr.xfer[k]].raw;
                im.push_back(piece_image(b, base, p, fmt, bpp, depth));
            }
            jimgs.push_back(std::move(im));
            ec_job j;
            memset(&j, 0, sizeof(j));
            j.mode = mode;
            j.n = (int32_t)jimgs.back().size();
            j.in = jimgs.back().data();
            j.order = nullptr;
            j.out = buf_target(sr.out, base, sr.out_rect, fmt, bpp, depth);
            jobs.push_back(j);
        }
        if ((int)fun[li].size() != lr.n_fused_units) return fail(EC_ERR_INVALID_ARG);
        if (!jobs.empty()) {
            const ec_status st = ec_batch_plan(ctx, jobs.data(), (int32_t)jobs.size(), &bcfg, &level_batch[li]);
            if (st != EC_OK) return fail(st);
            S->batches.push_back(level_batch[li]);
        }
        if (!fst[li].empty() &&
            (cudaMemcpy(base + lr.fst_off, fst[li].data(), fst[li].size() * sizeof(FusedStage), cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(base + lr.fun_off, fun[li].data(), fun[li].size() * sizeof(FusedUnit), cudaMemcpyHostToDevice) != cudaSuccess))
            return fail(EC_ERR_CUDA);
    }
    if (L.empty()) {
        // one resource: its image against the background, written in place
        ec_job j;
        memset(&j, 0, sizeof(j));
        j.mode = mode;
        j.n = 1;
        j.in = &in[src[0]];
        j.out = *out;
        const ec_status st = ec_batch_plan(ctx, &j, 1, &bcfg, &level_batch[0]);
        if (st != EC_OK) return fail(st);
        S->batches.push_back(level_batch[0]);
    }

    // ---- phase 3: launch records, then the graph
    S->scratch = base + scratch_off;
    S->scratch_bytes = scratch_bytes;
    const uint64_t pxb = (uint64_t)bpp + (depth ? 4u : 0u);    // bytes per pixel with depth
    for (size_t li = 0; li < L.size(); ++li) {
        for (int kind = EC_SCHED_LAUNCH_COMPRESS; kind <= EC_SCHED_LAUNCH_DECOMPRESS; ++kind) {
            std::vector<RleJobDesc>& jobs = kind == EC_SCHED_LAUNCH_COMPRESS ? cjobs[li] : djobs[li];
            for (size_t b = 0; b < jobs.size(); b += ec::kRleJobsPerLaunch) {
                const int cnt = (int)std::min<size_t>(ec::kRleJobsPerLaunch, jobs.size() - b);
                SchedLaunch r;
                r.kind = kind;
                r.level = (int)li;
                for (int i = 0; i < cnt; ++i) {
                    RleJobDesc d = jobs[b + i];
                    d.first_unit = r.units;
                    r.units += (uint32_t)std::max<uint64_t>(1, chunks(ec_rect{0, 0, d.w, d.h}));
                    r.bytes += 4ull * (uint64_t)d.w * (uint64_t)d.h;
                    r.jobs.push_back(d);
                }
                S->launches.push_back(std::move(r));
            }
        }
        if (L[li].n_fused_units > 0) {
            SchedLaunch r;
            r.kind = EC_SCHED_LAUNCH_FUSED;
            r.level = (int)li;
            r.stages = reinterpret_cast<const FusedStage*>(base + L[li].fst_off);
            r.funits = reinterpret_cast<const FusedUnit*>(base + L[li].fun_off);
            r.n_units = L[li].n_fused_units;
            for (const StageRec& sr : L[li].stages) {
                if (!sr.fused || is_empty(sr.out_rect)) continue;
                r.bytes += 8ull * sr.out_rect.w * sr.out_rect.h;
                for (size_t k = 0; k < sr.st.pieces.size(); ++k)
                    if (sr.xfer[k] < 0) r.bytes += 8ull * sr.st.pieces[k].r.w * sr.st.pieces[k].r.h;
            }
            S->launches.push_back(std::move(r));
        }
        if (level_batch[li]) {
            SchedLaunch r;
            r.kind = EC_SCHED_LAUNCH_COMPOSITE;
            r.level = (int)li;
            r.batch = level_batch[li];
            for (const StageRec& sr : L[li].stages) {
                if (sr.fused || is_empty(sr.out_rect)) continue;
                r.bytes += pxb * sr.out_rect.w * sr.out_rect.h;
                for (const Piece& p : sr.st.pieces) r.bytes += pxb * p.r.w * p.r.h;
            }
            S->launches.push_back(std::move(r));
        }
    }
    if (L.empty()) {
        SchedLaunch r;
        r.kind = EC_SCHED_LAUNCH_COMPOSITE;
        r.batch = level_batch[0];
        const ec_rect c = P.roi[0];
        r.bytes = pxb * ((uint64_t)out->pvp.w * out->pvp.h + (uint64_t)c.w * c.h);
        S->launches.push_back(std::move(r));
    }
    S->n_launches = (int)S->launches.size();
    if (cudaStreamBeginCapture(S->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return fail(EC_ERR_CUDA);
    cudaError_t e = cudaSuccess;
    for (const SchedLaunch& r : S->launches)
        if (e == cudaSuccess) e = enqueue(S, r, S->stream);
    const cudaError_t e2 = cudaStreamEndCapture(S->stream, &S->graph);
    if (e != cudaSuccess || e2 != cudaSuccess) return fail(EC_ERR_CUDA);
    if (cudaGraphInstantiate(&S->exec, S->graph, 0) != cudaSuccess) return fail(EC_ERR_CUDA);
    *plan = S;
    return EC_OK;
}

ec_status ec_schedule_geometry(int32_t algorithm, const ec_rect* rois, int32_t n, ec_rect frame,
                               ec_sched_message* msgs, int32_t cap, int32_t* n_messages, int32_t* n_levels,
                               ec_rect* regions)
{
    if (n < 1 || !rois || cap < 0 || (cap > 0 && !msgs) || frame.w < 0 || frame.h < 0) return EC_ERR_INVALID_ARG;
    if (n > EC_MAX_SOURCES) return EC_ERR_UNSUPPORTED;
    Planner P;
    P.n = n;
    P.frame = frame;
    for (int i = 0; i < n; ++i) {
        if (rois[i].w < 0 || rois[i].h < 0) return EC_ERR_INVALID_ARG;
        P.roi.push_back(isect(rois[i], frame));
    }
    const ec_status st = P.plan(algorithm);
    if (st != EC_OK) return st;
    int32_t m = 0;
    for (size_t li = 0; li < P.levels.size(); ++li)
        for (const Stage& sg : P.levels[li])
            for (const Piece& p : sg.pieces) {
                if (p.sender == sg.receiver) continue;
                if (m < cap) {
                    msgs[m].level = (int32_t)li;
                    msgs[m].sender = p.sender;
                    msgs[m].receiver = sg.receiver;
                    msgs[m].fused = 0;
                    msgs[m].piece = p.r;
                }
                ++m;
            }
    if (n_messages) *n_messages = m;
    if (n_levels) *n_levels = (int32_t)P.levels.size();
    if (regions)
        for (int i = 0; i < n; ++i) regions[i] = P.region[i];
    return m > cap ? EC_ERR_CAPACITY : EC_OK;
}

ec_status ec_schedule_run(ec_schedule* S, ec_stream_t s)
{
    if (!S || !S->exec) return EC_ERR_INVALID_ARG;
    DeviceGuard g(S->ctx->device);
    if (!g.ok) return EC_ERR_CUDA;
    return cudaGraphLaunch(S->exec, (cudaStream_t)s) == cudaSuccess ? EC_OK : EC_ERR_CUDA;
}

ec_status ec_schedule_info(const ec_schedule* S, int32_t* n_levels, int32_t* n_messages, int32_t* n_launches,
                           uint64_t* arena_bytes)
{
    if (!S) return EC_ERR_INVALID_ARG;
    if (n_levels) *n_levels = S->n_levels;
    if (n_messages) *n_messages = (int32_t)S->msgs.size();
    if (n_launches) *n_launches = S->n_launches;
    if (arena_bytes) *arena_bytes = S->arena_bytes;
    return EC_OK;
}

ec_status ec_schedule_launches(const ec_schedule* S, ec_sched_launch* out, int32_t cap)
{
    if (!S || cap < 0 || (cap > 0 && !out)) return EC_ERR_INVALID_ARG;
    if ((size_t)cap < S->launches.size()) return EC_ERR_CAPACITY;
    for (size_t i = 0; i < S->launches.size(); ++i) {
        out[i].level = S->launches[i].level;
        out[i].kind = S->launches[i].kind;
        out[i].bytes = S->launches[i].bytes;
    }
    return EC_OK;
}

ec_status ec_schedule_run_launch(ec_schedule* S, int32_t i, ec_stream_t s)
{
    if (!S || i < 0 || (size_t)i >= S->launches.size()) return EC_ERR_INVALID_ARG;
    DeviceGuard g(S->ctx->device);
    if (!g.ok) return EC_ERR_CUDA;
    return enqueue(S, S->launches[i], (cudaStream_t)s) == cudaSuccess ? EC_OK : EC_ERR_CUDA;
}

ec_status ec_schedule_messages(const ec_schedule* S, ec_sched_message* msgs, int32_t cap)
{
    if (!S || cap < 0 || (cap > 0 && !msgs)) return EC_ERR_INVALID_ARG;
    if ((size_t)cap < S->msgs.size()) return EC_ERR_CAPACITY;
    if (!S->msgs.empty()) memcpy(msgs, S->msgs.data(), S->msgs.size() * sizeof(ec_sched_message));
    return EC_OK;
}

ec_status ec_schedule_stream_sizes(ec_schedule* S, uint64_t* sizes, int32_t cap, ec_stream_t s)
{
    if (!S || cap < 0 || (cap > 0 && !sizes)) return EC_ERR_INVALID_ARG;
    if ((size_t)cap < 2 * S->msgs.size()) return EC_ERR_CAPACITY;
    if (!(S->flags & EC_SCHED_RLE)) return EC_ERR_UNSUPPORTED;
    DeviceGuard g(S->ctx->device);
    if (!g.ok) return EC_ERR_CUDA;
    if (cudaStreamSynchronize((cudaStream_t)s) != cudaSuccess) return EC_ERR_CUDA;
    for (size_t i = 0; i < S->msgs.size(); ++i)
        if (cudaMemcpy(sizes + 2 * i, S->arena + S->size_offs[i], 16, cudaMemcpyDeviceToHost) != cudaSuccess)
            return EC_ERR_CUDA;
    return EC_OK;
}

void ec_schedule_free(ec_schedule* S)
{
    if (!S) return;
    DeviceGuard g(S->ctx->device);
    if (S->exec) cudaGraphExecDestroy(S->exec);
    if (S->graph) cudaGraphDestroy(S->graph);
    for (ec_batch* b : S->batches) ec_batch_free(b);
    if (S->stream) cudaStreamDestroy(S->stream);
    if (S->arena) cudaFree(S->arena);
    delete S;
}

}  // extern "C"
