// k_fused.cu -- fused decode-and-composite for the stages of multi-stage
// compositing schedules (thesis 5.2.2 binary swap, 5.2.3 streaming
// compositing): a resource receives RLE-coded pieces (thesis 5.5.1) of another
// resource's partial frame and depth-merges them with its own image
// (thesis 5.2.1) without writing the decoded pieces to memory first.
//
// One CTA of eight warps per work unit.  A decode unit is one 4096-element
// chunk of a received piece: warps 0-3 walk the colour stream's four byte
// planes and warps 4-7 the depth stream's (the decoder of the RLE kernels,
// including its validation).  When every plane has at most 255 runs they
// record the runs only: between the union of the eight planes' run starts
// colour and depth are constant, so each segment's pair is assembled once and
// a pixel's pair is found by its rank among the run starts.  Otherwise they
// decode the planes into shared memory, and pixels are transposed back from
// them with funnel shifts.  The threads take the chunk's pixels four at a
// time (quads aligned to the output's 16-byte boundaries), read the local
// input at the same frame pixels and write the merge.  A fill unit,
// a band of rows that no piece reaches, writes the local input (or the
// background) there.
//
// The merge of a front and a back partial: the front is first merged with the
// cleared background (depth not below 1.0, or NaN, gives the background), then
// the back replaces it where its depth is strictly smaller.  A partial that is
// already a composite is unchanged by the first step, a raw source image is
// made one, and ties stay with the front, the lower source indices.
#include "ec_internal.cuh"
#include "rle_codec.cuh"

namespace ec {
namespace {

constexpr int kFT = 256;
constexpr int kChunk = rlec::kChunk;
constexpr uint32_t kBgDepth = 0x3F800000u;   // 1.0f
constexpr int kStageWords = 1024;             // staged stream bytes per stream: 4 KB

__device__ __forceinline__ bool below_one(uint32_t d) { return __uint_as_float(d) < 1.0f; }
__device__ __forceinline__ bool less(uint32_t a, uint32_t b) { return __uint_as_float(a) < __uint_as_float(b); }

// Merge one pixel: front (fc, fd) and back (bc, bd) as raw bits.
__device__ __forceinline__ void merge(uint32_t fc, uint32_t fd, uint32_t bc, uint32_t bd, uint32_t& oc, uint32_t& od)
{
    if (!below_one(fd)) { fc = 0u; fd = kBgDepth; }
    const bool b = less(bd, fd);
    oc = b ? bc : fc;
    od = b ? bd : fd;
}

// Pixels are handled in quads: four horizontally adjacent pixels whose first
// one sits at a 16-byte boundary of the output buffer (x - ox a multiple of
// 4), so that a quad inside the unit is one 16-byte store.  A unit covers
// `nrows` rows of its rectangle from row `ra`; a decode unit only the elements
// [q0, q0 + len) of its chunk (element q = row * w + column).
struct Quad {
    int fx, fy, lo, hi, qa;       // frame position, pixels [lo, hi) inside the unit, element of pixel 0
    uint32_t lc[4], ld[4];        // the receiver's own image there
};

struct Grid {
    int qx0, nq, slots;
    float inv;
};

template <bool CODED>
__device__ __forceinline__ bool quad_at(const FusedUnit& u, const Grid& g, int s, int ra, int q0, int len, Quad& Q)
{
    int r = (int)((float)s * g.inv);
    if (r * g.nq > s) --r;
    else if ((r + 1) * g.nq <= s) ++r;
    const int row = ra + r;
    Q.fx = g.qx0 + 4 * (s - r * g.nq);
    Q.fy = u.y + row;
    const int xs = Q.fx - u.x;
    Q.lo = max(0, -xs);
    Q.hi = min(4, u.w - xs);
    Q.qa = row * u.w + xs;
    if (CODED) {
        Q.lo = max(Q.lo, q0 - Q.qa);
        Q.hi = min(Q.hi, q0 + len - Q.qa);
    }
    return Q.lo < Q.hi;
}

// The receiver's own image at the quad (background outside its ROI).
__device__ __forceinline__ void load_local(const FusedStage& S, Quad& Q)
{
    const bool in_y = Q.fy >= S.r0y && Q.fy < S.r1y;
    const size_t le = (size_t)(Q.fy - S.ly) * S.lpitch + (Q.fx - S.lx);
    if (in_y && Q.fx >= S.r0x && Q.fx + 3 < S.r1x && S.lvec && (le & 3) == 0) {
        const uint4 c = __ldcs(reinterpret_cast<const uint4*>(S.lc + le));
        const uint4 d = __ldcs(reinterpret_cast<const uint4*>(S.ld + le));
        Q.lc[0] = c.x; Q.lc[1] = c.y; Q.lc[2] = c.z; Q.lc[3] = c.w;
        Q.ld[0] = d.x; Q.ld[1] = d.y; Q.ld[2] = d.z; Q.ld[3] = d.w;
        return;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        Q.lc[k] = 0u;
        Q.ld[k] = kBgDepth;
        if (k >= Q.lo && k < Q.hi && in_y && Q.fx + k >= S.r0x && Q.fx + k < S.r1x) {
            Q.lc[k] = __ldcs(S.lc + le + k);
            Q.ld[k] = __ldcs(reinterpret_cast<const uint32_t*>(S.ld) + le + k);
        }
    }
}

// Run path of a decode unit: the chunk's elements are constant between the
// union of its eight planes' run starts.  U: that union (128 words), PU: the
// segments starting before each word, SC / SD: each segment's colour and depth.
struct Segs {
    const uint32_t* U;
    const uint32_t* PU;
    const uint32_t* SC;
    const uint32_t* SD;
};

template <bool CODED>
__device__ __forceinline__ void finish(const FusedStage& S, const Quad& Q, int q0, const uint8_t (*planes)[kChunk],
                                       bool csw, bool dsw, const Segs* G = nullptr)
{
    uint32_t oc[4], od[4];
    if (CODED && G) {
        const int i0 = Q.qa - q0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t ic = 0u, id = kBgDepth;
            if (k >= Q.lo && k < Q.hi) {
                const int i = i0 + k;
                const uint32_t u = G->U[i >> 5];
                const uint32_t s = G->PU[i >> 5] + __popc(u & ((2u << (i & 31)) - 1u)) - 1u;
                ic = G->SC[s];
                id = G->SD[s];
            }
            if (S.front) merge(ic, id, Q.lc[k], Q.ld[k], oc[k], od[k]);
            else merge(Q.lc[k], Q.ld[k], ic, id, oc[k], od[k]);
        }
    } else if (CODED) {
        // bytes of elements qa - q0 .. +3 of every plane: two words and a funnel shift
        const int i0 = Q.qa - q0;
        const int wi = i0 >> 2, sh = 8 * (i0 & 3);
        const int w0 = max(wi, 0), w1 = min(wi + 1, kChunk / 4 - 1);
        uint32_t pb[8];
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            const uint32_t* pl = reinterpret_cast<const uint32_t*>(planes[p]);
            pb[p] = __funnelshift_r(pl[w0], pl[w1], sh);
        }
        const uint4 C = rlec::transpose4(pb[0], pb[1], pb[2], pb[3]);
        const uint4 D = rlec::transpose4(pb[4], pb[5], pb[6], pb[7]);
        uint32_t ic[4] = {C.x, C.y, C.z, C.w}, id[4] = {D.x, D.y, D.z, D.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (csw) ic[k] = rlec::swizzle(ic[k]);
            if (dsw) id[k] = rlec::swizzle(id[k]);
            if (S.front) merge(ic[k], id[k], Q.lc[k], Q.ld[k], oc[k], od[k]);
            else merge(Q.lc[k], Q.ld[k], ic[k], id[k], oc[k], od[k]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool keep = below_one(Q.ld[k]);
            oc[k] = keep ? Q.lc[k] : 0u;
            od[k] = keep ? Q.ld[k] : kBgDepth;
        }
    }
    const size_t oe = (size_t)(Q.fy - S.oy) * S.opitch + (Q.fx - S.ox);
    if (Q.lo == 0 && Q.hi == 4 && S.ovec) {
        st_stream(reinterpret_cast<uint4*>(S.oc + oe), make_uint4(oc[0], oc[1], oc[2], oc[3]));
        st_stream(reinterpret_cast<uint4*>(S.od + oe), make_uint4(od[0], od[1], od[2], od[3]));
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (k >= Q.lo && k < Q.hi) {
                S.oc[oe + k] = oc[k];
                reinterpret_cast<uint32_t*>(S.od)[oe + k] = od[k];
            }
    }
}

__device__ __forceinline__ Grid grid_of(const FusedStage& S, const FusedUnit& u, int nrows)
{
    Grid g;
    g.qx0 = u.x - ((u.x - S.ox) & 3);
    g.nq = (u.x + u.w - g.qx0 + 3) >> 2;
    g.slots = nrows * g.nq;
    g.inv = 1.0f / (float)g.nq;
    return g;
}

// Two quads per thread at a time: both local loads are in flight together.
template <bool CODED>
__device__ __forceinline__ void compose(const FusedStage& S, const FusedUnit& u, int ra, int nrows,
                                        int q0, int len, const uint8_t (*planes)[kChunk], bool csw, bool dsw,
                                        const Segs* G = nullptr)
{
    const Grid g = grid_of(S, u, nrows);
    for (int s = threadIdx.x; s < g.slots; s += 2 * kFT) {
        Quad A, B;
        const bool a = quad_at<CODED>(u, g, s, ra, q0, len, A);
        const bool b = s + kFT < g.slots && quad_at<CODED>(u, g, s + kFT, ra, q0, len, B);
        if (a) load_local(S, A);
        if (b) load_local(S, B);
        if (a) finish<CODED>(S, A, q0, planes, csw, dsw, G);
        if (b) finish<CODED>(S, B, q0, planes, csw, dsw, G);
    }
}

__global__ void __launch_bounds__(kFT, 5)
k_fused_depth(const FusedStage* __restrict__ stages, const FusedUnit* __restrict__ units, uint32_t* status)
{
    __shared__ __align__(16) uint8_t planes[8][kChunk];
    __shared__ __align__(16) uint32_t staged[2][kStageWords];
    __shared__ uint8_t s_hdr[2][rlec::kHdrBytes];
    __shared__ uint32_t s_beg[2][5];
    __shared__ int s_mode[2];
    __shared__ int s_fail, s_over;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const FusedUnit u = units[blockIdx.x];
    const FusedStage S = stages[u.stage];

    if (u.cs == nullptr) {                    // fill: rows [chunk, chunk + nrows) of the rectangle
        compose<false>(S, u, (int)u.chunk, u.nrows, 0, 0, planes, false, false);
        return;
    }
    const uint32_t n = (uint32_t)u.w * (uint32_t)u.h;
    const uint32_t q0 = u.chunk * (uint32_t)kChunk;
    const int len = (int)min((uint32_t)kChunk, n - q0);
    const uint32_t nc = (n + kChunk - 1) / kChunk;
    const int ra = (int)(q0 / (uint32_t)u.w), rb = (int)((q0 + (uint32_t)len - 1u) / (uint32_t)u.w);
    // header bytes are read within the streams' capacity, in parallel with
    // their sizes; the validation then uses the sizes
    const uint64_t csz = *u.csize, dsz = *u.dsize;
    if (tid < rlec::kHdrBytes) s_hdr[0][tid] = rlec::header_byte(u.cs, (uint64_t)u.cap, nc, u.chunk, tid);
    else if (tid >= 64 && tid < 64 + rlec::kHdrBytes)
        s_hdr[1][tid - 64] = rlec::header_byte(u.ds, (uint64_t)u.cap, nc, u.chunk, tid - 64);
    if (tid == 0) { s_fail = 0; s_over = 0; }
    // the run bitmaps (aliased with the planes) start empty
    uint32_t* bm = reinterpret_cast<uint32_t*>(&planes[0][0]);       // [8][128] run starts per plane
    for (int i = tid; i < 8 * 128; i += kFT) bm[i] = 0u;
    __syncthreads();
    if (tid == 0 || tid == 32) {
        const int k = tid >> 5;
        if (rlec::check_header(s_hdr[k], k ? dsz : csz, (uint32_t)u.w, (uint32_t)u.h, nc, u.chunk,
                               s_beg[k], &s_mode[k]))
            s_fail = 1;
    }
    __syncthreads();
    if (s_fail) {
        if (tid == 0) set_status(status, EC_ERR_CORRUPT);
        return;
    }
    // stage each stream's bytes of this chunk (its four planes are contiguous)
    // in shared memory when they fit, so that the decoder's dependent steps wait
    // on shared memory instead of global memory
    const uint8_t* cpay = u.cs + 32 + 16ull * nc;
    const uint8_t* dpay = u.ds + 32 + 16ull * nc;
    const int cw0 = (int)(s_beg[0][0] >> 2), cnw = (int)((s_beg[0][4] + 3u) >> 2) - cw0;
    const int dw0 = (int)(s_beg[1][0] >> 2), dnw = (int)((s_beg[1][4] + 3u) >> 2) - dw0;
    if (cnw <= kStageWords)
        for (int i = tid; i < cnw; i += kFT) staged[0][i] = __ldg(reinterpret_cast<const uint32_t*>(cpay) + cw0 + i);
    if (dnw <= kStageWords)
        for (int i = tid; i < dnw; i += kFT) staged[1][i] = __ldg(reinterpret_cast<const uint32_t*>(dpay) + dw0 + i);
    __syncthreads();
    // run path: warp k*4+p walks stream k's plane p, recording its runs
    uint8_t* const base8 = &planes[0][0];
    {
        const int k = warp >> 2, p = warp & 3;
        const int b = (int)s_beg[k][p], e = (int)s_beg[k][p + 1];
        const int w0 = k ? dw0 : cw0, nw = k ? dnw : cnw;
        uint8_t* val = base8 + 4096 + 256 * warp;                   // [8][256] run bytes
        int nr = 0;
        const int r = nw <= kStageWords
            ? rlec::decode_plane_runs(rlec::SharedBytes{reinterpret_cast<const uint8_t*>(staged[k]), 4 * w0},
                                      b, e, len, bm + 128 * warp, val, 255, &nr, lane)
            : rlec::decode_plane_runs(rlec::GlobalBytes{k ? dpay : cpay}, b, e, len, bm + 128 * warp, val, 255,
                                      &nr, lane);
        if (r == 1 && lane == 0) s_fail = 1;
        if (r == 2 && lane == 0) s_over = 1;
    }
    __syncthreads();
    if (s_fail) {
        if (tid == 0) set_status(status, EC_ERR_CORRUPT);
        return;
    }
    if (!s_over) {
        uint32_t* U = reinterpret_cast<uint32_t*>(base8 + 6144);
        uint32_t* PU = U + 128;
        uint32_t* wt = PU + 128;                                     // scan scratch
        uint32_t* SC = reinterpret_cast<uint32_t*>(base8 + 7296);    // <= 8 * 255 segments
        uint32_t* SD = SC + 2040;
        const uint8_t* val = base8 + 4096;
        const bool csw = s_mode[0] == 2, dsw = s_mode[1] == 2;
        uint32_t un = 0u, eu = 0u, ec = 0u, ed = 0u, wb[8];
        if (tid < 128) {
#pragma unroll
            for (int q = 0; q < 8; ++q) { wb[q] = bm[128 * q + tid]; un |= wb[q]; }
            const uint32_t cu = __popc(un);
            const uint32_t cc = __popc(wb[0]) | (__popc(wb[1]) << 8) | (__popc(wb[2]) << 16) | ((uint32_t)__popc(wb[3]) << 24);
            const uint32_t cd = __popc(wb[4]) | (__popc(wb[5]) << 8) | (__popc(wb[6]) << 16) | ((uint32_t)__popc(wb[7]) << 24);
            uint32_t iu = cu, ic = cc, id = cd;      // (a plane has <= 255 runs: its byte never carries)
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t yu = __shfl_up_sync(0xffffffffu, iu, o), yc = __shfl_up_sync(0xffffffffu, ic, o);
                const uint32_t yd = __shfl_up_sync(0xffffffffu, id, o);
                if (lane >= o) { iu += yu; ic += yc; id += yd; }
            }
            if (lane == 31) { wt[3 * warp] = iu; wt[3 * warp + 1] = ic; wt[3 * warp + 2] = id; }
            eu = iu - cu; ec = ic - cc; ed = id - cd;
        }
        __syncthreads();
        if (tid < 128) {
            for (int w = 0; w < warp; ++w) { eu += wt[3 * w]; ec += wt[3 * w + 1]; ed += wt[3 * w + 2]; }
            U[tid] = un;
            PU[tid] = eu;
            for (uint32_t m = un; m; m &= m - 1u) {
                const int bb = __ffs(m) - 1;
                const uint32_t le = (2u << bb) - 1u;
                uint32_t c = 0u, d = 0u;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t rc = ((ec >> (8 * q)) & 0xFFu) + __popc(wb[q] & le) - 1u;
                    const uint32_t rd = ((ed >> (8 * q)) & 0xFFu) + __popc(wb[4 + q] & le) - 1u;
                    c |= (uint32_t)val[256 * q + rc] << (8 * q);
                    d |= (uint32_t)val[256 * (4 + q) + rd] << (8 * q);
                }
                const uint32_t sidx = eu + __popc(un & (le >> 1));
                SC[sidx] = csw ? rlec::swizzle(c) : c;
                SD[sidx] = dsw ? rlec::swizzle(d) : d;
            }
        }
        __syncthreads();
        const Segs G{U, PU, SC, SD};
        compose<true>(S, u, ra, rb - ra + 1, (int)q0, len, planes, false, false, &G);
        return;
    }
    // many runs: decode the planes into shared memory
    {
        const int k = warp >> 2, p = warp & 3;
        const int b = (int)s_beg[k][p], e = (int)s_beg[k][p + 1];
        const int w0 = k ? dw0 : cw0, nw = k ? dnw : cnw;
        const int bad = nw <= kStageWords
            ? rlec::decode_plane(rlec::SharedBytes{reinterpret_cast<const uint8_t*>(staged[k]), 4 * w0},
                                 b, e, len, planes[warp], lane)
            : rlec::decode_plane(rlec::GlobalBytes{k ? dpay : cpay}, b, e, len, planes[warp], lane);
        if (bad && lane == 0) s_fail = 1;
    }
    __syncthreads();
    if (s_fail) {
        if (tid == 0) set_status(status, EC_ERR_CORRUPT);
        return;
    }
    compose<true>(S, u, ra, rb - ra + 1, (int)q0, len, planes, s_mode[0] == 2, s_mode[1] == 2);
}

}  // namespace

cudaError_t launch_fused_depth(const FusedStage* stages, const FusedUnit* units, int n_units,
                               uint32_t* status, cudaStream_t s)
{
    if (n_units <= 0) return cudaSuccess;
    k_fused_depth<<<n_units, kFT, 0, s>>>(stages, units, status);
    return cudaGetLastError();
}

}  // namespace ec
