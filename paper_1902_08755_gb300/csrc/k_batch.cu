// k_batch.cu -- many independent composites in one persistent launch.
//
// Thesis 4.2.4 ("tile" compounds): fixed-size work packages sit in a queue
// and resources pull them until the queue is empty, which balances uneven
// work without a static assignment.  Here a work item is one output tile of
// one job (a job is a full composite: its inputs, mode and destination); a
// grid sized to the resident-CTA count of the device loops, each CTA taking
// the next item with one atomicAdd on a queue head.  Items are sorted by
// estimated cost, largest first (longest-processing-time order), so the tail
// of the launch is made of small items.  No CTA ever waits for another.
//
// Every item runs exactly the per-thread arithmetic of the one-frame kernels
// (composite_body.cuh), so results are bit-identical to per-job launches and
// independent of the tile shape the autotuner picks.
#include "composite_body.cuh"

namespace ec {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// A work item's active input descriptors are staged in shared memory.
// One body for every job kind.  The load phase is the same code for all of
// them: U inputs' 16-byte colour words (and, for depth jobs, their depth
// words) are requested back to back.  The fold then interprets one shared
// 12-word state per kind, so the kinds share registers instead of adding up:
//   kind 0 (depth RGBA8, 4 px/lane):  depth[0..3] colour[4..7] winner[8..11]
//   kind 1 (depth RGBA32F, 1 px/lane): depth[0] winner[1] colour[4..7]
//   kind 2 (alpha RGBA32F, 1 px/lane): C[0..3] T[4]
//   kind 3 (alpha RGBA16F, 2 px/lane): C0[0..3] C1[4..7] T0[8] T1[9]
// The per-pixel operations and their order are those of composite_body.cuh.
__device__ __forceinline__ int lane_px(int mode) { return mode == 0 ? 4 : (mode == 3 ? 2 : 1); }
__device__ __forceinline__ int warp_px(int mode) { return 32 * lane_px(mode); }

__device__ __forceinline__ void load_words(int mode, const SrcDesc& s, int x, int y, uint4& c, uint4& d)
{
    const size_t e = (size_t)(y - s.oy) * (size_t)s.pitch + (size_t)(x - s.ox);
    if (mode == 0) {
        if (s.vec) {
            c = ld_stream(reinterpret_cast<const uint4*>(reinterpret_cast<const uint32_t*>(s.color) + e));
            d = ld_stream(reinterpret_cast<const uint4*>(reinterpret_cast<const uint32_t*>(s.depth) + e));
        } else {
            uint32_t cw[4], dw[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const bool in = x + j >= s.x0 && x + j < s.x1;
                cw[j] = in ? __ldcs(reinterpret_cast<const unsigned int*>(s.color) + e + j) : 0u;
                dw[j] = in ? __ldcs(reinterpret_cast<const unsigned int*>(s.depth) + e + j) : 0x3F800000u;
            }
            c = make_uint4(cw[0], cw[1], cw[2], cw[3]);
            d = make_uint4(dw[0], dw[1], dw[2], dw[3]);
        }
    } else if (mode == 3 && !s.vec) {
        uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            if (x + j >= s.x0 && x + j < s.x1) {
                const unsigned short* h = reinterpret_cast<const unsigned short*>(s.color) + 4 * (e + j);
                w[2 * j] = (uint32_t)__ldcs(h) | ((uint32_t)__ldcs(h + 1) << 16);
                w[2 * j + 1] = (uint32_t)__ldcs(h + 2) | ((uint32_t)__ldcs(h + 3) << 16);
            }
        }
        c = make_uint4(w[0], w[1], w[2], w[3]);
    } else {                                       // one 16-byte pixel or two half pixels
        const uint8_t* p = reinterpret_cast<const uint8_t*>(s.color) + e * (mode == 3 ? 8 : 16);
        if ((reinterpret_cast<uintptr_t>(p) & 15u) == 0) {
            c = ld_stream(reinterpret_cast<const uint4*>(p));
        } else {
            const unsigned int* f = reinterpret_cast<const unsigned int*>(p);
            c = make_uint4(__ldcs(f), __ldcs(f + 1), __ldcs(f + 2), __ldcs(f + 3));
        }
        if (mode == 1) d.x = __ldcs(reinterpret_cast<const unsigned int*>(s.depth) + e);
    }
}

__device__ __forceinline__ void fold_alpha(uint32_t* st, int ai, int ti, float4 c)
{
    float T = __uint_as_float(st[ti]);
    st[ai + 0] = __float_as_uint(fmaf(T, c.x, __uint_as_float(st[ai + 0])));
    st[ai + 1] = __float_as_uint(fmaf(T, c.y, __uint_as_float(st[ai + 1])));
    st[ai + 2] = __float_as_uint(fmaf(T, c.z, __uint_as_float(st[ai + 2])));
    st[ai + 3] = __float_as_uint(fmaf(T, c.w, __uint_as_float(st[ai + 3])));
    st[ti] = __float_as_uint(fmaf(-T, c.w, T));
}

__device__ __noinline__ void batch_px(int mode, const SrcDesc* sd, const int16_t* act, int nact,
                                      int x, int y, const DstDesc& D)
{
    constexpr int U = 4;
    const int px = lane_px(mode);
    uint32_t st[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) st[k] = 0u;
    if (mode == 0) {
#pragma unroll
        for (int j = 0; j < 4; ++j) { st[j] = 0x3F800000u; st[8 + j] = 0xFFFFFFFFu; }   // 1.0, -1
    } else if (mode == 1) {
        st[0] = 0x3F800000u;
        st[1] = 0xFFFFFFFFu;
    } else if (mode == 2) {
        st[4] = 0x3F800000u;
    } else {
        st[8] = st[9] = 0x3F800000u;
    }

    for (int a = 0; a < nact; a += U) {
        uint4 c[U], d[U];
        bool live[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            live[u] = false;
            if (a + u < nact) {
                const SrcDesc& s = sd[a + u];
                live[u] = y >= s.y0 && y < s.y1 && x + px > s.x0 && x < s.x1;
                if (live[u]) load_words(mode, s, x, y, c[u], d[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!live[u]) continue;
            const SrcDesc& s = sd[a + u];
            const int idx = act[a + u];
            if (mode == 0) {
                const uint32_t cw[4] = {c[u].x, c[u].y, c[u].z, c[u].w};
                const uint32_t dw[4] = {d[u].x, d[u].y, d[u].z, d[u].w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // strict '<': ties keep the lower index or the background
                    if (x + j >= s.x0 && x + j < s.x1 && __uint_as_float(dw[j]) < __uint_as_float(st[j])) {
                        st[j] = dw[j];
                        st[4 + j] = cw[j];
                        st[8 + j] = (uint32_t)idx;
                    }
                }
            } else if (mode == 1) {
                if (__uint_as_float(d[u].x) < __uint_as_float(st[0])) {
                    st[0] = d[u].x;
                    st[1] = (uint32_t)idx;
                    st[4] = c[u].x; st[5] = c[u].y; st[6] = c[u].z; st[7] = c[u].w;
                }
            } else if (mode == 2) {
                fold_alpha(st, 0, 4, make_float4(__uint_as_float(c[u].x), __uint_as_float(c[u].y),
                                                 __uint_as_float(c[u].z), __uint_as_float(c[u].w)));
            } else {
                if (x >= s.x0 && x < s.x1) fold_alpha(st, 0, 8, half4_to_float4(make_uint2(c[u].x, c[u].y)));
                if (x + 1 >= s.x0 && x + 1 < s.x1) fold_alpha(st, 4, 9, half4_to_float4(make_uint2(c[u].z, c[u].w)));
            }
        }
    }

    const size_t o = (size_t)y * (size_t)D.pitch + (size_t)x;
    if (mode == 0) {
        uint32_t* oc = reinterpret_cast<uint32_t*>(D.color) + o;
        if (D.vec && x + 4 <= D.W) {
            st_stream(reinterpret_cast<uint4*>(oc), make_uint4(st[4], st[5], st[6], st[7]));
            if (D.depth) st_stream(reinterpret_cast<uint4*>(D.depth + o), make_uint4(st[0], st[1], st[2], st[3]));
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (x + j < D.W) {
                    oc[j] = st[4 + j];
                    if (D.depth) D.depth[o + j] = __uint_as_float(st[j]);
                }
        }
        if (D.winner)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (x + j < D.W) D.winner[(size_t)y * D.W + x + j] = (int16_t)st[8 + j];
    } else if (mode == 1) {
        uint4* oc = reinterpret_cast<uint4*>(D.color) + o;
        const uint4 v = make_uint4(st[4], st[5], st[6], st[7]);
        if ((reinterpret_cast<uintptr_t>(oc) & 15u) == 0) st_stream(oc, v);
        else { uint32_t* w = reinterpret_cast<uint32_t*>(oc); w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w; }
        if (D.depth) D.depth[o] = __uint_as_float(st[0]);
        if (D.winner) D.winner[(size_t)y * D.W + x] = (int16_t)st[1];
    } else if (mode == 2) {
        const uint4 v = make_uint4(st[0], st[1], st[2], st[3]);
        uint4* op = reinterpret_cast<uint4*>(D.color) + o;
        if (D.vec) st_stream(op, v);
        else { uint32_t* w = reinterpret_cast<uint32_t*>(op); w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w; }
        if (D.tfinal) D.tfinal[(size_t)y * D.W + x] = __uint_as_float(st[4]);
    } else {
        const uint2 h0 = float4_to_half4(make_float4(__uint_as_float(st[0]), __uint_as_float(st[1]),
                                                     __uint_as_float(st[2]), __uint_as_float(st[3])));
        const uint2 h1 = float4_to_half4(make_float4(__uint_as_float(st[4]), __uint_as_float(st[5]),
                                                     __uint_as_float(st[6]), __uint_as_float(st[7])));
        uint2* op = reinterpret_cast<uint2*>(D.color) + o;
        if (D.vec && x + 2 <= D.W) {
            st_stream(reinterpret_cast<uint4*>(op), make_uint4(h0.x, h0.y, h1.x, h1.y));
        } else {
            unsigned short* hp = reinterpret_cast<unsigned short*>(op);
            hp[0] = (unsigned short)h0.x; hp[1] = (unsigned short)(h0.x >> 16);
            hp[2] = (unsigned short)h0.y; hp[3] = (unsigned short)(h0.y >> 16);
            if (x + 1 < D.W) {
                hp[4] = (unsigned short)h1.x; hp[5] = (unsigned short)(h1.x >> 16);
                hp[6] = (unsigned short)h1.y; hp[7] = (unsigned short)(h1.y >> 16);
            }
        }
        if (D.tfinal) {
            D.tfinal[(size_t)y * D.W + x] = __uint_as_float(st[8]);
            if (x + 1 < D.W) D.tfinal[(size_t)y * D.W + x + 1] = __uint_as_float(st[9]);
        }
    }
}

__global__ void __launch_bounds__(kThreads, 4)
k_batch(const BatchJob* __restrict__ jobs, const SrcDesc* __restrict__ srcs,
        const BatchItem* __restrict__ items, int n_items, uint32_t* head, BatchShape shape)
{
    __shared__ int16_t act[EC_MAX_BATCH_INPUTS];
    __shared__ SrcDesc sdesc[EC_MAX_BATCH_INPUTS];
    __shared__ int nact_s;
    __shared__ int s_item;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd(head, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;                   // uniform: the queue is empty
        const BatchItem bi = items[it];
        const BatchJob& J = jobs[bi.job];
        const int mode = J.mode;
        const int TW = shape.tw[mode], TH = shape.th[mode];
        const int tx0 = bi.tx * TW, ty0 = bi.ty * TH;
        const int tx1 = min(tx0 + TW, J.D.W), ty1 = min(ty0 + TH, J.D.H);
        const SrcDesc* js = srcs + J.first;
        build_active([&](int, int i) -> const SrcDesc& { return js[i]; }, J.n, tx0, ty0, tx1, ty1, act,
                     &nact_s);
        __syncthreads();
        const int nact = nact_s;
        for (int k = tid; k < nact; k += kThreads) sdesc[k] = js[act[k]];
        __syncthreads();
        const int wpx = warp_px(mode), lpx = lane_px(mode);
        const int segs = TW / wpx, tasks = TH * segs;
        const DstDesc D = J.D;
        for (int r = warp; r < tasks; r += kWarps) {
            const int y = ty0 + r / segs, x = tx0 + (r % segs) * wpx + lane * lpx;
            if (y < ty1 && x < tx1) batch_px(mode, sdesc, act, nact, x, y, D);
        }
        __syncthreads();                            // act / s_item are reused by the next item
    }
}

}  // namespace

int batch_warp_px(int mode) { return 32 * (mode == 0 ? 4 : (mode == 3 ? 2 : 1)); }

int batch_ctas_per_sm()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch, kThreads, 0) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_batch(const BatchJob* jobs, const SrcDesc* srcs, const BatchItem* items,
                         int n_items, uint32_t* head, const BatchShape& shape, int grid,
                         cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(head, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    if (n_items <= 0) return cudaSuccess;
    k_batch<<<grid, kThreads, 0, s>>>(jobs, srcs, items, n_items, head, shape);
    return cudaGetLastError();
}

}  // namespace ec
