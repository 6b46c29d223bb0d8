// composite_body.cuh -- per-thread bodies of the compositing kernels, shared by
// the one-launch-per-frame kernels (k_composite.cu, input descriptors in the
// kernel parameters) and the persistent batch kernel (k_batch.cu, descriptors
// staged in shared memory per work item).  `at(pos, i)` returns the SrcDesc of
// input i, which sits at position pos of the tile's active list.
//
// Depth merge: thesis 5.2.1 (front-most depth wins), 3.6/5.6 (any arrival
// order, so ties go to the lower index).  Ordered "over": thesis 5.2.1
// (partial images of a spatial decomposition blended in sorted order).  Both
// read inputs only inside their ROI (thesis 5.3).
#pragma once

#include "ec_internal.cuh"

namespace ec {

// Inputs 0..n-1 whose clipped ROI meets [tx0,tx1) x [ty0,ty1), in ascending
// order, compacted by warp 0 with ballots.  Caller synchronises.
template <class At>
__device__ __forceinline__ void build_active(At at, int n, int tx0, int ty0, int tx1, int ty1,
                                             int16_t* act, int* nact)
{
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        int base = 0;
        for (int i0 = 0; i0 < n; i0 += 32) {
            const int i = i0 + lane;
            bool hit = false;
            if (i < n) {
                const SrcDesc& s = at(i, i);
                hit = s.x0 < tx1 && s.x1 > tx0 && s.y0 < ty1 && s.y1 > ty0;
            }
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (hit) act[base + __popc(m & ((1u << lane) - 1u))] = (int16_t)i;
            base += __popc(m);
        }
        if (lane == 0) *nact = base;
    }
}

// ----------------------------------------------------------------- depth ---

template <int CB> struct ColorT;
template <> struct ColorT<4> { using T = uint32_t; };
template <> struct ColorT<16> { using T = float4; };

__device__ __forceinline__ void zero(uint32_t& c) { c = 0u; }
__device__ __forceinline__ void zero(float4& c) { c = make_float4(0.f, 0.f, 0.f, 0.f); }

// 4 consecutive pixels of one source: 16-byte loads (vec) or per-pixel loads.
template <int CB>
__device__ __forceinline__ void load4(const SrcDesc& s, int x, int y, float (&d)[4],
                                      typename ColorT<CB>::T (&c)[4])
{
    using C = typename ColorT<CB>::T;
    const size_t e = (size_t)(y - s.oy) * (size_t)s.pitch + (size_t)(x - s.ox);
    const float* dp = s.depth + e;
    const C* cp = reinterpret_cast<const C*>(s.color) + e;
    if (s.vec) {
        const float4 d4 = ld_stream(reinterpret_cast<const float4*>(dp));
        d[0] = d4.x; d[1] = d4.y; d[2] = d4.z; d[3] = d4.w;
        if constexpr (CB == 4) {
            const uint4 c4 = ld_stream(reinterpret_cast<const uint4*>(cp));
            c[0] = c4.x; c[1] = c4.y; c[2] = c4.z; c[3] = c4.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) c[j] = ld_stream(cp + j);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int xj = x + j;
            if (xj >= s.x0 && xj < s.x1) {
                d[j] = __ldcs(dp + j);
                if constexpr (CB == 4) c[j] = __ldcs(reinterpret_cast<const unsigned int*>(cp + j));
                else c[j] = __ldcs(cp + j);
            } else {
                d[j] = 1.0f;
                zero(c[j]);
            }
        }
    }
}

// Depth merge of the 4 pixels x..x+3 of row y (output-relative coordinates),
// U inputs' loads in flight per thread.
template <int CB, class At, int U = 4>
__device__ __forceinline__ void depth_px4(At at, const int16_t* act, int nact, int x, int y,
                                          const DstDesc& D)
{
    using C = typename ColorT<CB>::T;
    float bd[4] = {1.0f, 1.0f, 1.0f, 1.0f};  // cleared depth
    C bc[4];
    int bi[4] = {-1, -1, -1, -1};
#pragma unroll
    for (int j = 0; j < 4; ++j) zero(bc[j]);

    for (int a = 0; a < nact; a += U) {
        float d[U][4];
        C c[U][4];
        int idx[U];
        bool live[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            idx[u] = (a + u < nact) ? act[a + u] : -1;
            live[u] = false;
            if (idx[u] >= 0) {
                const SrcDesc& s = at(a + u, idx[u]);
                live[u] = y >= s.y0 && y < s.y1 && x + 4 > s.x0 && x < s.x1;
                if (live[u]) load4<CB>(s, x, y, d[u], c[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!live[u]) continue;
            const SrcDesc& s = at(a + u, idx[u]);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int xj = x + j;
                // strict '<': ties keep the earlier (lower-index) winner or the
                // background; NaN never compares less
                if (xj >= s.x0 && xj < s.x1 && d[u][j] < bd[j]) {
                    bd[j] = d[u][j];
                    bc[j] = c[u][j];
                    bi[j] = idx[u];
                }
            }
        }
    }

    const size_t o = (size_t)y * (size_t)D.pitch + (size_t)x;
    C* oc = reinterpret_cast<C*>(D.color) + o;
    if (D.vec && x + 4 <= D.W) {
        if constexpr (CB == 4) st_stream(reinterpret_cast<uint4*>(oc), make_uint4(bc[0], bc[1], bc[2], bc[3]));
        else {
#pragma unroll
            for (int j = 0; j < 4; ++j) st_stream(oc + j, bc[j]);
        }
        if (D.depth) st_stream(reinterpret_cast<float4*>(D.depth + o), make_float4(bd[0], bd[1], bd[2], bd[3]));
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (x + j < D.W) {
                oc[j] = bc[j];
                if (D.depth) D.depth[o + j] = bd[j];
            }
        }
    }
    if (D.winner) {
        int16_t* w = D.winner + (size_t)y * D.W + x;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (x + j < D.W) w[j] = (int16_t)bi[j];
    }
}

// ----------------------------------------------------------------- alpha ---

__device__ __forceinline__ float4 half4_to_float4(uint2 v)
{
    const __half2 lo = *reinterpret_cast<const __half2*>(&v.x);
    const __half2 hi = *reinterpret_cast<const __half2*>(&v.y);
    const float2 a = __half22float2(lo), b = __half22float2(hi);
    return make_float4(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ uint2 float4_to_half4(float4 f)
{
    const __half2 lo = __floats2half2_rn(f.x, f.y);
    const __half2 hi = __floats2half2_rn(f.z, f.w);
    uint2 v;
    v.x = *reinterpret_cast<const uint32_t*>(&lo);
    v.y = *reinterpret_cast<const uint32_t*>(&hi);
    return v;
}

// Raw 16 bytes of one premultiplied layer at the thread's pixels (1 RGBA32F or
// 2 RGBA16F pixels), zero outside the layer's ROI on the per-pixel path.
template <bool F16>
__device__ __forceinline__ uint4 load_raw(const SrcDesc& s, int x, int y)
{
    const size_t e = (size_t)(y - s.oy) * (size_t)s.pitch + (size_t)(x - s.ox);
    if constexpr (!F16) {
        const uint4* p = reinterpret_cast<const uint4*>(s.color) + e;
        if (s.vec) return ld_stream(p);
        const unsigned int* f = reinterpret_cast<const unsigned int*>(p);
        return make_uint4(__ldcs(f), __ldcs(f + 1), __ldcs(f + 2), __ldcs(f + 3));
    } else {
        const uint2* p = reinterpret_cast<const uint2*>(s.color) + e;
        if (s.vec) return ld_stream(reinterpret_cast<const uint4*>(p));
        uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int xj = x + j;
            if (xj >= s.x0 && xj < s.x1) {
                const unsigned short* h = reinterpret_cast<const unsigned short*>(p + j);
                w[2 * j] = (uint32_t)__ldcs(h) | ((uint32_t)__ldcs(h + 1) << 16);
                w[2 * j + 1] = (uint32_t)__ldcs(h + 2) | ((uint32_t)__ldcs(h + 3) << 16);
            }
        }
        return make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Pixel j of a raw 16-byte word as float RGBA.
template <bool F16>
__device__ __forceinline__ float4 pixel_of(const uint4& v, int j)
{
    if constexpr (!F16) {
        return make_float4(__uint_as_float(v.x), __uint_as_float(v.y), __uint_as_float(v.z),
                           __uint_as_float(v.w));
    } else {
        return j == 0 ? half4_to_float4(make_uint2(v.x, v.y)) : half4_to_float4(make_uint2(v.z, v.w));
    }
}

// Front-to-back "over" of the active layers at the thread's PX pixels, U
// layers' loads in flight per thread.  full (uniform over the CTA): every
// active layer's ROI covers the CTA's whole tile, so the per-layer and
// per-pixel range tests are skipped (pixels past the frame's right edge are
// computed but never stored).
template <bool F16, class At, int U = 8>
__device__ __forceinline__ void alpha_px(At at, const int16_t* act, int nact, int x, int y,
                                         const DstDesc& D, bool full = false)
{
    constexpr int PX = F16 ? 2 : 1;      // pixels per 16 bytes
    float4 acc[PX];
    float T[PX];
#pragma unroll
    for (int j = 0; j < PX; ++j) { acc[j] = make_float4(0.f, 0.f, 0.f, 0.f); T[j] = 1.0f; }

    for (int a = 0; a < nact; a += U) {
        uint4 raw[U];
        bool live[U];
        int idx[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            idx[u] = (a + u < nact) ? act[a + u] : -1;
            live[u] = false;
            if (idx[u] >= 0) {
                const SrcDesc& s = at(a + u, idx[u]);
                live[u] = full || (y >= s.y0 && y < s.y1 && x + PX > s.x0 && x < s.x1);
                if (live[u]) raw[u] = load_raw<F16>(s, x, y);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!live[u]) continue;
            const SrcDesc& s = at(a + u, idx[u]);
#pragma unroll
            for (int j = 0; j < PX; ++j) {
                const int xj = x + j;
                if (!full && (xj < s.x0 || xj >= s.x1)) continue;   // transparent outside the ROI
                const float4 c = pixel_of<F16>(raw[u], j);
                // C += T c (premultiplied, all four channels); T *= (1 - a)
                acc[j].x = fmaf(T[j], c.x, acc[j].x);
                acc[j].y = fmaf(T[j], c.y, acc[j].y);
                acc[j].z = fmaf(T[j], c.z, acc[j].z);
                acc[j].w = fmaf(T[j], c.w, acc[j].w);
                T[j] = fmaf(-T[j], c.w, T[j]);
            }
        }
    }

    const size_t o = (size_t)y * (size_t)D.pitch + (size_t)x;
    if constexpr (!F16) {
        float4* op = reinterpret_cast<float4*>(D.color) + o;
        if (D.vec) st_stream(op, acc[0]);
        else { float* f = reinterpret_cast<float*>(op); f[0] = acc[0].x; f[1] = acc[0].y; f[2] = acc[0].z; f[3] = acc[0].w; }
    } else {
        uint2* op = reinterpret_cast<uint2*>(D.color) + o;
        const uint2 h0 = float4_to_half4(acc[0]), h1 = float4_to_half4(acc[1]);
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
    }
    if (D.tfinal) {
        float* t = D.tfinal + (size_t)y * D.W + x;
#pragma unroll
        for (int j = 0; j < PX; ++j)
            if (x + j < D.W) t[j] = T[j];
    }
}

}  // namespace ec
