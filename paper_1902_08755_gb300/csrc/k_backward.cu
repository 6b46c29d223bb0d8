// k_backward.cu -- gradients of the compositing operators for sm_103a.
//
// Ordered compositing (thesis 5.2.1) is differentiated through its front-to-
// back recurrence C += T c_k, T *= (1 - a_k):
//   dL/dc_k^{RGB} = g^{RGB} T_k,   dL/da_k = T_k (g^A - R_k),
//   R_{n-1} = 0,  R_{k-1} = g.c_k + (1 - a_k) R_k      (reverse "behind" scan).
// Nothing per layer is kept from the forward.  A CTA owns a tile of 32 lanes
// by 16 or 32 rows, one pixel per lane (the kernel also takes two adjacent pixels
// per lane, read and written as one 16-byte word, with segments of at most 4
// layers); its warps split the tile's layer stack into contiguous segments of
// at most 8 layers.  A warp loads its layers'
// pixels straight into registers (zero outside a layer's ROI, which is
// exactly a transparent layer), runs its segment's forward, and keeps per
// layer only T', g.c and a.  Both recurrences split exactly across segments:
//   forward  T_k = T_start(s) * T'_k, T'_k the transmittance inside segment s,
//            T_start(s) = prod over earlier segments of P_u = prod (1 - a);
//   reverse  R entering segment s from behind = sum_{t>s} A_t prod_{s<u<t} P_u
//            with A_t = sum_{j in t} T'_j (g.c_j), evaluated Horner-style,
// so after one exchange of (P, A) through shared memory every warp runs the
// exact reverse recurrence over its own layers and writes their gradients.
// Layers are read from HBM once; per-layer tile records (addresses, clipped
// ranges) are built once per CTA in shared memory and read as broadcasts.
// Tiles that every active layer covers, inside the frame, with whole-pixel
// vector access and one pitch ("lean" tiles, the usual case) run a row pass
// without range tests; for FP16 layers that pass is software-pipelined (the
// next row's loads in flight behind the exchange, the row's per-layer state
// parked in shared memory).
//
// The fused variant takes the loss weights w up front (L = sum w * out, so
// the upstream gradient is w) and also writes out and T_final; the output is
// composed from the segments' partials by (pixel, channel) lanes.
//
// Depth compositing (thesis 5.2.1) copies the winner's colour, so its
// gradient routes grad_out to the winning input and writes zero elsewhere.
#include <algorithm>
#include <type_traits>

#include "ec_internal.cuh"

namespace ec {
namespace {

constexpr int kRows = 16;         // rows per alpha-backward CTA (stacks of up to 64 layers)
constexpr int kRowsDeep = 32;     // rows per CTA for deeper stacks (their per-CTA setup is larger)
constexpr int kMaxWarps = 32;     // segments (warps) per CTA
static_assert(8 * kMaxWarps >= kMaxBwdLayers, "every stack fits one CTA");

__device__ __forceinline__ float4 h4_to_f4(uint2 v)
{
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
    return make_float4(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ uint2 f4_to_h4(float4 f)
{
    const __half2 lo = __floats2half2_rn(f.x, f.y), hi = __floats2half2_rn(f.z, f.w);
    uint2 v;
    v.x = *reinterpret_cast<const uint32_t*>(&lo);
    v.y = *reinterpret_cast<const uint32_t*>(&hi);
    return v;
}

// What a CTA needs of one layer for its tile (TW columns by ROWS rows),
// built once per CTA: addresses of pixel (tx0, ty0) in the colour and
// gradient buffers (offset only by rows and columns that lie inside the ROI /
// pvp before use), the pitch, the ROI and gradient ranges (columns relative
// to tx0), the colour alignment class, and whether pixel pairs starting at an
// even column may be read (wide) or their gradients written (gwide) as one
// 16-byte word.
struct BandTile {
    uintptr_t src;
    uintptr_t grad;
    int32_t pitch;
    int32_t ry0, ry1, gy0, gy1;
    int16_t rx0, rx1, gx0, gx1;
    int8_t cls, gvec, wide, gwide;
};
static_assert(sizeof(BandTile) == 48, "tile record");

template <bool F16, bool G16, int TW>
__device__ __forceinline__ BandTile make_band_tile(const BwdDesc& d, int tx0, int ty0)
{
    constexpr int S = F16 ? 8 : 16, GS = G16 ? 8 : 16;
    BandTile t;
    const int64_t e = (int64_t)(ty0 - d.oy) * d.pitch + (int64_t)(tx0 - d.ox);
    t.src = reinterpret_cast<uintptr_t>(d.color) + (uintptr_t)(e * S);
    t.grad = reinterpret_cast<uintptr_t>(d.grad) + (uintptr_t)(e * GS);
    t.pitch = d.pitch;
    t.ry0 = d.y0; t.ry1 = d.y1;
    t.gy0 = d.gy0; t.gy1 = d.gy1;
    t.rx0 = (int16_t)max(min(d.x0 - tx0, TW), 0);
    t.rx1 = (int16_t)max(min(d.x1 - tx0, TW), 0);
    t.gx0 = (int16_t)max(min(d.gx0 - tx0, TW), 0);
    t.gx1 = (int16_t)max(min(d.gx1 - tx0, TW), 0);
    t.cls = (int8_t)d.cls;
    t.gvec = (int8_t)d.gvec;
    const bool even = (d.pitch & 1) == 0;
    t.wide = (int8_t)(F16 && even && d.cls >= 8 && (t.src & 15u) == 0);
    t.gwide = (int8_t)(G16 && even && d.gvec && (t.grad & 15u) == 0);
    return t;
}

// One pixel of a layer as stored (FP16: 8 bytes, FP32: 16), read with the
// widest loads its alignment class allows.
template <bool F16> struct Px;
template <> struct Px<true> { using T = uint2; };
template <> struct Px<false> { using T = float4; };

__device__ __forceinline__ uint2 load_px16(uintptr_t a, int cls)
{
    if (cls >= 8) return __ldcs(reinterpret_cast<const uint2*>(a));
    if (cls >= 4) {
        const uint32_t* p = reinterpret_cast<const uint32_t*>(a);
        return make_uint2(__ldcs(p), __ldcs(p + 1));
    }
    const unsigned short* h = reinterpret_cast<const unsigned short*>(a);
    return make_uint2((uint32_t)__ldcs(h) | ((uint32_t)__ldcs(h + 1) << 16),
                      (uint32_t)__ldcs(h + 2) | ((uint32_t)__ldcs(h + 3) << 16));
}

__device__ __forceinline__ float4 load_px32(uintptr_t a, int cls)
{
    if (cls >= 16) return __ldcs(reinterpret_cast<const float4*>(a));
    const float* f = reinterpret_cast<const float*>(a);
    return make_float4(__ldcs(f), __ldcs(f + 1), __ldcs(f + 2), __ldcs(f + 3));
}

template <bool G16>
__device__ __forceinline__ void store_grad_at(uintptr_t addr, bool vec, float4 v)
{
    if constexpr (G16) {
        uint2* p = reinterpret_cast<uint2*>(addr);
        const uint2 h = f4_to_h4(v);
        if (vec) __stcs(p, h);
        else {
            unsigned short* s = reinterpret_cast<unsigned short*>(p);
            s[0] = (unsigned short)h.x; s[1] = (unsigned short)(h.x >> 16);
            s[2] = (unsigned short)h.y; s[3] = (unsigned short)(h.y >> 16);
        }
    } else {
        float4* p = reinterpret_cast<float4*>(addr);
        if (vec) __stcs(p, v);
        else { float* f = reinterpret_cast<float*>(p); f[0] = v.x; f[1] = v.y; f[2] = v.z; f[3] = v.w; }
    }
}

template <bool G16>
__device__ __forceinline__ void store_grad(const BwdDesc& d, int x, int y, float4 v)
{
    const size_t e = (size_t)(y - d.oy) * (size_t)d.pitch + (size_t)(x - d.ox);
    const uintptr_t a = reinterpret_cast<uintptr_t>(d.grad) + e * (G16 ? 8 : 16);
    store_grad_at<G16>(a, d.gvec != 0, v);
}

// Alpha backward (and fused forward + backward) for one tile of 32 * PX
// pixels (PX per lane, adjacent) by ROWS rows.  blockDim.x = 32 * NS: warp s
// owns segment s of the tile's active layers, at most MS of them.  Tiles that
// every active layer covers entirely (ROI and gradient rectangle) skip the
// per-row range checks; lean tiles (also aligned, one pitch, inside the
// frame) take the row passes without any tests.
template <int N, bool F16, bool G16, bool FUSED, int PX, int MS, int ROWS>
__global__ void __launch_bounds__(32 * kMaxWarps, 1)
k_alpha_bwd(const __grid_constant__ BwdList<N> L, const __grid_constant__ DstDesc D,
            const float4* __restrict__ g, int cap)
{
    constexpr int S = F16 ? 8 : 16, GS = G16 ? 8 : 16, TW = 32 * PX;
    using RawPx = typename Px<F16>::T;
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int16_t act[N];
    __shared__ int nact_s;
    BandTile* tiles = reinterpret_cast<BandTile*>(smem);                    // [cap]
    const int NS = (int)(blockDim.x / 32);
    // per row parity, segment and pixel: [2][NS][PX][32], pixel (lane, q) at
    // q * 32 + lane.  Rows alternate between the two copies, so a row's writes
    // never meet the previous row's reads and one barrier per row suffices.
    float* const Ps0 = reinterpret_cast<float*>(smem + (size_t)cap * sizeof(BandTile));
    float* const As0 = Ps0 + 2 * NS * TW;
    float4* const Cs0 = reinterpret_cast<float4*>(As0 + 2 * NS * TW);       // (fused)
    // FP16 lean tiles: each warp's per-layer state of its row, [MS][32] per
    // warp -- (T', g.c) as floats and a as the half it was read as (exact) --
    // so that the registers can hold the next row's loads
    float2* const St0 = reinterpret_cast<float2*>(Cs0 + (FUSED ? 2 * NS * TW : 0));
    float2* const St = St0 + (threadIdx.x / 32) * MS * 32;
    unsigned short* const Sa = reinterpret_cast<unsigned short*>(St0 + NS * MS * 32) + (threadIdx.x / 32) * MS * 32;

    const int lane = threadIdx.x & 31, sg = threadIdx.x / 32;
    const int tx0 = blockIdx.x * TW, ty0 = blockIdx.y * ROWS;
    const int tx1 = min(tx0 + TW, D.W), ty1 = min(ty0 + ROWS, D.H);

    // layers whose gradient rectangle meets the tile, in compositing order
    if (threadIdx.x < 32) {
        int base = 0;
        for (int i0 = 0; i0 < L.n; i0 += 32) {
            const int i = i0 + lane;
            bool hit = false;
            if (i < L.n) {
                const BwdDesc& d = L.d[i];
                hit = d.gx0 < tx1 && d.gx1 > tx0 && d.gy0 < ty1 && d.gy1 > ty0;
            }
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (hit) act[base + __popc(m & ((1u << lane) - 1u))] = (int16_t)i;
            base += __popc(m);
        }
        if (lane == 0) nact_s = base;
    }
    __syncthreads();
    const int nact = nact_s;
    const int pitch0 = nact > 0 ? L.d[act[0]].pitch : 0;
    bool covers = true, lean = true;
    for (int k = threadIdx.x; k < nact; k += blockDim.x) {
        const BwdDesc& dk = L.d[act[k]];
        const BandTile t = make_band_tile<F16, G16, TW>(dk, tx0, ty0);
        tiles[k] = t;
        covers = covers && t.rx0 == 0 && t.rx1 >= tx1 - tx0 && t.ry0 <= ty0 && t.ry1 >= ty1 &&
                 t.gx0 == 0 && t.gx1 >= tx1 - tx0 && t.gy0 <= ty0 && t.gy1 >= ty1;
        lean = lean && dk.pitch == pitch0 && dk.cls >= S && dk.gvec;
    }
    const bool full = __syncthreads_and(covers);
    // lean tiles: every active layer covers the whole tile, which lies inside
    // the frame, with whole-pixel vector loads and stores and one pitch, so a
    // row's addresses are one offset from the tile records
    const bool lean_all = __syncthreads_and(covers && lean);
    const bool fast = PX == 1 && tx0 + TW <= D.W && lean_all;

    const int k0 = (sg * nact) / NS, cnt = ((sg + 1) * nact) / NS - k0;   // cnt <= MS
    const int c0 = PX * lane;                                              // first column of this lane
    bool valid[PX];
#pragma unroll
    for (int q = 0; q < PX; ++q) valid[q] = tx0 + c0 + q < D.W;

    // Fused output of row y: out = sum over segments u of Tstart(u) C_u,
    // evaluated front to back.  Lane (pixel, channel) of the first warps takes
    // one channel of one pixel (TW * 4 of them), so no single warp carries the
    // whole composite; T_final is the running product after the last segment.
    auto composite_row = [&](int y, const float* Ps, const float4* Cs) {
        for (int i = threadIdx.x; i < 4 * TW; i += blockDim.x) {
            const int idx = i >> 2, ch = i & 3;
            const int x = tx0 + PX * (idx & 31) + (idx >> 5);
            if (x >= D.W) continue;
            float Tacc = 1.0f, o = 0.0f;
#pragma unroll 4
            for (int u = 0; u < NS; ++u) {
                o = fmaf(Tacc, reinterpret_cast<const float*>(Cs + u * TW + idx)[ch], o);
                Tacc *= Ps[u * TW + idx];
            }
            const size_t e = ((size_t)y * (size_t)D.pitch + (size_t)x) * 4 + ch;
            if constexpr (F16) reinterpret_cast<__half*>(D.color)[e] = __float2half_rn(o);
            else reinterpret_cast<float*>(D.color)[e] = o;
            if (ch == 0 && D.tfinal) D.tfinal[(size_t)y * D.W + x] = Tacc;
        }
    };

    // Row pass of a lean tile (one pixel per lane): no range or alignment
    // tests, one row offset for every layer's load and gradient store.
    auto row_fast = [&](int y) {
        float* const Ps = Ps0 + (y & 1) * NS * TW;
        float* const As = As0 + (y & 1) * NS * TW;
        float4* const Cs = Cs0 + (y & 1) * NS * TW;
        const float4 gp = __ldcs(g + (size_t)y * D.W + tx0 + lane);
        const int64_t r = (int64_t)(y - ty0) * pitch0 + lane;
        RawPx raw[MS];
#pragma unroll
        for (int j = 0; j < MS; ++j) {
            if constexpr (F16) raw[j] = make_uint2(0u, 0u);
            else raw[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (j < cnt) {
                const uintptr_t a = tiles[k0 + j].src + (uintptr_t)(r * S);
                if constexpr (F16) raw[j] = __ldcs(reinterpret_cast<const uint2*>(a));
                else raw[j] = __ldcs(reinterpret_cast<const float4*>(a));
            }
        }
        float Tl[MS], gcl[MS], al[MS];
        float Tp = 1.0f, A = 0.0f;
        float4 Cl = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int j = 0; j < MS; ++j) {
            float4 c;
            if constexpr (F16) c = h4_to_f4(raw[j]);
            else c = raw[j];
            const float gc = fmaf(gp.x, c.x, fmaf(gp.y, c.y, fmaf(gp.z, c.z, gp.w * c.w)));
            Tl[j] = Tp;
            gcl[j] = gc;
            al[j] = c.w;
            if (j < cnt) {
                if (FUSED) {
                    Cl.x = fmaf(Tp, c.x, Cl.x);
                    Cl.y = fmaf(Tp, c.y, Cl.y);
                    Cl.z = fmaf(Tp, c.z, Cl.z);
                    Cl.w = fmaf(Tp, c.w, Cl.w);
                }
                A = fmaf(Tp, gc, A);
                Tp = fmaf(-Tp, c.w, Tp);
            }
        }
        Ps[sg * TW + lane] = Tp;
        As[sg * TW + lane] = A;
        if (FUSED) Cs[sg * TW + lane] = Cl;
        __syncthreads();

        float Tstart = 1.0f, R = 0.0f;
        for (int u = 0; u < sg; ++u) Tstart *= Ps[u * TW + lane];
        for (int u = NS - 1; u > sg; --u) R = fmaf(Ps[u * TW + lane], R, As[u * TW + lane]);
        if (FUSED) composite_row(y, Ps, Cs);

#pragma unroll
        for (int j = MS - 1; j >= 0; --j) {
            if (j < cnt) {
                const float Tk = Tstart * Tl[j];
                const float4 gr = make_float4(gp.x * Tk, gp.y * Tk, gp.z * Tk, Tk * (gp.w - R));
                const uintptr_t ga = tiles[k0 + j].grad + (uintptr_t)(r * GS);
                store_grad_at<G16>(ga, true, gr);
                R = fmaf(1.0f - al[j], R, gcl[j]);
            }
        }
    };

    // FP16 lean tiles, software-pipelined: the next row's layers and upstream
    // gradient are loaded while this row's exchange and reverse scan run.
    // The per-layer state lives in shared memory (St) meanwhile.
    auto rows_fast16 = [&]() {
        RawPx raw[MS];
        float4 gn;
        auto load_row = [&](int y) {
            const int64_t r = (int64_t)(y - ty0) * pitch0 + lane;
            gn = __ldcs(g + (size_t)y * D.W + tx0 + lane);
#pragma unroll
            for (int j = 0; j < MS; ++j) {
                if constexpr (F16) raw[j] = make_uint2(0u, 0u);
                else raw[j] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (j < cnt) {
                    const uintptr_t a = tiles[k0 + j].src + (uintptr_t)(r * S);
                    if constexpr (F16) raw[j] = __ldcs(reinterpret_cast<const uint2*>(a));
                    else raw[j] = __ldcs(reinterpret_cast<const float4*>(a));
                }
            }
        };
        load_row(ty0);
        for (int y = ty0; y < ty1; ++y) {
            float* const Ps = Ps0 + (y & 1) * NS * TW;
            float* const As = As0 + (y & 1) * NS * TW;
            float4* const Cs = Cs0 + (y & 1) * NS * TW;
            const float4 gp = gn;
            float Tp = 1.0f, A = 0.0f;
            float4 Cl = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int j = 0; j < MS; ++j) {
                float4 c;
                if constexpr (F16) c = h4_to_f4(raw[j]);
                else c = raw[j];
                const float gc = fmaf(gp.x, c.x, fmaf(gp.y, c.y, fmaf(gp.z, c.z, gp.w * c.w)));
                St[j * 32 + lane] = make_float2(Tp, gc);
                if constexpr (F16) Sa[j * 32 + lane] = (unsigned short)(raw[j].y >> 16);
                if (j < cnt) {
                    if (FUSED) {
                        Cl.x = fmaf(Tp, c.x, Cl.x);
                        Cl.y = fmaf(Tp, c.y, Cl.y);
                        Cl.z = fmaf(Tp, c.z, Cl.z);
                        Cl.w = fmaf(Tp, c.w, Cl.w);
                    }
                    A = fmaf(Tp, gc, A);
                    Tp = fmaf(-Tp, c.w, Tp);
                }
            }
            Ps[sg * TW + lane] = Tp;
            As[sg * TW + lane] = A;
            if (FUSED) Cs[sg * TW + lane] = Cl;
            __syncthreads();
            if (y + 1 < ty1) load_row(y + 1);

            float Tstart = 1.0f, R = 0.0f;
            for (int u = 0; u < sg; ++u) Tstart *= Ps[u * TW + lane];
            for (int u = NS - 1; u > sg; --u) R = fmaf(Ps[u * TW + lane], R, As[u * TW + lane]);
            if (FUSED) composite_row(y, Ps, Cs);

            const int64_t r = (int64_t)(y - ty0) * pitch0 + lane;
#pragma unroll
            for (int j = MS - 1; j >= 0; --j) {
                if (j < cnt) {
                    const float2 st = St[j * 32 + lane];
                    const float a = __half2float(__ushort_as_half(Sa[j * 32 + lane]));
                    const float Tk = Tstart * st.x;
                    const float4 gr = make_float4(gp.x * Tk, gp.y * Tk, gp.z * Tk, Tk * (gp.w - R));
                    const uintptr_t ga = tiles[k0 + j].grad + (uintptr_t)(r * GS);
                    store_grad_at<G16>(ga, true, gr);
                    R = fmaf(1.0f - a, R, st.y);
                }
            }
        }
    };

    auto row_pass = [&](auto full_c, int y) {
        constexpr bool FULL = decltype(full_c)::value;
        float* const Ps = Ps0 + (y & 1) * NS * TW;
        float* const As = As0 + (y & 1) * NS * TW;
        float4* const Cs = Cs0 + (y & 1) * NS * TW;
        float4 gp[PX];
#pragma unroll
        for (int q = 0; q < PX; ++q)
            gp[q] = valid[q] ? __ldcs(g + (size_t)y * D.W + tx0 + c0 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        // this segment's pixels, all loads in flight before any is used
        RawPx raw[MS][PX];
#pragma unroll
        for (int j = 0; j < MS; ++j) {
#pragma unroll
            for (int q = 0; q < PX; ++q) {
                if constexpr (F16) raw[j][q] = make_uint2(0u, 0u);
                else raw[j][q] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            if (j < cnt) {
                const BandTile& t = tiles[k0 + j];
                if (FULL || (y >= t.ry0 && y < t.ry1)) {
                    const uintptr_t a = t.src + (uintptr_t)(((int64_t)(y - ty0) * t.pitch + c0) * S);
                    bool in[PX];
#pragma unroll
                    for (int q = 0; q < PX; ++q)
                        in[q] = valid[q] && (FULL || (c0 + q >= t.rx0 && c0 + q < t.rx1));
                    bool done = false;
                    if constexpr (PX == 2) {
                        if (t.wide && in[0] && in[1]) {
                            const uint4 v = __ldcs(reinterpret_cast<const uint4*>(a));
                            raw[j][0] = make_uint2(v.x, v.y);
                            raw[j][1] = make_uint2(v.z, v.w);
                            done = true;
                        }
                    }
                    if (!done) {
#pragma unroll
                        for (int q = 0; q < PX; ++q) {
                            if (!in[q]) continue;
                            if constexpr (F16) raw[j][q] = load_px16(a + q * S, t.cls);
                            else raw[j][q] = load_px32(a + q * S, t.cls);
                        }
                    }
                }
            }
        }
        // local forward; keep T', g.c and a per layer and pixel
        float Tl[MS][PX], gcl[MS][PX], al[MS][PX];
        float Tp[PX], A[PX];
        float4 Cl[PX];
#pragma unroll
        for (int q = 0; q < PX; ++q) { Tp[q] = 1.0f; A[q] = 0.0f; Cl[q] = make_float4(0.f, 0.f, 0.f, 0.f); }
#pragma unroll
        for (int j = 0; j < MS; ++j) {
#pragma unroll
            for (int q = 0; q < PX; ++q) {
                float4 c;
                if constexpr (F16) c = h4_to_f4(raw[j][q]);
                else c = raw[j][q];
                const float gc = fmaf(gp[q].x, c.x, fmaf(gp[q].y, c.y, fmaf(gp[q].z, c.z, gp[q].w * c.w)));
                Tl[j][q] = Tp[q];
                gcl[j][q] = gc;
                al[j][q] = c.w;
                if (j < cnt) {
                    if (FUSED) {
                        Cl[q].x = fmaf(Tp[q], c.x, Cl[q].x);
                        Cl[q].y = fmaf(Tp[q], c.y, Cl[q].y);
                        Cl[q].z = fmaf(Tp[q], c.z, Cl[q].z);
                        Cl[q].w = fmaf(Tp[q], c.w, Cl[q].w);
                    }
                    A[q] = fmaf(Tp[q], gc, A[q]);
                    Tp[q] = fmaf(-Tp[q], c.w, Tp[q]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < PX; ++q) {
            Ps[sg * TW + q * 32 + lane] = Tp[q];
            As[sg * TW + q * 32 + lane] = A[q];
            if (FUSED) Cs[sg * TW + q * 32 + lane] = Cl[q];
        }
        __syncthreads();

        float Tstart[PX], R[PX];
#pragma unroll
        for (int q = 0; q < PX; ++q) {
            Tstart[q] = 1.0f;
            for (int u = 0; u < sg; ++u) Tstart[q] *= Ps[u * TW + q * 32 + lane];
            R[q] = 0.0f;
            for (int u = NS - 1; u > sg; --u) R[q] = fmaf(Ps[u * TW + q * 32 + lane], R[q], As[u * TW + q * 32 + lane]);
        }

        if (FUSED) composite_row(y, Ps, Cs);

        // reverse over this segment, entering with the R of the layers behind it
#pragma unroll
        for (int j = MS - 1; j >= 0; --j) {
            if (j < cnt) {
                const BandTile& t = tiles[k0 + j];
                if (FULL || (y >= t.gy0 && y < t.gy1)) {
                    const bool rrow = FULL || (y >= t.ry0 && y < t.ry1);
                    float4 gr[PX];
                    bool gin[PX];
#pragma unroll
                    for (int q = 0; q < PX; ++q) {
                        const int c = c0 + q;
                        gin[q] = valid[q] && (FULL || (c >= t.gx0 && c < t.gx1));
                        const float Tk = Tstart[q] * Tl[j][q];
                        const bool in = FULL || (rrow && c >= t.rx0 && c < t.rx1);
                        gr[q] = in ? make_float4(gp[q].x * Tk, gp[q].y * Tk, gp[q].z * Tk, Tk * (gp[q].w - R[q]))
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                    const uintptr_t ga = t.grad + (uintptr_t)(((int64_t)(y - ty0) * t.pitch + c0) * GS);
                    bool done = false;
                    if constexpr (PX == 2 && G16) {
                        if (t.gwide && gin[0] && gin[1]) {
                            const uint2 h0 = f4_to_h4(gr[0]), h1 = f4_to_h4(gr[1]);
                            __stcs(reinterpret_cast<uint4*>(ga), make_uint4(h0.x, h0.y, h1.x, h1.y));
                            done = true;
                        }
                    }
                    if (!done) {
#pragma unroll
                        for (int q = 0; q < PX; ++q)
                            if (gin[q]) store_grad_at<G16>(ga + q * GS, t.gvec != 0, gr[q]);
                    }
                }
#pragma unroll
                for (int q = 0; q < PX; ++q) R[q] = fmaf(1.0f - al[j][q], R[q], gcl[j][q]);
            }
        }
    };
    if (fast) {
        if constexpr (F16) rows_fast16();
        else for (int y = ty0; y < ty1; ++y) row_fast(y);
    } else if (full) {
        for (int y = ty0; y < ty1; ++y) row_pass(std::true_type{}, y);
    } else {
        for (int y = ty0; y < ty1; ++y) row_pass(std::false_type{}, y);
    }
}

// ----------------------------------------------------------- depth grad ---

template <int N>
__global__ void __launch_bounds__(256)
k_depth_bwd(const __grid_constant__ BwdList<N> L, int W, int H, const int16_t* __restrict__ winner,
            const float4* __restrict__ g)
{
    __shared__ int16_t act[N];
    __shared__ int nact_s;
    const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
    const int tx0 = blockIdx.x * 128, ty0 = blockIdx.y * 8;
    const int tx1 = min(tx0 + 128, W), ty1 = min(ty0 + 8, H);
    if (threadIdx.x < 32) {
        int base = 0;
        for (int i0 = 0; i0 < L.n; i0 += 32) {
            const int i = i0 + lane;
            bool hit = false;
            if (i < L.n) {
                const BwdDesc& d = L.d[i];
                hit = d.gx0 < tx1 && d.gx1 > tx0 && d.gy0 < ty1 && d.gy1 > ty0;
            }
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (hit) act[base + __popc(m & ((1u << lane) - 1u))] = (int16_t)i;
            base += __popc(m);
        }
        if (lane == 0) nact_s = base;
    }
    __syncthreads();
    const int nact = nact_s;
    const int x = tx0 + lane * 4, y = ty0 + row;
    if (x >= W || y >= H) return;
    int win[4];
    float4 gv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const bool ok = x + j < W;
        win[j] = ok ? winner[(size_t)y * W + x + j] : -2;
        gv[j] = ok ? __ldcs(g + (size_t)y * W + x + j) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int a = 0; a < nact; ++a) {
        const int i = act[a];
        const BwdDesc& d = L.d[i];
        if (y < d.gy0 || y >= d.gy1) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int xj = x + j;
            if (xj < d.gx0 || xj >= d.gx1) continue;
            const float4 v = win[j] == i ? gv[j] : make_float4(0.f, 0.f, 0.f, 0.f);
            store_grad<false>(d, xj, y, v);
        }
    }
}

template <int N>
BwdList<N> make_bwd(const BwdDesc* d, int n)
{
    BwdList<N> L;
    L.n = n;
    L.pad[0] = L.pad[1] = L.pad[2] = 0;
    for (int i = 0; i < n; ++i) L.d[i] = d[i];
    return L;
}

// Warps (segments) per alpha-backward CTA for a stack of n layers: enough for
// ms layers each, and at least four (or n) so that short stacks still split
// their scans.
int alpha_bwd_warps(int n, int ms)
{
    const int need = (n + ms - 1) / ms;
    return std::max(1, std::min(kMaxWarps, std::max(need, std::min(n, 4))));
}

template <int N, bool F16, bool G16, bool FUSED, int PX, int MS, int ROWS>
cudaError_t alpha_bwd_n(const BwdDesc* d, int n, const DstDesc& D, const float4* g, cudaStream_t s)
{
    const int ns = alpha_bwd_warps(n, MS), cap = std::max(n, 1), tw = 32 * PX;
    const size_t smem = (size_t)cap * sizeof(BandTile) + 2 * (size_t)ns * tw * (8 + (FUSED ? 16 : 0)) +
                        (F16 ? (size_t)ns * MS * 32 * (sizeof(float2) + sizeof(unsigned short)) : 0);
    auto kern = k_alpha_bwd<N, F16, G16, FUSED, PX, MS, ROWS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid(ceil_div(D.W, tw), ceil_div(D.H, ROWS));
    kern<<<grid, 32 * ns, smem, s>>>(make_bwd<N>(d, n), D, g, cap);
    return cudaGetLastError();
}

// One pixel per lane and eight layers per warp, FP32 and FP16 alike (two FP16
// pixels per lane with four layers per warp was 1.5% slower on 32 x 2048^2; the
// kernel keeps the two-pixel form for other tile choices); 16 rows per CTA, 32
// for stacks deeper than 64 layers (128 x 3840x2160 FP16: 3.74 ms instead of
// 3.87; on 32 x 2048^2 32 rows were 2-3% slower).
template <int N, bool F16, bool G16, bool FUSED>
cudaError_t alpha_bwd_px(const BwdDesc* d, int n, const DstDesc& D, const float4* g, cudaStream_t s)
{
    if (n > 64) return alpha_bwd_n<N, F16, G16, FUSED, 1, 8, kRowsDeep>(d, n, D, g, s);
    return alpha_bwd_n<N, F16, G16, FUSED, 1, 8, kRows>(d, n, D, g, s);
}

template <int N>
cudaError_t alpha_bwd_dispatch(const BwdDesc* d, int n, bool f16, bool g16, bool fused,
                               const DstDesc& D, const float4* g, cudaStream_t s)
{
    if (f16) {
        if (g16) return fused ? alpha_bwd_px<N, true, true, true>(d, n, D, g, s)
                              : alpha_bwd_px<N, true, true, false>(d, n, D, g, s);
        return fused ? alpha_bwd_px<N, true, false, true>(d, n, D, g, s)
                     : alpha_bwd_px<N, true, false, false>(d, n, D, g, s);
    }
    if (g16) return fused ? alpha_bwd_px<N, false, true, true>(d, n, D, g, s)
                          : alpha_bwd_px<N, false, true, false>(d, n, D, g, s);
    return fused ? alpha_bwd_px<N, false, false, true>(d, n, D, g, s)
                 : alpha_bwd_px<N, false, false, false>(d, n, D, g, s);
}

}  // namespace

cudaError_t launch_alpha_bwd(const BwdDesc* d, int n, bool f16, bool g16, bool fused,
                             const DstDesc& D, const float* g, cudaStream_t s)
{
    if (D.W <= 0 || D.H <= 0) return cudaSuccess;
    if (n > kMaxBwdLayers) return cudaErrorInvalidValue;
    const float4* g4 = reinterpret_cast<const float4*>(g);
    if (n <= 16) return alpha_bwd_dispatch<16>(d, n, f16, g16, fused, D, g4, s);
    if (n <= 64) return alpha_bwd_dispatch<64>(d, n, f16, g16, fused, D, g4, s);
    return alpha_bwd_dispatch<kMaxBwdLayers>(d, n, f16, g16, fused, D, g4, s);
}

cudaError_t launch_depth_bwd(const BwdDesc* d, int n, int W, int H, const int16_t* winner,
                             const float* g, cudaStream_t s)
{
    if (W <= 0 || H <= 0 || n <= 0) return cudaSuccess;
    const dim3 grid(ceil_div(W, 128), ceil_div(H, 8));
    const float4* g4 = reinterpret_cast<const float4*>(g);
    if (n <= 16) k_depth_bwd<16><<<grid, 256, 0, s>>>(make_bwd<16>(d, n), W, H, winner, g4);
    else if (n <= 64) k_depth_bwd<64><<<grid, 256, 0, s>>>(make_bwd<64>(d, n), W, H, winner, g4);
    else k_depth_bwd<kMaxBwdLayers><<<grid, 256, 0, s>>>(make_bwd<kMaxBwdLayers>(d, n), W, H, winner, g4);
    return cudaGetLastError();
}

}  // namespace ec
