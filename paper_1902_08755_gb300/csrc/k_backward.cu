// k_backward.cu -- gradients of the compositing operators for sm_103a.
//
// Ordered compositing (thesis 5.2.1) is differentiated through its front-to-
// back recurrence C += T c_k, T *= (1 - a_k):
//   dL/dc_k^{RGB} = g^{RGB} T_k,   dL/da_k = T_k (g^A - R_k),
//   R_{n-1} = 0,  R_{k-1} = g.c_k + (1 - a_k) R_k      (reverse "behind" scan).
// Nothing per layer is kept from the forward: a CTA stages the layer stack of
// its 64-pixel row segment in shared memory with cp.async (16/8/4-byte copies,
// zero-filled outside a layer's ROI, which is exactly a transparent layer),
// runs the forward scan (recording T_k in shared memory), then the reverse
// scan, and writes every layer's gradient.  Layers are read from HBM once.
// Stacks larger than the shared-memory budget are processed in chunks: the
// forward keeps T at each chunk start, and the reverse reloads the chunks in
// reverse order (all but the last are then read twice).
//
// The fused variant takes the loss weights w up front (L = sum w * out, so
// the upstream gradient is w) and also writes out and T_final.
//
// Depth compositing (thesis 5.2.1) copies the winner's colour, so its
// gradient routes grad_out to the winning input and writes zero elsewhere.
#include <algorithm>

#include "ec_internal.cuh"

namespace ec {
namespace {

constexpr int kP = 64;            // pixels (= threads) per alpha-backward CTA
constexpr int kMaxChunks = 16;

__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes, int src_bytes)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if (bytes == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
    else if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

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

template <int N>
__device__ __forceinline__ int active_grad_layers(const BwdList<N>& L, int tx0, int tx1, int y,
                                                  int16_t* act, int* nact)
{
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        int base = 0;
        for (int i0 = 0; i0 < L.n; i0 += 32) {
            const int i = i0 + lane;
            bool hit = false;
            if (i < L.n) {
                const BwdDesc& d = L.d[i];
                hit = d.gx0 < tx1 && d.gx1 > tx0 && d.gy0 <= y && d.gy1 > y;
            }
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (hit) act[base + __popc(m & ((1u << lane) - 1u))] = (int16_t)i;
            base += __popc(m);
        }
        if (lane == 0) *nact = base;
    }
    __syncthreads();
    return *nact;
}

// What a CTA needs of one layer for its 64-pixel row segment, built once per
// CTA: addresses of the segment's first pixel in the colour and gradient
// buffers (only offset by columns that lie inside the ROI / pvp before use)
// and the clipped column ranges relative to the segment start.
struct LayerTile {
    uintptr_t src;          // colour address of pixel (tx0, y)
    uintptr_t grad;         // gradient address of pixel (tx0, y)
    int16_t rx0, rx1;       // ROI columns [rx0, rx1) (empty if row y is outside)
    int16_t gx0, gx1;       // gradient columns [gx0, gx1) (empty if row y is outside)
    int16_t cls, gvec;
    int32_t pad;
};
static_assert(sizeof(LayerTile) == 32, "tile record");

template <bool F16, bool G16>
__device__ __forceinline__ LayerTile make_tile(const BwdDesc& d, int tx0, int y)
{
    constexpr int S = F16 ? 8 : 16, GS = G16 ? 8 : 16;
    LayerTile t;
    const int64_t e = (int64_t)(y - d.oy) * d.pitch + (int64_t)(tx0 - d.ox);
    t.src = reinterpret_cast<uintptr_t>(d.color) + (uintptr_t)(e * S);
    t.grad = reinterpret_cast<uintptr_t>(d.grad) + (uintptr_t)(e * GS);
    const bool rrow = y >= d.y0 && y < d.y1, grow = y >= d.gy0 && y < d.gy1;
    t.rx0 = (int16_t)(rrow ? max(d.x0 - tx0, 0) : 0);
    t.rx1 = (int16_t)(rrow ? min(d.x1 - tx0, kP) : 0);
    t.gx0 = (int16_t)(grow ? max(d.gx0 - tx0, 0) : 0);
    t.gx1 = (int16_t)(grow ? min(d.gx1 - tx0, kP) : 0);
    t.cls = d.cls;
    t.gvec = d.gvec;
    t.pad = 0;
    return t;
}

// Stage this thread's pixel of one layer into its slot (zero outside the ROI;
// `dummy` is any valid global address, never read when zero-filling).
template <bool F16>
__device__ __forceinline__ void stage_px(uint8_t* slot, const LayerTile& t, int tid, const void* dummy)
{
    constexpr int S = F16 ? 8 : 16;
    const bool in = tid >= t.rx0 && tid < t.rx1;
    const uint8_t* src = in ? reinterpret_cast<const uint8_t*>(t.src) + tid * S
                            : reinterpret_cast<const uint8_t*>(dummy);
    if (t.cls >= S) {
        cp_async(slot, src, S, in ? S : 0);
    } else if (t.cls >= 4) {
#pragma unroll
        for (int o = 0; o < S; o += 4) cp_async(slot + o, in ? src + o : src, 4, in ? 4 : 0);
    } else {                          // 2-byte aligned half data: synchronous copy
        const unsigned short* h = reinterpret_cast<const unsigned short*>(src);
        unsigned short* d = reinterpret_cast<unsigned short*>(slot);
#pragma unroll
        for (int o = 0; o < S / 2; ++o) d[o] = in ? h[o] : (unsigned short)0;
    }
}

template <bool F16>
__device__ __forceinline__ float4 read_slot(const uint8_t* slot)
{
    if constexpr (F16) return h4_to_f4(*reinterpret_cast<const uint2*>(slot));
    else return *reinterpret_cast<const float4*>(slot);
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

template <int N, bool F16, bool G16, bool FUSED>
__global__ void __launch_bounds__(kP)
k_alpha_bwd(const __grid_constant__ BwdList<N> L, const __grid_constant__ DstDesc D,
            const float4* __restrict__ g, int chunk)
{
    constexpr int S = F16 ? 8 : 16, GS = G16 ? 8 : 16;
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int16_t act[N];
    __shared__ LayerTile tiles[N];
    __shared__ int nact_s;
    __shared__ float Tc[kMaxChunks][kP];
    uint8_t* stage = smem;                                             // [chunk][kP][S]
    float* Ts = reinterpret_cast<float*>(smem + (size_t)chunk * kP * S);  // [chunk][kP]

    const int tid = threadIdx.x;
    const int tx0 = blockIdx.x * kP, y = blockIdx.y;
    const int nact = active_grad_layers(L, tx0, min(tx0 + kP, D.W), y, act, &nact_s);
    for (int k = tid; k < nact; k += kP) tiles[k] = make_tile<F16, G16>(L.d[act[k]], tx0, y);
    __syncthreads();
    const int x = tx0 + tid;
    if (x >= D.W) return;                      // no block-wide barrier follows

    const float4* gpix = g + (size_t)y * D.W + x;
    const float4 gp = __ldcs(gpix);
    const int nchunks = (nact + chunk - 1) / chunk;
    float T = 1.0f;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    uint8_t* myslot = stage + (size_t)tid * S;
    float* myT = Ts + tid;

    // forward: T_k for every layer, and (fused) the composite
    for (int ch = 0; ch < nchunks; ++ch) {
        const int k0 = ch * chunk, k1 = min(nact, k0 + chunk);
        asm volatile("" ::: "memory");        // reads of the previous chunk come first
        for (int k = k0; k < k1; ++k) stage_px<F16>(myslot + (size_t)(k - k0) * kP * S, tiles[k], tid, gpix);
        cp_async_wait_all();
        Tc[ch][tid] = T;
#pragma unroll 4
        for (int k = k0; k < k1; ++k) {
            const float4 c = read_slot<F16>(myslot + (size_t)(k - k0) * kP * S);
            myT[(k - k0) * kP] = T;
            if (FUSED) {
                acc.x = fmaf(T, c.x, acc.x);
                acc.y = fmaf(T, c.y, acc.y);
                acc.z = fmaf(T, c.z, acc.z);
                acc.w = fmaf(T, c.w, acc.w);
            }
            T = fmaf(-T, c.w, T);
        }
    }
    if (FUSED) {
        const size_t o = (size_t)y * (size_t)D.pitch + (size_t)x;
        if constexpr (F16) {
            const uint2 h = f4_to_h4(acc);
            unsigned short* hp = reinterpret_cast<unsigned short*>(reinterpret_cast<uint2*>(D.color) + o);
            if (D.vec) __stcs(reinterpret_cast<uint2*>(hp), h);
            else { hp[0] = (unsigned short)h.x; hp[1] = (unsigned short)(h.x >> 16); hp[2] = (unsigned short)h.y; hp[3] = (unsigned short)(h.y >> 16); }
        } else {
            float4* op = reinterpret_cast<float4*>(D.color) + o;
            if (D.vec) __stcs(op, acc);
            else { float* f = reinterpret_cast<float*>(op); f[0] = acc.x; f[1] = acc.y; f[2] = acc.z; f[3] = acc.w; }
        }
        if (D.tfinal) D.tfinal[(size_t)y * D.W + x] = T;
    }

    // reverse: R_k and the gradients, back to front
    float R = 0.0f;
    for (int ch = nchunks - 1; ch >= 0; --ch) {
        const int k0 = ch * chunk, k1 = min(nact, k0 + chunk);
        if (ch != nchunks - 1) {               // reload and recompute T inside the chunk
            asm volatile("" ::: "memory");
            for (int k = k0; k < k1; ++k) stage_px<F16>(myslot + (size_t)(k - k0) * kP * S, tiles[k], tid, gpix);
            cp_async_wait_all();
            float t = Tc[ch][tid];
            for (int k = k0; k < k1; ++k) {
                const float4 c = read_slot<F16>(myslot + (size_t)(k - k0) * kP * S);
                myT[(k - k0) * kP] = t;
                t = fmaf(-t, c.w, t);
            }
        }
#pragma unroll 4
        for (int k = k1 - 1; k >= k0; --k) {
            const LayerTile& t = tiles[k];
            const float4 c = read_slot<F16>(myslot + (size_t)(k - k0) * kP * S);
            const float Tk = myT[(k - k0) * kP];
            if (tid >= t.gx0 && tid < t.gx1) {
                const bool in = tid >= t.rx0 && tid < t.rx1;
                const float4 gr = in ? make_float4(gp.x * Tk, gp.y * Tk, gp.z * Tk, Tk * (gp.w - R))
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
                store_grad_at<G16>(t.grad + (uintptr_t)tid * GS, t.gvec != 0, gr);
            }
            const float gc = fmaf(gp.x, c.x, fmaf(gp.y, c.y, fmaf(gp.z, c.z, gp.w * c.w)));
            R = fmaf(1.0f - c.w, R, gc);
        }
    }
}

// Segmented variant for stacks that fit in shared memory: NS threads share a
// pixel, each owning a contiguous segment of its layers (threads p, p+64, ...
// of the CTA).  Both recurrences split exactly across segments:
//   forward  T_k = T_start(s) * T'_k, T'_k the transmittance inside segment s,
//            T_start(s) = prod over earlier segments of P_u = prod (1 - a);
//   reverse  R entering segment s from behind = sum_{t>s} A_t prod_{s<u<t} P_u
//            with A_t = sum_{j in t} T'_j (g.c_j), evaluated Horner-style,
// after which every segment runs the exact reverse recurrence over its own
// layers.  NS times more threads per pixel hide the shared-memory latency
// that a one-thread-per-pixel scan exposes at this occupancy.
template <int N, bool F16, bool G16, bool FUSED, int NS>
__global__ void __launch_bounds__(kP * NS)
k_alpha_bwd_seg(const __grid_constant__ BwdList<N> L, const __grid_constant__ DstDesc D,
                const float4* __restrict__ g, int cap)
{
    constexpr int S = F16 ? 8 : 16, GS = G16 ? 8 : 16;
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int16_t act[N];
    __shared__ LayerTile tiles[N];
    __shared__ int nact_s;
    __shared__ float Pseg[NS][kP], Aseg[NS][kP];
    __shared__ float4 Cseg[FUSED ? NS : 1][kP];
    uint8_t* stage = smem;                                          // [cap][kP][S]
    float* Tl = reinterpret_cast<float*>(smem + (size_t)cap * kP * S);  // [cap][kP]

    const int tid = threadIdx.x, p = tid % kP, sg = tid / kP;
    const int tx0 = blockIdx.x * kP, y = blockIdx.y;
    const int nact = active_grad_layers(L, tx0, min(tx0 + kP, D.W), y, act, &nact_s);
    for (int k = tid; k < nact; k += kP * NS) tiles[k] = make_tile<F16, G16>(L.d[act[k]], tx0, y);
    __syncthreads();
    const int x = tx0 + p;
    const bool valid = x < D.W;                // every thread reaches the barrier below
    const int k0 = (sg * nact) / NS, k1 = ((sg + 1) * nact) / NS;
    const float4* gpix = g + (size_t)y * D.W + (valid ? x : 0);
    const float4 gp = valid ? __ldcs(gpix) : make_float4(0.f, 0.f, 0.f, 0.f);
    uint8_t* myslot = stage + (size_t)p * S;
    float* myT = Tl + p;

    // local forward over this segment
    if (valid)
        for (int k = k0; k < k1; ++k) stage_px<F16>(myslot + (size_t)k * kP * S, tiles[k], p, gpix);
    cp_async_wait_all();
    float Tp = 1.0f, A = 0.0f;
    float4 Cl = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
    for (int k = k0; k < k1; ++k) {
        const float4 c = valid ? read_slot<F16>(myslot + (size_t)k * kP * S) : make_float4(0.f, 0.f, 0.f, 0.f);
        myT[k * kP] = Tp;
        if (FUSED) {
            Cl.x = fmaf(Tp, c.x, Cl.x);
            Cl.y = fmaf(Tp, c.y, Cl.y);
            Cl.z = fmaf(Tp, c.z, Cl.z);
            Cl.w = fmaf(Tp, c.w, Cl.w);
        }
        const float gc = fmaf(gp.x, c.x, fmaf(gp.y, c.y, fmaf(gp.z, c.z, gp.w * c.w)));
        A = fmaf(Tp, gc, A);
        Tp = fmaf(-Tp, c.w, Tp);
    }
    Pseg[sg][p] = Tp;
    Aseg[sg][p] = A;
    if (FUSED) Cseg[sg][p] = Cl;
    __syncthreads();
    if (!valid) return;

    float Tstart = 1.0f;
    for (int u = 0; u < sg; ++u) Tstart *= Pseg[u][p];
    float R = 0.0f;
    for (int t = NS - 1; t > sg; --t) R = fmaf(Pseg[t][p], R, Aseg[t][p]);

    if (FUSED && sg == 0) {
        float Tacc = 1.0f;
        float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int u = 0; u < NS; ++u) {
            const float4 c = Cseg[u][p];
            out.x = fmaf(Tacc, c.x, out.x);
            out.y = fmaf(Tacc, c.y, out.y);
            out.z = fmaf(Tacc, c.z, out.z);
            out.w = fmaf(Tacc, c.w, out.w);
            Tacc *= Pseg[u][p];
        }
        const size_t o = (size_t)y * (size_t)D.pitch + (size_t)x;
        if constexpr (F16) {
            const uint2 h = f4_to_h4(out);
            unsigned short* hp = reinterpret_cast<unsigned short*>(reinterpret_cast<uint2*>(D.color) + o);
            if (D.vec) __stcs(reinterpret_cast<uint2*>(hp), h);
            else { hp[0] = (unsigned short)h.x; hp[1] = (unsigned short)(h.x >> 16); hp[2] = (unsigned short)h.y; hp[3] = (unsigned short)(h.y >> 16); }
        } else {
            float4* op = reinterpret_cast<float4*>(D.color) + o;
            if (D.vec) __stcs(op, out);
            else { float* f = reinterpret_cast<float*>(op); f[0] = out.x; f[1] = out.y; f[2] = out.z; f[3] = out.w; }
        }
        if (D.tfinal) D.tfinal[(size_t)y * D.W + x] = Tacc;
    }

    // reverse over this segment, entering with the R of the layers behind it
#pragma unroll 4
    for (int k = k1 - 1; k >= k0; --k) {
        const LayerTile& t = tiles[k];
        const float4 c = read_slot<F16>(myslot + (size_t)k * kP * S);
        const float Tk = Tstart * myT[k * kP];
        if (p >= t.gx0 && p < t.gx1) {
            const bool in = p >= t.rx0 && p < t.rx1;
            const float4 gr = in ? make_float4(gp.x * Tk, gp.y * Tk, gp.z * Tk, Tk * (gp.w - R))
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
            store_grad_at<G16>(t.grad + (uintptr_t)p * GS, t.gvec != 0, gr);
        }
        const float gc = fmaf(gp.x, c.x, fmaf(gp.y, c.y, fmaf(gp.z, c.z, gp.w * c.w)));
        R = fmaf(1.0f - c.w, R, gc);
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

template <int N, bool F16, bool G16, bool FUSED, int NS>
cudaError_t alpha_bwd_seg_n(const BwdDesc* d, int n, const DstDesc& D, const float4* g,
                            cudaStream_t s)
{
    const int cap = std::max(n, 1);
    const size_t smem = (size_t)cap * kP * ((F16 ? 8 : 16) + 4);
    auto kern = k_alpha_bwd_seg<N, F16, G16, FUSED, NS>;
    // static + dynamic shared memory may pass the default 48 KB window
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid(ceil_div(D.W, kP), D.H);
    kern<<<grid, kP * NS, smem, s>>>(make_bwd<N>(d, n), D, g, cap);
    return cudaGetLastError();
}

template <int N, bool F16, bool G16, bool FUSED>
cudaError_t alpha_bwd_n(const BwdDesc* d, int n, const DstDesc& D, const float4* g, int chunk,
                        cudaStream_t s)
{
    if (chunk >= n) {                          // whole stack fits: segmented kernel
        if (n >= 32) return alpha_bwd_seg_n<N, F16, G16, FUSED, 8>(d, n, D, g, s);
        if (n >= 16) return alpha_bwd_seg_n<N, F16, G16, FUSED, 4>(d, n, D, g, s);
        if (n >= 8) return alpha_bwd_seg_n<N, F16, G16, FUSED, 2>(d, n, D, g, s);
        return alpha_bwd_seg_n<N, F16, G16, FUSED, 1>(d, n, D, g, s);
    }
    const size_t smem = (size_t)chunk * kP * ((F16 ? 8 : 16) + 4);
    auto kern = k_alpha_bwd<N, F16, G16, FUSED>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid(ceil_div(D.W, kP), D.H);
    kern<<<grid, kP, smem, s>>>(make_bwd<N>(d, n), D, g, chunk);
    return cudaGetLastError();
}

template <int N>
cudaError_t alpha_bwd_dispatch(const BwdDesc* d, int n, bool f16, bool g16, bool fused,
                               const DstDesc& D, const float4* g, int chunk, cudaStream_t s)
{
    if (f16) {
        if (g16) return fused ? alpha_bwd_n<N, true, true, true>(d, n, D, g, chunk, s)
                              : alpha_bwd_n<N, true, true, false>(d, n, D, g, chunk, s);
        return fused ? alpha_bwd_n<N, true, false, true>(d, n, D, g, chunk, s)
                     : alpha_bwd_n<N, true, false, false>(d, n, D, g, chunk, s);
    }
    if (g16) return fused ? alpha_bwd_n<N, false, true, true>(d, n, D, g, chunk, s)
                          : alpha_bwd_n<N, false, true, false>(d, n, D, g, chunk, s);
    return fused ? alpha_bwd_n<N, false, false, true>(d, n, D, g, chunk, s)
                 : alpha_bwd_n<N, false, false, false>(d, n, D, g, chunk, s);
}

}  // namespace

int alpha_bwd_chunk(int n, bool f16)
{
    // shared-memory budget per CTA: ~96 KB leaves room for two CTAs per SM
    const int per_layer = kP * ((f16 ? 8 : 16) + 4);
    const int cap = (100 * 1024) / per_layer;
    const int need = (n + kMaxChunks - 1) / kMaxChunks;
    return std::max(1, std::max(std::min(n, cap), need));
}

cudaError_t launch_alpha_bwd(const BwdDesc* d, int n, bool f16, bool g16, bool fused,
                             const DstDesc& D, const float* g, cudaStream_t s)
{
    if (D.W <= 0 || D.H <= 0) return cudaSuccess;
    const int chunk = alpha_bwd_chunk(n, f16);
    const float4* g4 = reinterpret_cast<const float4*>(g);
    if (n <= 16) return alpha_bwd_dispatch<16>(d, n, f16, g16, fused, D, g4, chunk, s);
    if (n <= 64) return alpha_bwd_dispatch<64>(d, n, f16, g16, fused, D, g4, chunk, s);
    return alpha_bwd_dispatch<kMaxBwdLayers>(d, n, f16, g16, fused, D, g4, chunk, s);
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
