// k_roi.cu -- automatic region of interest (thesis 5.3: the ROI computed by
// analysing the frame buffer instead of being supplied by the application,
// which also reveals holes).
//
// One CTA scans one 64 x 64 block of an image's pvp (blocks of all images of
// a launch form one grid).  Threads read the searched pixels of the block
// with 16-byte loads where the layout allows (a depth or RGBA8 word is 4
// bytes, so a load covers 4 / 2 / 1 pixels for 4 / 8 / 16-byte pixels),
// test each pixel for data, mark the block's occupancy tiles in shared
// memory and keep the block's extreme coordinates.  Warp and block min / max
// reductions leave one set of four atomicMax per block on the image's box
// accumulators, stored as (B - x0, x1 + 1, B - y0, y1 + 1) so that all of
// them start at zero.  The last block to finish (a done counter after a
// fence) turns every image's accumulators into its rectangle.  The kernel
// reads each searched pixel once: HBM-bound.
#include "ec_internal.cuh"

namespace ec {
namespace {

constexpr int kBlk = 64;          // block edge in pixels
constexpr int kRT = 256;          // threads per CTA
constexpr uint32_t kBig = 1u << 30;

template <int N>
__device__ __forceinline__ int find_image(const RoiList<N>& L, uint32_t blk)
{
    int lo = 0, hi = L.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (L.d[mid].first_block <= blk) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ bool half4_data(uint32_t a, uint32_t b) { return ((a | b) & 0x7FFF7FFFu) != 0u; }

__device__ __forceinline__ bool f4_data(float4 v) { return v.x != 0.0f || v.y != 0.0f || v.z != 0.0f || v.w != 0.0f; }

// Data bits of one 16-byte chunk: bit k for its k-th pixel (kind 0: 4 depths,
// 1: 4 RGBA8 words, 2: 1 RGBA32F pixel, 3: 2 RGBA16F pixels).
__device__ __forceinline__ uint32_t chunk_bits(int kind, uint4 v)
{
    switch (kind) {
    case 0:
        return (__uint_as_float(v.x) < 1.0f ? 1u : 0u) | (__uint_as_float(v.y) < 1.0f ? 2u : 0u) |
               (__uint_as_float(v.z) < 1.0f ? 4u : 0u) | (__uint_as_float(v.w) < 1.0f ? 8u : 0u);
    case 1:
        return (v.x ? 1u : 0u) | (v.y ? 2u : 0u) | (v.z ? 4u : 0u) | (v.w ? 8u : 0u);
    case 2:
        return f4_data(make_float4(__uint_as_float(v.x), __uint_as_float(v.y), __uint_as_float(v.z),
                                   __uint_as_float(v.w))) ? 1u : 0u;
    default:
        return (half4_data(v.x, v.y) ? 1u : 0u) | (half4_data(v.z, v.w) ? 2u : 0u);
    }
}

// Data test of one pixel read with element-sized loads.
__device__ __forceinline__ bool pixel_data(int kind, const void* base, size_t e)
{
    switch (kind) {
    case 0: return reinterpret_cast<const float*>(base)[e] < 1.0f;
    case 1: return reinterpret_cast<const uint32_t*>(base)[e] != 0u;
    case 2: {
        const float* f = reinterpret_cast<const float*>(base) + 4 * e;
        return f[0] != 0.0f || f[1] != 0.0f || f[2] != 0.0f || f[3] != 0.0f;
    }
    default: {
        const uint16_t* h = reinterpret_cast<const uint16_t*>(base) + 4 * e;
        return ((h[0] | h[1] | h[2] | h[3]) & 0x7FFFu) != 0u;
    }
    }
}

template <int N>
__global__ void __launch_bounds__(kRT)
k_detect_roi(const __grid_constant__ RoiList<N> L, uint32_t* acc, uint32_t* done, ec_rect* out)
{
    __shared__ uint8_t occ_s[(kBlk / 8) * (kBlk / 8)];
    __shared__ uint4 wred[kRT / 32];
    __shared__ int last_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t blk = blockIdx.x;
    const int tile = L.tile, tpb = kBlk / tile;           // occupancy tiles per block edge
    if (tid < tpb * tpb) occ_s[tid] = 0;
    __syncthreads();

    uint32_t mnx = 0xFFFFFFFFu, mxx = 0u, mny = 0xFFFFFFFFu, mxy = 0u;   // mx* hold coordinate + 1
    int img = -1;
    if (blk < L.blocks) {
        img = find_image(L, blk);
        const RoiDesc& d = L.d[img];
        const uint32_t b = blk - d.first_block;
        const int px0 = (int)(b % (uint32_t)d.bw) * kBlk, py0 = (int)(b / (uint32_t)d.bw) * kBlk;
        const int ex0 = max(d.x0, px0), ex1 = min(d.x1, px0 + kBlk);
        const int ey0 = max(d.y0, py0), ey1 = min(d.y1, py0 + kBlk);
        if (ex0 < ex1 && ey0 < ey1) {
            const int kind = d.kind;
            const int bpp = kind == 2 ? 16 : kind == 3 ? 8 : 4, ppc = 16 / bpp;   // pixels per chunk
            const int cpr = kBlk / ppc;                                           // chunks per row
            const uint8_t* base = reinterpret_cast<const uint8_t*>(d.data);
#pragma unroll 4
            for (int c = tid; c < kBlk * cpr; c += kRT) {
                const int y = py0 + c / cpr, x = px0 + (c % cpr) * ppc;       // chunk's first pixel
                if (y < ey0 || y >= ey1 || x + ppc <= ex0 || x >= ex1) continue;
                uint32_t bits = 0;
                const size_t e = (size_t)y * (size_t)d.pitch + (size_t)x;
                if (d.vec) {
                    bits = chunk_bits(kind, __ldcs(reinterpret_cast<const uint4*>(base + e * bpp)));
                } else {
                    for (int k = 0; k < ppc; ++k)
                        if (x + k >= ex0 && x + k < ex1 && pixel_data(kind, base, e + k)) bits |= 1u << k;
                }
                // only the searched pixels of the chunk count
                const int lo = max(ex0 - x, 0), hi = min(ex1 - x, ppc);
                bits &= ((1u << hi) - 1u) & ~((1u << lo) - 1u);
                if (!bits) continue;
                occ_s[((y - py0) / tile) * tpb + (x - px0) / tile] = 1;       // a chunk lies in one tile
                mnx = min(mnx, (uint32_t)(x + __ffs(bits) - 1));
                mxx = max(mxx, (uint32_t)(x + 32 - __clz(bits)));
                mny = min(mny, (uint32_t)y);
                mxy = max(mxy, (uint32_t)y + 1u);
            }
        }
    }
    mnx = __reduce_min_sync(0xffffffffu, mnx);
    mxx = __reduce_max_sync(0xffffffffu, mxx);
    mny = __reduce_min_sync(0xffffffffu, mny);
    mxy = __reduce_max_sync(0xffffffffu, mxy);
    if (lane == 0) wred[warp] = make_uint4(mnx, mxx, mny, mxy);
    __syncthreads();
    if (img >= 0) {
        const RoiDesc& d = L.d[img];
        const uint32_t b = blk - d.first_block;
        const int bx = (int)(b % (uint32_t)d.bw), by = (int)(b / (uint32_t)d.bw);
        if (d.occ && tid < tpb * tpb) {
            const int gx = bx * tpb + tid % tpb, gy = by * tpb + tid / tpb;
            if (gx < d.gw && gy < d.gh) d.occ[(size_t)gy * d.gw + gx] = occ_s[tid];
        }
        if (tid == 0) {
            uint4 r = wred[0];
            for (int w = 1; w < kRT / 32; ++w) {
                const uint4 v = wred[w];
                r.x = min(r.x, v.x); r.y = max(r.y, v.y); r.z = min(r.z, v.z); r.w = max(r.w, v.w);
            }
            if (r.y) {
                uint32_t* a = acc + 4 * img;
                atomicMax(a + 0, kBig - r.x);
                atomicMax(a + 1, r.y);
                atomicMax(a + 2, kBig - r.z);
                atomicMax(a + 3, r.w);
            }
        }
    }
    // the last block to finish writes every image's rectangle
    if (tid == 0) {
        __threadfence();
        last_s = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last_s) return;
    __threadfence();
    for (int i = tid; i < L.n; i += kRT) {
        const RoiDesc& d = L.d[i];
        const uint32_t a1 = __ldcg(acc + 4 * i + 1);
        ec_rect r{0, 0, 0, 0};
        if (a1) {
            const int x0 = (int)(kBig - __ldcg(acc + 4 * i + 0)), y0 = (int)(kBig - __ldcg(acc + 4 * i + 2));
            const int y1 = (int)__ldcg(acc + 4 * i + 3);
            r = ec_rect{d.ox + x0, d.oy + y0, (int)a1 - x0, y1 - y0};
        }
        out[i] = r;
    }
}

}  // namespace

cudaError_t launch_detect_roi(const RoiDesc* d, int n, int tile, uint32_t blocks, uint32_t* scratch,
                              ec_rect* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(scratch, 0, (4ull * n + 1) * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    RoiList<kRoiPerLaunch> L;
    L.n = n;
    L.blocks = blocks;
    L.tile = tile;
    L.pad = 0;
    for (int i = 0; i < n; ++i) L.d[i] = d[i];
    const uint32_t grid = blocks > 0 ? blocks : 1u;        // one block to write empty results
    k_detect_roi<kRoiPerLaunch><<<grid, kRT, 0, s>>>(L, scratch, scratch + 4 * n, out);
    return cudaGetLastError();
}

}  // namespace ec
