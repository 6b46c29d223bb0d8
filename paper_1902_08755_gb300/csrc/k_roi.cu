// k_roi.cu -- automatic region of interest (thesis 5.3: the ROI computed by
// analysing the frame buffer instead of being supplied by the application,
// which also reveals holes).
//
// One CTA scans one kRoiBlkW x kRoiBlkH block of an image's pvp; the blocks of all
// images of one pixel kind form one launch (kernels are specialised per kind,
// so each launch carries only its kind's registers).  Threads read the
// searched pixels of the block with 16-byte loads where the layout allows (a
// depth or RGBA8 word is 4 bytes, so a load covers 4 / 2 / 1 pixels for
// 4 / 8 / 16-byte pixels), a thread's loads all in flight before any is
// tested; they mark the block's occupancy tiles in shared memory and keep its
// extreme coordinates.  Warp and block min / max reductions leave one set of
// four atomicMax per block on the image's box accumulators, stored as
// (B - x0, x1 + 1, B - y0, y1 + 1) so that all start at zero; a small
// kernel then turns them into rectangles and zeroes them again.  Every searched pixel is read once:
// HBM-bound.
#include "ec_internal.cuh"

#include <algorithm>

namespace ec {
namespace {

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


// Data bits of one 16-byte chunk: bit k for its k-th pixel (KIND 0: 4 depths,
// 1: 4 RGBA8 words, 2: 1 RGBA32F pixel, 3: 2 RGBA16F pixels).
template <int KIND>
__device__ __forceinline__ uint32_t chunk_bits(uint4 v)
{
    if constexpr (KIND == 0)
        return (__uint_as_float(v.x) < 1.0f ? 1u : 0u) | (__uint_as_float(v.y) < 1.0f ? 2u : 0u) |
               (__uint_as_float(v.z) < 1.0f ? 4u : 0u) | (__uint_as_float(v.w) < 1.0f ? 8u : 0u);
    else if constexpr (KIND == 1)
        return (v.x ? 1u : 0u) | (v.y ? 2u : 0u) | (v.z ? 4u : 0u) | (v.w ? 8u : 0u);
    else if constexpr (KIND == 2)
        return (__uint_as_float(v.x) != 0.0f || __uint_as_float(v.y) != 0.0f || __uint_as_float(v.z) != 0.0f ||
                __uint_as_float(v.w) != 0.0f) ? 1u : 0u;
    else
        return (half4_data(v.x, v.y) ? 1u : 0u) | (half4_data(v.z, v.w) ? 2u : 0u);
}

// Data test of one pixel read with element-sized loads.
template <int KIND>
__device__ __forceinline__ bool pixel_data(const void* base, size_t e)
{
    if constexpr (KIND == 0) return reinterpret_cast<const float*>(base)[e] < 1.0f;
    else if constexpr (KIND == 1) return reinterpret_cast<const uint32_t*>(base)[e] != 0u;
    else if constexpr (KIND == 2) {
        const float* f = reinterpret_cast<const float*>(base) + 4 * e;
        return f[0] != 0.0f || f[1] != 0.0f || f[2] != 0.0f || f[3] != 0.0f;
    } else {
        const uint16_t* h = reinterpret_cast<const uint16_t*>(base) + 4 * e;
        return ((h[0] | h[1] | h[2] | h[3]) & 0x7FFFu) != 0u;
    }
}

struct Box { uint32_t mnx, mxx, mny, mxy; };   // mx* hold coordinate + 1, 0 = none

// Scan the searched pixels [ex0,ex1) x [ey0,ey1) of the block at (px0, py0):
// occupancy tiles into occ_s (tpbx per row), extremes into b.  Batches of a
// thread's 16-byte chunks are loaded before any is tested.  INNER: the block
// lies inside the searched region, so no chunk needs a range test.
template <int KIND, bool INNER>
__device__ __forceinline__ void scan_block(const RoiDesc& d, int px0, int py0, int ex0, int ex1, int ey0, int ey1,
                                           int tile, int tpbx, uint8_t* occ_s, Box& b)
{
    constexpr int bpp = KIND == 2 ? 16 : KIND == 3 ? 8 : 4, ppc = 16 / bpp, cpr = kRoiBlkW / ppc;
    constexpr int iters = kRoiBlkH * cpr / kRT, batch = iters < 8 ? iters : 8;
    const uint8_t* base = reinterpret_cast<const uint8_t*>(d.data);
    const bool vec = INNER || d.vec;
#pragma unroll
    for (int k0 = 0; k0 < iters; k0 += batch) {
        uint4 v[batch];
        uint32_t ok = 0;
#pragma unroll
        for (int k = 0; k < batch; ++k) {
            const int c = threadIdx.x + (k0 + k) * kRT;
            const int y = py0 + c / cpr, x = px0 + (c % cpr) * ppc;       // chunk's first pixel
            v[k] = make_uint4(0u, 0u, 0u, 0u);
            if (!INNER && (y < ey0 || y >= ey1 || x + ppc <= ex0 || x >= ex1)) continue;
            ok |= 1u << k;
            const size_t e = (size_t)y * (size_t)d.pitch + (size_t)x;
            if (vec) {
                v[k] = __ldcs(reinterpret_cast<const uint4*>(base + e * bpp));
            } else {
                uint32_t bits = 0;
#pragma unroll
                for (int j = 0; j < ppc; ++j)
                    if (x + j >= ex0 && x + j < ex1 && pixel_data<KIND>(base, e + j)) bits |= 1u << j;
                v[k].x = bits;                               // element-wise result, already bits
            }
        }
#pragma unroll
        for (int k = 0; k < batch; ++k) {
            uint32_t bits;
            if (INNER) {
                bits = chunk_bits<KIND>(v[k]);
            } else {
                if (!((ok >> k) & 1u)) continue;
                bits = vec ? chunk_bits<KIND>(v[k]) : v[k].x;
            }
            if (!bits) continue;
            const int c = threadIdx.x + (k0 + k) * kRT;
            const int y = py0 + c / cpr, x = px0 + (c % cpr) * ppc;
            if (!INNER) {                                    // only the searched pixels count
                const int lo = max(ex0 - x, 0), hi = min(ex1 - x, ppc);
                bits &= ((1u << hi) - 1u) & ~((1u << lo) - 1u);
                if (!bits) continue;
            }
            occ_s[((y - py0) / tile) * tpbx + (x - px0) / tile] = 1;         // a chunk lies in one tile
            b.mnx = min(b.mnx, (uint32_t)(x + __ffs(bits) - 1));
            b.mxx = max(b.mxx, (uint32_t)(x + 32 - __clz(bits)));
            b.mny = min(b.mny, (uint32_t)y);
            b.mxy = max(b.mxy, (uint32_t)y + 1u);
        }
    }
}

// One CTA per block of the images of one pixel kind.
template <int N, int KIND>
__global__ void __launch_bounds__(kRT)
k_detect_roi(const __grid_constant__ RoiList<N> L, uint32_t* acc)
{
    __shared__ uint8_t occ_s[(kRoiBlkW / 8) * (kRoiBlkH / 8)];
    __shared__ uint4 wred[kRT / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile = L.tile, tpbx = kRoiBlkW / tile, ntiles = tpbx * (kRoiBlkH / tile);
    const uint32_t blk = blockIdx.x;
    if (tid < ntiles) occ_s[tid] = 0;
    __syncthreads();
    const int img = find_image(L, blk);
    const RoiDesc& d = L.d[img];
    const uint32_t bi = blk - d.first_block;
    const int bx = (int)(bi % (uint32_t)d.bw), by = (int)(bi / (uint32_t)d.bw);
    const int px0 = bx * kRoiBlkW, py0 = by * kRoiBlkH;
    const int ex0 = max(d.x0, px0), ex1 = min(d.x1, px0 + kRoiBlkW);
    const int ey0 = max(d.y0, py0), ey1 = min(d.y1, py0 + kRoiBlkH);
    Box b{0xFFFFFFFFu, 0u, 0xFFFFFFFFu, 0u};
    if (ex0 < ex1 && ey0 < ey1) {
        const bool inner = d.vec && ex0 == px0 && ex1 == px0 + kRoiBlkW && ey0 == py0 && ey1 == py0 + kRoiBlkH;
        if (inner) scan_block<KIND, true>(d, px0, py0, ex0, ex1, ey0, ey1, tile, tpbx, occ_s, b);
        else scan_block<KIND, false>(d, px0, py0, ex0, ex1, ey0, ey1, tile, tpbx, occ_s, b);
    }
    b.mnx = __reduce_min_sync(0xffffffffu, b.mnx);
    b.mxx = __reduce_max_sync(0xffffffffu, b.mxx);
    b.mny = __reduce_min_sync(0xffffffffu, b.mny);
    b.mxy = __reduce_max_sync(0xffffffffu, b.mxy);
    if (lane == 0) wred[warp] = make_uint4(b.mnx, b.mxx, b.mny, b.mxy);
    __syncthreads();
    if (d.occ && tid < ntiles) {
        const int gx = bx * tpbx + tid % tpbx, gy = by * (kRoiBlkH / tile) + tid / tpbx;
        if (gx < d.gw && gy < d.gh) d.occ[(size_t)gy * d.gw + gx] = occ_s[tid];
    }
    if (tid == 0) {
        uint4 r = wred[0];
        for (int w = 1; w < kRT / 32; ++w) {
            const uint4 v = wred[w];
            r.x = min(r.x, v.x); r.y = max(r.y, v.y); r.z = min(r.z, v.z); r.w = max(r.w, v.w);
        }
        if (r.y) {
            uint32_t* a = acc + 4 * d.idx;
            atomicMax(a + 0, kBig - r.x);
            atomicMax(a + 1, r.y);
            atomicMax(a + 2, kBig - r.z);
            atomicMax(a + 3, r.w);
        }
    }
}

struct RoiOrigins {
    int32_t n;
    int32_t pad;
    int2 o[kRoiPerLaunch];      // pvp origin of every image
};

// Turn every image's accumulators into its rectangle (one thread per image)
// and zero them for the next launch.
__global__ void k_roi_finalize(const __grid_constant__ RoiOrigins O, uint32_t* acc, ec_rect* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= O.n) return;
    const uint4 a = reinterpret_cast<const uint4*>(acc)[i];
    ec_rect r{0, 0, 0, 0};
    if (a.y) {
        const int x0 = (int)(kBig - a.x), y0 = (int)(kBig - a.z);
        r = ec_rect{O.o[i].x + x0, O.o[i].y + y0, (int)a.y - x0, (int)a.w - y0};
    }
    out[i] = r;
    reinterpret_cast<uint4*>(acc)[i] = make_uint4(0u, 0u, 0u, 0u);
}

template <int KIND>
cudaError_t scan_kind(RoiDesc* d, const int* kinds, const uint32_t* nblocks, int n, int tile,
                      uint32_t* acc, cudaStream_t s)
{
    RoiList<kRoiPerLaunch> L;
    L.n = 0;
    L.tile = tile;
    L.pad = 0;
    uint32_t blocks = 0;
    for (int i = 0; i < n; ++i) {
        if (kinds[i] != KIND || nblocks[i] == 0) continue;
        RoiDesc r = d[i];
        r.first_block = blocks;
        blocks += nblocks[i];
        L.d[L.n++] = r;
    }
    L.blocks = blocks;
    if (blocks == 0) return cudaSuccess;
    k_detect_roi<kRoiPerLaunch, KIND><<<blocks, kRT, 0, s>>>(L, acc);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_detect_roi(RoiDesc* d, const int* kinds, const uint32_t* nblocks, int n, int tile,
                              uint32_t* scratch, ec_rect* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    cudaError_t e = scan_kind<0>(d, kinds, nblocks, n, tile, scratch, s);
    if (e == cudaSuccess) e = scan_kind<1>(d, kinds, nblocks, n, tile, scratch, s);
    if (e == cudaSuccess) e = scan_kind<2>(d, kinds, nblocks, n, tile, scratch, s);
    if (e == cudaSuccess) e = scan_kind<3>(d, kinds, nblocks, n, tile, scratch, s);
    if (e != cudaSuccess) return e;
    RoiOrigins O;
    O.n = n;
    O.pad = 0;
    for (int i = 0; i < n; ++i) O.o[i] = make_int2(d[i].ox, d[i].oy);
    k_roi_finalize<<<(n + 127) / 128, 128, 0, s>>>(O, scratch, out);
    return cudaGetLastError();
}

}  // namespace ec
