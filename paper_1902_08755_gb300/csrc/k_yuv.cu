// k_yuv.cu -- the lossy YUV compressor of thesis 5.5.3 for sm_103a: a colour
// space conversion with chroma subsampling run before the RLE codec, and its
// inverse after decoding.
//
// Full-range BT.601 in 8-bit fixed point (coefficients x 256, divisions
// rounding down).  Every 2x2 block of RGBA8 pixels keeps its four luma values
// and the rounded means of its pixels' chroma and alpha.  The packed image is
// ceil(w/2) words wide: rows [0, ceil(h/2)) hold luma words (byte k = Y of
// pixel (2bx + (k & 1), 2by + (k >> 1)), 0 where the image has no pixel),
// rows [ceil(h/2), 2 ceil(h/2)) chroma words (bytes U, V, A, 0).
//
// One thread per block; a row pair of the block is one 8-byte access where
// the buffer allows it.  A launch covers many images: CTA tiles of 32 x 8
// blocks are numbered across the images and each CTA finds its image by a
// binary search of the images' first tiles.  Both kernels are HBM-bound: 4
// bytes read and 2 written per pixel to encode, the reverse to decode.
#include "ec_internal.cuh"

namespace ec {
namespace {

constexpr int kYX = 32, kYY = 8;     // blocks per CTA: 32 x 8

// floor(x / 256) for x > -2^20
__device__ __forceinline__ int floor256(int x) { return ((x + (1 << 20)) >> 8) - (1 << 12); }
__device__ __forceinline__ int clamp8(int v) { return min(255, max(0, v)); }

__device__ __forceinline__ void to_yuv(uint32_t p, int& Y, int& U, int& V)
{
    const int R = (int)(p & 0xFFu), G = (int)((p >> 8) & 0xFFu), B = (int)((p >> 16) & 0xFFu);
    Y = (77 * R + 150 * G + 29 * B + 128) >> 8;
    U = min(255, (-43 * R - 85 * G + 128 * B + 32896) >> 8);   // 128 + ... (never negative)
    V = min(255, (128 * R - 107 * G - 21 * B + 32896) >> 8);
}

// CTA tile t of a job list: the job whose tiles [first, first + ntiles) hold it.
template <int N>
__device__ __forceinline__ const YuvJob& tile_job(const YuvJobList<N>& J, uint32_t t, int& bx, int& by)
{
    int lo = 0, hi = J.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (J.j[mid].first <= t) lo = mid;
        else hi = mid - 1;
    }
    const YuvJob& jb = J.j[lo];
    const uint32_t r = t - jb.first, tx = r % jb.tiles_x;
    bx = (int)(tx * kYX) + threadIdx.x;
    by = (int)((r / jb.tiles_x) * kYY) + threadIdx.y;
    return jb;
}

template <int N>
__global__ void __launch_bounds__(kYX * kYY)
k_yuv_encode(const __grid_constant__ YuvJobList<N> J)
{
    int bx, by;
    const YuvJob& jb = tile_job(J, blockIdx.x, bx, by);
    const uint32_t* __restrict__ src = jb.src;
    uint32_t* __restrict__ dst = jb.dst;
    const int w = jb.w, h = jb.h, pitch = jb.pitch, dpitch = jb.dpitch;
    const bool vec = jb.vec;
    const int bw = (w + 1) >> 1, bh = (h + 1) >> 1;
    if (bx >= bw || by >= bh) return;
    const int x = 2 * bx;
    uint32_t px[4] = {0u, 0u, 0u, 0u};
    bool has[4] = {false, false, false, false};
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int y = 2 * by + r;
        if (y >= h) continue;
        const uint32_t* row = src + (size_t)y * pitch;
        if (vec && x + 1 < w) {
            const uint2 v = __ldcs(reinterpret_cast<const uint2*>(row + x));
            px[2 * r] = v.x;
            px[2 * r + 1] = v.y;
            has[2 * r] = has[2 * r + 1] = true;
        } else {
            px[2 * r] = __ldcs(row + x);
            has[2 * r] = true;
            if (x + 1 < w) {
                px[2 * r + 1] = __ldcs(row + x + 1);
                has[2 * r + 1] = true;
            }
        }
    }
    uint32_t luma = 0u;
    int su = 0, sv = 0, sa = 0, cnt = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (!has[k]) continue;
        int Y, U, V;
        to_yuv(px[k], Y, U, V);
        luma |= (uint32_t)Y << (8 * k);
        su += U;
        sv += V;
        sa += (int)(px[k] >> 24);
        ++cnt;
    }
    const int sh = cnt == 4 ? 2 : (cnt == 2 ? 1 : 0);          // cnt is 1, 2 or 4
    const int half = cnt >> 1;
    dst[(size_t)by * dpitch + bx] = luma;
    dst[(size_t)(bh + by) * dpitch + bx] = (uint32_t)((su + half) >> sh) | ((uint32_t)((sv + half) >> sh) << 8) |
                                          ((uint32_t)((sa + half) >> sh) << 16);
}

template <int N>
__global__ void __launch_bounds__(kYX * kYY)
k_yuv_decode(const __grid_constant__ YuvJobList<N> J)
{
    int bx, by;
    const YuvJob& jb = tile_job(J, blockIdx.x, bx, by);
    const uint32_t* __restrict__ src = jb.src;
    uint32_t* __restrict__ dst = jb.dst;
    const int w = jb.w, h = jb.h, pitch = jb.pitch, spitch = jb.dpitch;
    const bool vec = jb.vec;
    const int bw = (w + 1) >> 1, bh = (h + 1) >> 1;
    if (bx >= bw || by >= bh) return;
    const uint32_t luma = __ldcs(src + (size_t)by * spitch + bx);
    const uint32_t ch = __ldcs(src + (size_t)(bh + by) * spitch + bx);
    const int U = (int)(ch & 0xFFu) - 128, V = (int)((ch >> 8) & 0xFFu) - 128;
    const uint32_t A = (ch >> 16) & 0xFFu;
    const int dR = floor256(359 * V + 128), dG = floor256(88 * U + 183 * V + 128), dB = floor256(454 * U + 128);
    uint32_t px[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int Y = (int)((luma >> (8 * k)) & 0xFFu);
        px[k] = (uint32_t)clamp8(Y + dR) | ((uint32_t)clamp8(Y - dG) << 8) | ((uint32_t)clamp8(Y + dB) << 16) |
                (A << 24);
    }
    const int x = 2 * bx;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int y = 2 * by + r;
        if (y >= h) continue;
        uint32_t* row = dst + (size_t)y * pitch;
        if (vec && x + 1 < w) {
            __stcs(reinterpret_cast<uint2*>(row + x), make_uint2(px[2 * r], px[2 * r + 1]));
        } else {
            __stcs(row + x, px[2 * r]);
            if (x + 1 < w) __stcs(row + x + 1, px[2 * r + 1]);
        }
    }
}

template <int N, bool ENC>
cudaError_t launch_n(const YuvJob* jobs, int n, uint32_t tiles, cudaStream_t s)
{
    YuvJobList<N> J;
    J.n = n;
    for (int i = 0; i < n; ++i) J.j[i] = jobs[i];
    if (ENC) k_yuv_encode<N><<<tiles, dim3(kYX, kYY), 0, s>>>(J);
    else k_yuv_decode<N><<<tiles, dim3(kYX, kYY), 0, s>>>(J);
    return cudaGetLastError();
}

}  // namespace

// Fills first/tiles_x of every job and launches (at most kYuvJobsPerLaunch jobs).
cudaError_t launch_yuv(YuvJob* jobs, int n, bool encode, cudaStream_t s)
{
    uint32_t tiles = 0;
    int m = 0;
    for (int i = 0; i < n; ++i) {
        const int bw = (jobs[i].w + 1) / 2, bh = (jobs[i].h + 1) / 2;
        if (bw <= 0 || bh <= 0) continue;
        jobs[m] = jobs[i];
        jobs[m].tiles_x = (uint32_t)((bw + kYX - 1) / kYX);
        jobs[m].first = tiles;
        tiles += jobs[m].tiles_x * (uint32_t)((bh + kYY - 1) / kYY);
        ++m;
    }
    if (m == 0) return cudaSuccess;
    if (m <= 8) return encode ? launch_n<8, true>(jobs, m, tiles, s) : launch_n<8, false>(jobs, m, tiles, s);
    return encode ? launch_n<kYuvJobsPerLaunch, true>(jobs, m, tiles, s)
                  : launch_n<kYuvJobsPerLaunch, false>(jobs, m, tiles, s);
}

}  // namespace ec
