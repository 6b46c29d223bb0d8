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
// Each thread owns NP pairs of horizontally adjacent blocks, 32 pairs apart,
// so every load instruction of a warp covers 512 contiguous bytes.  A row
// pair of two blocks is one 16-byte access, and their two luma or chroma
// words one 8-byte access, where the buffers allow it.  All of a thread's
// loads are issued before any result is computed.  One block per thread left
// HBM idle between waves of short loads; the decoder takes two pairs per
// thread, the encoder one (a second pair's registers cost it more occupancy
// than its loads gain).  A launch covers many images: CTA tiles of 32 NP
// pairs x 8 block rows are numbered across the images and each CTA finds its
// image by a binary search of the images' first tiles.  Both kernels are
// HBM-bound: 4 bytes read and 2 written per pixel to encode, the reverse to
// decode.
#include "ec_internal.cuh"

namespace ec {
namespace {

constexpr int kYX = 32, kYY = 8;     // threads per CTA: 32 x 8
constexpr int kEncNP = 1, kDecNP = 2; // block pairs per thread
constexpr int kVec8 = 1, kVec16 = 2, kPacked8 = 4;   // YuvJob::vec bits

// floor(x / 256) for x > -2^20
__device__ __forceinline__ int floor256(int x) { return ((x + (1 << 20)) >> 8) - (1 << 12); }
__device__ __forceinline__ int clamp8(int v) { return min(255, max(0, v)); }

// The three weighted sums are byte dot products of the pixel word (R, G, B,
// A in bytes 0..3) with unsigned coefficient bytes: 77R + 150G + 29B for Y,
// and the negative parts 43R + 85G of U and 107G + 21B of V, whose positive
// part is 128 times one channel.  Integer arithmetic, exact.
__device__ __forceinline__ void to_yuv(uint32_t p, int& Y, int& U, int& V)
{
    const int R = (int)(p & 0xFFu), B = (int)((p >> 16) & 0xFFu);
    Y = (int)__dp4a(p, 0x001D964Du, 128u) >> 8;                              // (77, 150, 29, 0)
    U = min(255, ((B << 7) - (int)__dp4a(p, 0x0000552Bu, 0u) + 32896) >> 8);   // (43, 85, 0, 0)
    V = min(255, ((R << 7) - (int)__dp4a(p, 0x00156B00u, 0u) + 32896) >> 8);   // (0, 107, 21, 0)
}

// CTA tile t of a job list: the job whose tiles [first, first + ntiles) hold
// it; bp = the thread's first block pair (its others follow 32 pairs apart),
// by = its block row.
template <int NP, int N>
__device__ __forceinline__ const YuvJob& tile_job(const YuvJobList<N>& J, uint32_t t, int& bp, int& by)
{
    int lo = 0, hi = J.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (J.j[mid].first <= t) lo = mid;
        else hi = mid - 1;
    }
    const YuvJob& jb = J.j[lo];
    const uint32_t r = t - jb.first, tx = r % jb.tiles_x;
    bp = (int)(tx * kYX * NP) + threadIdx.x;
    by = (int)((r / jb.tiles_x) * kYY) + threadIdx.y;
    return jb;
}

// The up to four pixels of block column b (pixel k at (2b + (k & 1), 2by + (k >> 1))).
__device__ __forceinline__ void load_block(const uint32_t* src, int pitch, int w, int h, int b, int by, bool vec8,
                                           uint32_t (&px)[4], bool (&has)[4])
{
    const int x = 2 * b;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int y = 2 * by + r;
        has[2 * r] = has[2 * r + 1] = false;
        px[2 * r] = px[2 * r + 1] = 0u;
        if (y >= h) continue;
        const uint32_t* row = src + (size_t)y * pitch;
        if (vec8 && x + 1 < w) {
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
}

// Luma word and chroma word (U, V, A, 0) of one block.
__device__ __forceinline__ void encode_block(const uint32_t (&px)[4], const bool (&has)[4], uint32_t& luma,
                                             uint32_t& chroma)
{
    luma = 0u;
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
    chroma = (uint32_t)((su + half) >> sh) | ((uint32_t)((sv + half) >> sh) << 8) |
             ((uint32_t)((sa + half) >> sh) << 16);
}

// Whole 2x2 blocks (the interior of an image): the same sums with no
// per-pixel presence tests.  Y is byte 1 of its dot product (which is below
// 2^16), so four of them pack into the luma word with three byte permutes;
// the alpha sum is one more byte dot product per pixel.
__device__ __forceinline__ uint32_t u_of(uint32_t p)
{
    return min(255u, (((p >> 9) & 0x7F80u) - __dp4a(p, 0x0000552Bu, 0u) + 32896u) >> 8);
}

__device__ __forceinline__ uint32_t v_of(uint32_t p)
{
    return min(255u, (((p << 7) & 0x7F80u) - __dp4a(p, 0x00156B00u, 0u) + 32896u) >> 8);
}

__device__ __forceinline__ void encode_full(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t& luma,
                                            uint32_t& chroma)
{
    const uint32_t ab = __byte_perm(__dp4a(a, 0x001D964Du, 128u), __dp4a(b, 0x001D964Du, 128u), 0x0051);
    const uint32_t cd = __byte_perm(__dp4a(c, 0x001D964Du, 128u), __dp4a(d, 0x001D964Du, 128u), 0x0051);
    luma = __byte_perm(ab, cd, 0x5410);
    const uint32_t su = u_of(a) + u_of(b) + u_of(c) + u_of(d);
    const uint32_t sv = v_of(a) + v_of(b) + v_of(c) + v_of(d);
    const uint32_t sa = __dp4a(a, 0x01000000u, __dp4a(b, 0x01000000u, __dp4a(c, 0x01000000u, __dp4a(d, 0x01000000u, 0u))));
    chroma = ((su + 2u) >> 2) | (((sv + 2u) >> 2) << 8) | (((sa + 2u) >> 2) << 16);
}

template <int N>
__global__ void __launch_bounds__(kYX * kYY)
k_yuv_encode(const __grid_constant__ YuvJobList<N> J)
{
    constexpr int kNP = kEncNP;
    int bp, by;
    const YuvJob& jb = tile_job<kNP>(J, blockIdx.x, bp, by);
    const uint32_t* __restrict__ src = jb.src;
    uint32_t* __restrict__ dst = jb.dst;
    const int w = jb.w, h = jb.h, pitch = jb.pitch, dpitch = jb.dpitch, vec = jb.vec;
    const int bw = (w + 1) >> 1, bh = (h + 1) >> 1;
    if (by >= bh) return;
    if (kNP == 1 && (vec & kVec16) && (vec & kPacked8) && 4 * bp + 3 < w && 2 * by + 1 < h) {
        // a pair of whole blocks: two 16-byte loads, two 8-byte stores
        const uint4 r0 = __ldcs(reinterpret_cast<const uint4*>(src + (size_t)(2 * by) * pitch + 4 * bp));
        const uint4 r1 = __ldcs(reinterpret_cast<const uint4*>(src + (size_t)(2 * by + 1) * pitch + 4 * bp));
        uint32_t l0, c0, l1, c1;
        encode_full(r0.x, r0.y, r1.x, r1.y, l0, c0);
        encode_full(r0.z, r0.w, r1.z, r1.w, l1, c1);
        *reinterpret_cast<uint2*>(dst + (size_t)by * dpitch + 2 * bp) = make_uint2(l0, l1);
        *reinterpret_cast<uint2*>(dst + (size_t)(bh + by) * dpitch + 2 * bp) = make_uint2(c0, c1);
        return;
    }
    uint32_t p0[kNP][4], p1[kNP][4];
    bool h0[kNP][4], h1[kNP][4];
#pragma unroll
    for (int q = 0; q < kNP; ++q) {              // every load first
        const int b0 = 2 * (bp + 32 * q), x = 2 * b0;
        if (b0 >= bw) continue;
        if ((vec & kVec16) && x + 3 < w) {
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int y = 2 * by + r;
                const bool in = y < h;
                const uint4 v = in ? __ldcs(reinterpret_cast<const uint4*>(src + (size_t)y * pitch + x))
                                   : make_uint4(0u, 0u, 0u, 0u);
                p0[q][2 * r] = v.x; p0[q][2 * r + 1] = v.y; p1[q][2 * r] = v.z; p1[q][2 * r + 1] = v.w;
                h0[q][2 * r] = h0[q][2 * r + 1] = h1[q][2 * r] = h1[q][2 * r + 1] = in;
            }
        } else {
            load_block(src, pitch, w, h, b0, by, vec & kVec8, p0[q], h0[q]);
            if (b0 + 1 < bw) load_block(src, pitch, w, h, b0 + 1, by, vec & kVec8, p1[q], h1[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < kNP; ++q) {
        const int b0 = 2 * (bp + 32 * q);
        if (b0 >= bw) continue;
        const bool two = b0 + 1 < bw;
        uint32_t l0, c0, l1 = 0u, c1 = 0u;
        encode_block(p0[q], h0[q], l0, c0);
        if (two) encode_block(p1[q], h1[q], l1, c1);
        uint32_t* lrow = dst + (size_t)by * dpitch + b0;
        uint32_t* crow = dst + (size_t)(bh + by) * dpitch + b0;
        if (two && (vec & kPacked8)) {
            *reinterpret_cast<uint2*>(lrow) = make_uint2(l0, l1);
            *reinterpret_cast<uint2*>(crow) = make_uint2(c0, c1);
        } else {
            lrow[0] = l0;
            crow[0] = c0;
            if (two) {
                lrow[1] = l1;
                crow[1] = c1;
            }
        }
    }
}

// The four RGBA8 pixels of one block from its luma and chroma words.
__device__ __forceinline__ void decode_block(uint32_t luma, uint32_t ch, uint32_t (&px)[4])
{
    const int U = (int)(ch & 0xFFu) - 128, V = (int)((ch >> 8) & 0xFFu) - 128;
    const uint32_t A = (ch >> 16) & 0xFFu;
    const int dR = floor256(359 * V + 128), dG = floor256(88 * U + 183 * V + 128), dB = floor256(454 * U + 128);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int Y = (int)((luma >> (8 * k)) & 0xFFu);
        px[k] = (uint32_t)clamp8(Y + dR) | ((uint32_t)clamp8(Y - dG) << 8) | ((uint32_t)clamp8(Y + dB) << 16) |
                (A << 24);
    }
}

__device__ __forceinline__ void store_block(uint32_t* dst, int pitch, int w, int h, int b, int by, bool vec8,
                                            const uint32_t (&px)[4])
{
    const int x = 2 * b;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int y = 2 * by + r;
        if (y >= h) continue;
        uint32_t* row = dst + (size_t)y * pitch;
        if (vec8 && x + 1 < w) {
            __stcs(reinterpret_cast<uint2*>(row + x), make_uint2(px[2 * r], px[2 * r + 1]));
        } else {
            __stcs(row + x, px[2 * r]);
            if (x + 1 < w) __stcs(row + x + 1, px[2 * r + 1]);
        }
    }
}

template <int N>
__global__ void __launch_bounds__(kYX * kYY)
k_yuv_decode(const __grid_constant__ YuvJobList<N> J)
{
    constexpr int kNP = kDecNP;
    int bp, by;
    const YuvJob& jb = tile_job<kNP>(J, blockIdx.x, bp, by);
    const uint32_t* __restrict__ src = jb.src;
    uint32_t* __restrict__ dst = jb.dst;
    const int w = jb.w, h = jb.h, pitch = jb.pitch, spitch = jb.dpitch, vec = jb.vec;
    const int bw = (w + 1) >> 1, bh = (h + 1) >> 1;
    if (by >= bh) return;
    uint32_t l0[kNP], c0[kNP], l1[kNP], c1[kNP];
#pragma unroll
    for (int q = 0; q < kNP; ++q) {              // every load first
        const int b0 = 2 * (bp + 32 * q);
        l0[q] = c0[q] = l1[q] = c1[q] = 0u;
        if (b0 >= bw) continue;
        const uint32_t* lrow = src + (size_t)by * spitch + b0;
        const uint32_t* crow = src + (size_t)(bh + by) * spitch + b0;
        if (b0 + 1 < bw && (vec & kPacked8)) {
            const uint2 l = __ldcs(reinterpret_cast<const uint2*>(lrow));
            const uint2 c = __ldcs(reinterpret_cast<const uint2*>(crow));
            l0[q] = l.x; l1[q] = l.y; c0[q] = c.x; c1[q] = c.y;
        } else {
            l0[q] = __ldcs(lrow);
            c0[q] = __ldcs(crow);
            if (b0 + 1 < bw) {
                l1[q] = __ldcs(lrow + 1);
                c1[q] = __ldcs(crow + 1);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kNP; ++q) {
        const int b0 = 2 * (bp + 32 * q), x = 2 * b0;
        if (b0 >= bw) continue;
        uint32_t p0[4], p1[4];
        decode_block(l0[q], c0[q], p0);
        decode_block(l1[q], c1[q], p1);
        if ((vec & kVec16) && x + 3 < w) {
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int y = 2 * by + r;
                if (y < h)
                    __stcs(reinterpret_cast<uint4*>(dst + (size_t)y * pitch + x),
                           make_uint4(p0[2 * r], p0[2 * r + 1], p1[2 * r], p1[2 * r + 1]));
            }
        } else {
            store_block(dst, pitch, w, h, b0, by, vec & kVec8, p0);
            if (b0 + 1 < bw) store_block(dst, pitch, w, h, b0 + 1, by, vec & kVec8, p1);
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
        const int per = 2 * kYX * (encode ? kEncNP : kDecNP);   // block columns per CTA tile
        jobs[m].tiles_x = (uint32_t)((bw + per - 1) / per);
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
