// k_assemble.cu -- assembly of the compound modes other than sort-last
// (thesis 4.2): sort-first and tile compounds copy complete pixels into place,
// pixel compounds interleave the sources' pixels over a pixel kernel, and
// subpixel compounds average every pixel's samples.
//
// All three are streaming copies / reductions: every thread owns one 16-byte
// group of output pixels (4 RGBA8, 2 RGBA16F or 1 RGBA32F pixels) of a
// 32-group x 8-row tile, reads each contributing source pixel once (16-byte
// loads where the layout allows) and writes the group once.  HBM-bound.
#include "composite_body.cuh"

#include <algorithm>

namespace ec {
namespace {

constexpr int kAT = 256;
constexpr int kARows = kAT / 32;          // rows a CTA covers at once
constexpr int kAPasses = 4;                 // row passes per CTA (average and pixel kernels)
constexpr int kTPasses = 2;                 // row passes per CTA (tile kernel)

template <int BPP> struct Grp;                 // one 16-byte group of pixels
template <> struct Grp<4> { static constexpr int PX = 4; };
template <> struct Grp<8> { static constexpr int PX = 2; };
template <> struct Grp<16> { static constexpr int PX = 1; };

// Pixel j of a 16-byte group as raw 32-bit words (BPP / 4 of them).
template <int BPP>
__device__ __forceinline__ void load_px(const uint8_t* p, uint32_t* w)
{
    if constexpr (BPP == 4) w[0] = __ldcs(reinterpret_cast<const uint32_t*>(p));
    else if constexpr (BPP == 8) {
        const uint2 v = __ldcs(reinterpret_cast<const uint2*>(p));
        w[0] = v.x; w[1] = v.y;
    } else {
        const uint4 v = __ldcs(reinterpret_cast<const uint4*>(p));
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    }
}

template <int BPP>
__device__ __forceinline__ void store_px(uint8_t* p, const uint32_t* w)
{
    if constexpr (BPP == 4) *reinterpret_cast<uint32_t*>(p) = w[0];
    else if constexpr (BPP == 8) *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
    else *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}

// Bit j set when pixel x + j of row y lies in the source's clipped roi.
template <int PX>
__device__ __forceinline__ uint32_t covered(const SrcDesc& s, int x, int y, int W)
{
    if (y < s.y0 || y >= s.y1) return 0u;
    uint32_t m = 0;
#pragma unroll
    for (int j = 0; j < PX; ++j)
        if (x + j >= s.x0 && x + j < s.x1 && x + j < W) m |= 1u << j;
    return m;
}

// ---- sort-first / tile assembly -----------------------------------------

// Up to 64 sources: which sources meet each column and each row of CTA tiles,
// as bit masks (bit i: source i), computed on the host.  A tile's sources are
// its column's mask and its row's, so a CTA finds them with two uniform
// parameter reads instead of testing every source.
constexpr int kMaskCols = 128, kMaskRows = 512;
struct TileMasks {
    uint64_t col[kMaskCols];
    uint64_t row[kMaskRows];
};

// MASK: the sources come from the tile masks (n <= 64), else each CTA lists
// them (build_active).  Every pixel walks them from last to first and stops
// once its 16-byte group is complete.
template <int N, int BPP, bool MASK>
__global__ void __launch_bounds__(kAT, 8)
k_assemble_tiles(const __grid_constant__ SrcList<N> L, const __grid_constant__ DstDesc D,
                 const __grid_constant__ TileMasks M)
{
    constexpr int PX = Grp<BPP>::PX, TW = 32 * PX, WPP = BPP / 4;
    __shared__ int16_t act[MASK ? 1 : (N > 0 ? N : 1)];
    __shared__ int nact_s;
    const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
    const int tx0 = blockIdx.x * TW, ty0 = blockIdx.y * (kARows * kTPasses);
    uint64_t amask = 0;
    if (MASK) {
        amask = M.col[blockIdx.x] & M.row[blockIdx.y];
    } else {
        auto at = [&](int, int i) -> const SrcDesc& { return L.s[i]; };
        build_active(at, L.n, tx0, ty0, min(tx0 + TW, D.W), min(ty0 + kARows * kTPasses, D.H), act, &nact_s);
        __syncthreads();
    }
    const int x = tx0 + lane * PX;
    if (x >= D.W) return;
    const uint32_t full = x + PX <= D.W ? (1u << PX) - 1u : (1u << (D.W - x)) - 1u;
    uint32_t fast = 0;                                   // passes already written
    if (MASK && PX * BPP == 16 && D.vec && full == (1u << PX) - 1u) {
        // groups that one source covers whole (the usual case): every such
        // pass's 16-byte load is issued before any store
        const uint4* fp[kTPasses];
#pragma unroll
        for (int pass = 0; pass < kTPasses; ++pass) {
            fp[pass] = nullptr;
            const int y = ty0 + pass * kARows + row;
            if (y >= D.H) continue;
            for (uint64_t mm = amask; mm;) {
                const int i = 63 - __clzll((long long)mm);
                mm ^= 1ull << i;
                const SrcDesc& s = L.s[i];
                const uint32_t m = covered<PX>(s, x, y, D.W);
                if (!m) continue;
                if (m == full && s.vec) {
                    const size_t e = (size_t)(y - s.oy) * (size_t)s.pitch + (size_t)(x - s.ox);
                    fp[pass] = reinterpret_cast<const uint4*>(reinterpret_cast<const uint8_t*>(s.color) + e * BPP);
                    fast |= 1u << pass;
                }
                break;
            }
        }
        uint4 v[kTPasses];
#pragma unroll
        for (int pass = 0; pass < kTPasses; ++pass)
            if ((fast >> pass) & 1u) v[pass] = __ldcs(fp[pass]);
#pragma unroll
        for (int pass = 0; pass < kTPasses; ++pass) {
            if (!((fast >> pass) & 1u)) continue;
            const int y = ty0 + pass * kARows + row;
            __stcs(reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(D.color) + ((size_t)y * (size_t)D.pitch + (size_t)x) * BPP),
                   v[pass]);
        }
    }
    for (int pass = 0; pass < kTPasses; ++pass) {
    const int y = ty0 + pass * kARows + row;
    if (y >= D.H) break;
    if ((fast >> pass) & 1u) continue;
    uint32_t w[PX][WPP];
    uint32_t have = 0;
    // the last source covering a pixel wins: walk back until every pixel is set
    uint64_t mm = amask;
    for (int a = MASK ? 0 : nact_s - 1; have != full; --a) {
        int i;
        if (MASK) {
            if (!mm) break;
            i = 63 - __clzll((long long)mm);
            mm ^= 1ull << i;
        } else {
            if (a < 0) break;
            i = act[a];
        }
        const SrcDesc& s = L.s[i];
        const uint32_t m = covered<PX>(s, x, y, D.W) & ~have;
        if (!m) continue;
        const size_t e = (size_t)(y - s.oy) * (size_t)s.pitch + (size_t)(x - s.ox);
        const uint8_t* p = reinterpret_cast<const uint8_t*>(s.color) + e * BPP;
        if (m == full && s.vec && PX * BPP == 16 && full == (1u << PX) - 1u) {
            const uint4 v = __ldcs(reinterpret_cast<const uint4*>(p));
            const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < PX; ++j)
#pragma unroll
                for (int k = 0; k < WPP; ++k) w[j][k] = vv[j * WPP + k];
        } else {
#pragma unroll
            for (int j = 0; j < PX; ++j)
                if ((m >> j) & 1u) load_px<BPP>(p + j * BPP, w[j]);
        }
        have |= m;
    }
    if (!have) continue;
    uint8_t* o = reinterpret_cast<uint8_t*>(D.color) + ((size_t)y * (size_t)D.pitch + (size_t)x) * BPP;
    if (have == (1u << PX) - 1u && D.vec) {
        uint32_t vv[4];
#pragma unroll
        for (int j = 0; j < PX; ++j)
#pragma unroll
            for (int k = 0; k < WPP; ++k) vv[j * WPP + k] = w[j][k];
        __stcs(reinterpret_cast<uint4*>(o), make_uint4(vv[0], vv[1], vv[2], vv[3]));
    } else {
#pragma unroll
        for (int j = 0; j < PX; ++j)
            if ((have >> j) & 1u) store_px<BPP>(o + j * BPP, w[j]);
    }
    }
}

// ---- subpixel average ------------------------------------------------------

// FMT: 0 RGBA8 (integer sums, (sum + count/2) / count), 1 RGBA32F, 2 RGBA16F
// (FP32 sums in input order, divided by the count).  Sources are read four
// at a time, all four groups in flight before any is added.
template <int N, int FMT>
__global__ void __launch_bounds__(kAT)
k_average(const __grid_constant__ SrcList<N> L, const __grid_constant__ DstDesc D)
{
    constexpr int BPP = FMT == 0 ? 4 : FMT == 1 ? 16 : 8, PX = Grp<BPP>::PX, WPP = BPP / 4, B = 4;
    __shared__ int16_t act[N > 0 ? N : 1];
    __shared__ int nact_s;
    auto at = [&](int, int i) -> const SrcDesc& { return L.s[i]; };
    const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
    const int tx0 = blockIdx.x * (32 * PX), ty0 = blockIdx.y * (kARows * kAPasses);
    const int tx1 = min(tx0 + 32 * PX, D.W), ty1 = min(ty0 + kARows * kAPasses, D.H);
    build_active(at, L.n, tx0, ty0, tx1, ty1, act, &nact_s);
    __syncthreads();
    const int nact = nact_s;
    // every active source covers the whole tile with 16-byte rows: no per-pixel masks
    bool cov = true;
    for (int a = threadIdx.x; a < nact; a += kAT) {
        const SrcDesc& s = L.s[act[a]];
        cov = cov && s.vec && s.x0 <= tx0 && s.x1 >= tx1 && s.y0 <= ty0 && s.y1 >= ty1;
    }
    const bool full = __syncthreads_and(cov) && tx1 - tx0 == 32 * PX;
    const int x = tx0 + lane * PX;
    if (x >= D.W) return;
    for (int pass = 0; pass < kAPasses; ++pass) {
        const int y = ty0 + pass * kARows + row;
        if (y >= D.H) break;
        uint32_t isum[PX][4];
        uint32_t lo[PX], hi[PX];            // RGBA8: channels 0,2 and 1,3 as 16-bit lanes
        float fsum[PX][4];
        int cnt[PX];
#pragma unroll
        for (int j = 0; j < PX; ++j) {
            cnt[j] = 0;
            lo[j] = hi[j] = 0u;
#pragma unroll
            for (int c = 0; c < 4; ++c) { isum[j][c] = 0u; fsum[j][c] = 0.0f; }
        }
        auto fold = [&]() {                 // 16-bit lanes into the 32-bit sums
#pragma unroll
            for (int j = 0; j < PX; ++j) {
                isum[j][0] += lo[j] & 0xFFFFu; isum[j][2] += lo[j] >> 16;
                isum[j][1] += hi[j] & 0xFFFFu; isum[j][3] += hi[j] >> 16;
                lo[j] = hi[j] = 0u;
            }
        };
        for (int a0 = 0; a0 < nact; a0 += B) {
            if (FMT == 0 && a0 % 256 == 0 && a0) fold();   // at most 256 * 255 per lane
            uint32_t w[B][PX][WPP];
            uint32_t m[B];
#pragma unroll
            for (int b = 0; b < B; ++b) {
                m[b] = 0u;
                if (a0 + b >= nact) continue;
                const SrcDesc& s = L.s[act[a0 + b]];
                m[b] = full ? (1u << PX) - 1u : covered<PX>(s, x, y, D.W);
                if (!m[b]) continue;
                const size_t e = (size_t)(y - s.oy) * (size_t)s.pitch + (size_t)(x - s.ox);
                const uint8_t* p = reinterpret_cast<const uint8_t*>(s.color) + e * BPP;
                if (m[b] == (1u << PX) - 1u && s.vec) {
                    const uint4 v = __ldcs(reinterpret_cast<const uint4*>(p));
                    const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int j = 0; j < PX; ++j)
#pragma unroll
                        for (int k = 0; k < WPP; ++k) w[b][j][k] = vv[j * WPP + k];
                } else {
#pragma unroll
                    for (int j = 0; j < PX; ++j)
                        if ((m[b] >> j) & 1u) load_px<BPP>(p + j * BPP, w[b][j]);
                }
            }
#pragma unroll
            for (int b = 0; b < B; ++b) {
#pragma unroll
                for (int j = 0; j < PX; ++j) {
                    if (!((m[b] >> j) & 1u)) continue;
                    ++cnt[j];
                    if constexpr (FMT == 0) {
                        lo[j] += w[b][j][0] & 0x00FF00FFu;
                        hi[j] += (w[b][j][0] >> 8) & 0x00FF00FFu;
                    } else if constexpr (FMT == 1) {
#pragma unroll
                        for (int c = 0; c < 4; ++c) fsum[j][c] += __uint_as_float(w[b][j][c]);
                    } else {
                        const float4 f = half4_to_float4(make_uint2(w[b][j][0], w[b][j][1]));
                        fsum[j][0] += f.x; fsum[j][1] += f.y; fsum[j][2] += f.z; fsum[j][3] += f.w;
                    }
                }
            }
        }
        if (FMT == 0) fold();
        uint32_t out[PX][WPP];
#pragma unroll
        for (int j = 0; j < PX; ++j) {
            const int n = cnt[j];
            if constexpr (FMT == 0) {
                uint32_t v = 0;
                if (n) {
                    // (sum + n/2) / n: a float estimate, exact after a +-1 correction
                    // (the numerator is < 2^18, so the estimate is off by < 1e-4)
                    const uint32_t un = (uint32_t)n;
                    const float r = 1.0f / (float)n;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const uint32_t x = isum[j][c] + un / 2u;
                        uint32_t q = (uint32_t)((float)x * r);
                        if (q * un > x) --q;
                        else if ((q + 1u) * un <= x) ++q;
                        v |= q << (8 * c);
                    }
                }
                out[j][0] = v;
            } else {
                float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
                if (n) {
                    const float fn = (float)n;
                    f = make_float4(fsum[j][0] / fn, fsum[j][1] / fn, fsum[j][2] / fn, fsum[j][3] / fn);
                }
                if constexpr (FMT == 1) {
                    out[j][0] = __float_as_uint(f.x); out[j][1] = __float_as_uint(f.y);
                    out[j][2] = __float_as_uint(f.z); out[j][3] = __float_as_uint(f.w);
                } else {
                    const uint2 h = float4_to_half4(f);
                    out[j][0] = h.x; out[j][1] = h.y;
                }
            }
        }
        uint8_t* o = reinterpret_cast<uint8_t*>(D.color) + ((size_t)y * (size_t)D.pitch + (size_t)x) * BPP;
        if (x + PX <= D.W && D.vec) {
            uint32_t vv[4];
#pragma unroll
            for (int j = 0; j < PX; ++j)
#pragma unroll
                for (int k = 0; k < WPP; ++k) vv[j * WPP + k] = out[j][k];
            __stcs(reinterpret_cast<uint4*>(o), make_uint4(vv[0], vv[1], vv[2], vv[3]));
        } else {
#pragma unroll
            for (int j = 0; j < PX; ++j)
                if (x + j < D.W) store_px<BPP>(o + j * BPP, out[j]);
        }
    }
}

// ---- pixel compound --------------------------------------------------------

template <int N, int BPP>
__global__ void __launch_bounds__(kAT)
k_assemble_pixels(const __grid_constant__ PixList<N> P, const __grid_constant__ DstDesc D)
{
    constexpr int PX = Grp<BPP>::PX, WPP = BPP / 4;
    const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
    const int x = blockIdx.x * (32 * PX) + lane * PX;
    if (x >= D.W) return;
    const int i00 = x / P.nx, rx00 = x - i00 * P.nx;    // one division; then step the residue
    // kAPasses rows per thread, every load issued before any store
    uint32_t w[kAPasses][PX][WPP];
    uint32_t have[kAPasses];
#pragma unroll
    for (int pass = 0; pass < kAPasses; ++pass) {
        const int y = blockIdx.y * (kARows * kAPasses) + pass * kARows + row;
        have[pass] = 0u;
        if (y >= D.H) continue;
        const int ry = y % P.ny, j0 = y / P.ny;
        int rx = rx00, i0 = i00;
#pragma unroll
        for (int j = 0; j < PX; ++j) {
            const int xj = x + j;
            const int k = xj < D.W ? P.owner[ry * P.nx + rx] : -1;
            if (k >= 0) {
                const PixSrc& s = P.s[k];
                const size_t e = (size_t)j0 * (size_t)s.pitch + (size_t)i0;
                load_px<BPP>(reinterpret_cast<const uint8_t*>(s.color) + e * BPP, w[pass][j]);
                have[pass] |= 1u << j;
            }
            if (++rx == P.nx) { rx = 0; ++i0; }
        }
    }
#pragma unroll
    for (int pass = 0; pass < kAPasses; ++pass) {
        if (!have[pass]) continue;
        const int y = blockIdx.y * (kARows * kAPasses) + pass * kARows + row;
        uint8_t* o = reinterpret_cast<uint8_t*>(D.color) + ((size_t)y * (size_t)D.pitch + (size_t)x) * BPP;
        if (have[pass] == (1u << PX) - 1u && D.vec) {
            uint32_t vv[4];
#pragma unroll
            for (int j = 0; j < PX; ++j)
#pragma unroll
                for (int k = 0; k < WPP; ++k) vv[j * WPP + k] = w[pass][j][k];
            __stcs(reinterpret_cast<uint4*>(o), make_uint4(vv[0], vv[1], vv[2], vv[3]));
        } else {
#pragma unroll
            for (int j = 0; j < PX; ++j)
                if ((have[pass] >> j) & 1u) store_px<BPP>(o + j * BPP, w[pass][j]);
        }
    }
}

template <int N>
SrcList<N> make_src_list(const SrcDesc* src, int n)
{
    SrcList<N> L;
    L.n = n;
    L.pad[0] = L.pad[1] = L.pad[2] = 0;
    for (int i = 0; i < n; ++i) L.s[i] = src[i];
    return L;
}

template <int N, int BPP, bool MASK>
void tiles_launch(const SrcList<N>& L, const DstDesc& D, const TileMasks& M, dim3 grid, cudaStream_t s)
{
    k_assemble_tiles<N, BPP, MASK><<<grid, kAT, 0, s>>>(L, D, M);
}

template <int N, bool MASK>
void tiles_bpp(const SrcList<N>& L, int bpp, const DstDesc& D, const TileMasks& M, dim3 grid, cudaStream_t s)
{
    if (bpp == 4) tiles_launch<N, 4, MASK>(L, D, M, grid, s);
    else if (bpp == 8) tiles_launch<N, 8, MASK>(L, D, M, grid, s);
    else tiles_launch<N, 16, MASK>(L, D, M, grid, s);
}

template <int N>
cudaError_t tiles_n(const SrcDesc* src, int n, int bpp, const DstDesc& D, cudaStream_t s)
{
    const SrcList<N> L = make_src_list<N>(src, n);
    const int tw = 32 * (16 / bpp), th = kARows * kTPasses;
    const dim3 grid(ceil_div(D.W, tw), ceil_div(D.H, th));
    static thread_local TileMasks M;
    if (N <= 64 && grid.x <= (unsigned)kMaskCols && grid.y <= (unsigned)kMaskRows) {
        for (unsigned c = 0; c < grid.x; ++c) M.col[c] = 0;
        for (unsigned r = 0; r < grid.y; ++r) M.row[r] = 0;
        for (int i = 0; i < n; ++i) {
            const SrcDesc& d = src[i];
            const int x0 = std::max(d.x0, 0), x1 = std::min(d.x1, D.W);
            const int y0 = std::max(d.y0, 0), y1 = std::min(d.y1, D.H);
            if (x0 >= x1 || y0 >= y1) continue;
            for (int c = x0 / tw; c < ceil_div(x1, tw); ++c) M.col[c] |= 1ull << i;
            for (int r = y0 / th; r < ceil_div(y1, th); ++r) M.row[r] |= 1ull << i;
        }
        tiles_bpp<N, true>(L, bpp, D, M, grid, s);
    } else {
        tiles_bpp<N, false>(L, bpp, D, M, grid, s);
    }
    return cudaGetLastError();
}

template <int N>
cudaError_t average_n(const SrcDesc* src, int n, int fmt, const DstDesc& D, cudaStream_t s)
{
    const SrcList<N> L = make_src_list<N>(src, n);
    const int px = fmt == 0 ? 4 : fmt == 1 ? 1 : 2;
    const dim3 grid(ceil_div(D.W, 32 * px), ceil_div(D.H, kARows * kAPasses));
    if (fmt == 0) k_average<N, 0><<<grid, kAT, 0, s>>>(L, D);
    else if (fmt == 1) k_average<N, 1><<<grid, kAT, 0, s>>>(L, D);
    else k_average<N, 2><<<grid, kAT, 0, s>>>(L, D);
    return cudaGetLastError();
}

template <int N>
cudaError_t pixels_n(const PixSrc* src, const int16_t* owner, int n, int nx, int ny, int bpp,
                     const DstDesc& D, cudaStream_t s)
{
    PixList<N> P;
    P.n = n;
    P.nx = nx;
    P.ny = ny;
    P.pad = 0;
    for (int i = 0; i < n; ++i) P.s[i] = src[i];
    for (int i = 0; i < nx * ny; ++i) P.owner[i] = owner[i];
    const int px = 16 / bpp;
    const dim3 grid(ceil_div(D.W, 32 * px), ceil_div(D.H, kARows * kAPasses));
    if (bpp == 4) k_assemble_pixels<N, 4><<<grid, kAT, 0, s>>>(P, D);
    else if (bpp == 8) k_assemble_pixels<N, 8><<<grid, kAT, 0, s>>>(P, D);
    else k_assemble_pixels<N, 16><<<grid, kAT, 0, s>>>(P, D);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_assemble_tiles(const SrcDesc* src, int n, int bpp, const DstDesc& D, cudaStream_t s)
{
    if (D.W <= 0 || D.H <= 0 || n <= 0) return cudaSuccess;
    if (n <= 16) return tiles_n<16>(src, n, bpp, D, s);
    if (n <= 64) return tiles_n<64>(src, n, bpp, D, s);
    return tiles_n<EC_MAX_SOURCES>(src, n, bpp, D, s);
}

cudaError_t launch_average(const SrcDesc* src, int n, int fmt, const DstDesc& D, cudaStream_t s)
{
    if (D.W <= 0 || D.H <= 0) return cudaSuccess;
    if (n <= 16) return average_n<16>(src, n, fmt, D, s);
    if (n <= 64) return average_n<64>(src, n, fmt, D, s);
    return average_n<EC_MAX_SOURCES>(src, n, fmt, D, s);
}

cudaError_t launch_assemble_pixels(const PixSrc* src, const int16_t* owner, int n, int nx, int ny, int bpp,
                                   const DstDesc& D, cudaStream_t s)
{
    if (D.W <= 0 || D.H <= 0 || n <= 0) return cudaSuccess;
    if (n <= 16) return pixels_n<16>(src, owner, n, nx, ny, bpp, D, s);
    return pixels_n<kPixMaxSources>(src, owner, n, nx, ny, bpp, D, s);
}

}  // namespace ec
