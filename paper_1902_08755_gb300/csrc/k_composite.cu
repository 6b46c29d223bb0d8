// k_composite.cu -- one launch per destination frame: depth merge (thesis
// 5.2.1, depth-sorted compositing; 3.6 unordered compositing) and ordered
// front-to-back "over" (thesis 5.2.1, spatial compositing), both restricted to
// each input's ROI (thesis 5.3).
//
// Design: the work is a streaming read of every input pixel inside its ROI
// plus one write of the output, so the kernels are HBM-bound.  A CTA owns a
// tile of output pixels and first intersects every input's ROI with its tile
// (one warp, ballot + popc compaction into shared memory, ascending input
// order).  Each thread then owns 16 bytes of every layer at its pixels (4
// RGBA8 pixels + their 4 depths, 1 RGBA32F pixel, 2 RGBA16F pixels), issues
// the loads of several inputs back to back (independent 16-byte loads in
// flight) and folds them in order in registers (composite_body.cuh).  The
// per-pixel order of operations is fixed by the input order alone, so results
// do not depend on the tile shape.
#include "composite_body.cuh"

namespace ec {
namespace {

constexpr int kThreads = 256;
constexpr int kRows = kThreads / 32;   // one warp per tile row

// The depth merge runs 128-thread CTAs (tiles of 128 x 4 pixels): small
// frames then split into enough CTAs that the last wave costs little.
constexpr int kDThreads = 128;
constexpr int kDRows = kDThreads / 32;

template <int N, int CB>
__global__ void __launch_bounds__(kDThreads)
k_depth(const __grid_constant__ SrcList<N> L, const __grid_constant__ DstDesc D)
{
    constexpr int kTW = 128;     // 32 lanes x 4 pixels
    __shared__ int16_t act[N > 0 ? N : 1];
    __shared__ int nact_s;
    auto at = [&](int, int i) -> const SrcDesc& { return L.s[i]; };

    const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
    const int tx0 = blockIdx.x * kTW, ty0 = blockIdx.y * kDRows;
    build_active(at, L.n, tx0, ty0, min(tx0 + kTW, D.W), min(ty0 + kDRows, D.H), act, &nact_s);
    __syncthreads();
    const int x = tx0 + lane * 4, y = ty0 + row;
    if (x >= D.W || y >= D.H) return;
    depth_px4<CB>(at, act, nact_s, x, y, D);
}

template <int N, bool F16>
__global__ void __launch_bounds__(kThreads)
k_alpha_fwd(const __grid_constant__ SrcList<N> L, const __grid_constant__ DstDesc D)
{
    constexpr int PX = F16 ? 2 : 1;      // pixels per 16 bytes
    constexpr int kTW = 32 * PX;
    __shared__ int16_t act[N > 0 ? N : 1];
    __shared__ int nact_s;
    auto at = [&](int, int i) -> const SrcDesc& { return L.s[i]; };

    const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
    const int tx0 = blockIdx.x * kTW, ty0 = blockIdx.y * kRows;
    const int tx1 = min(tx0 + kTW, D.W), ty1 = min(ty0 + kRows, D.H);
    build_active(at, L.n, tx0, ty0, tx1, ty1, act, &nact_s);
    __syncthreads();
    const int nact = nact_s;
    // FP16 tiles that every active layer covers skip the range tests (FP32
    // keeps one path: its second path would cost more registers than it saves)
    bool full = false;
    if constexpr (F16) {
        bool covers = true;
        for (int k = threadIdx.x; k < nact; k += kThreads) {
            const SrcDesc& s = L.s[act[k]];
            covers = covers && s.x0 <= tx0 && s.x1 >= tx1 && s.y0 <= ty0 && s.y1 >= ty1;
        }
        full = __syncthreads_and(covers);
    }
    const int x = tx0 + lane * PX, y = ty0 + row;
    if (x >= D.W || y >= D.H) return;
    alpha_px<F16>(at, act, nact, x, y, D, full);
}

template <int N>
SrcList<N> make_list(const SrcDesc* src, int n)
{
    SrcList<N> L;
    L.n = n;
    L.pad[0] = L.pad[1] = L.pad[2] = 0;
    for (int i = 0; i < n; ++i) L.s[i] = src[i];
    return L;
}

template <int N>
cudaError_t depth_n(const SrcDesc* src, int n, int cb, const DstDesc& D, cudaStream_t s)
{
    const dim3 grid(ceil_div(D.W, 128), ceil_div(D.H, kDRows));
    const SrcList<N> L = make_list<N>(src, n);
    if (cb == 4) k_depth<N, 4><<<grid, kDThreads, 0, s>>>(L, D);
    else k_depth<N, 16><<<grid, kDThreads, 0, s>>>(L, D);
    return cudaGetLastError();
}

template <int N>
cudaError_t alpha_n(const SrcDesc* src, int n, bool f16, const DstDesc& D, cudaStream_t s)
{
    const SrcList<N> L = make_list<N>(src, n);
    if (f16) {
        const dim3 grid(ceil_div(D.W, 64), ceil_div(D.H, kRows));
        k_alpha_fwd<N, true><<<grid, kThreads, 0, s>>>(L, D);
    } else {
        const dim3 grid(ceil_div(D.W, 32), ceil_div(D.H, kRows));
        k_alpha_fwd<N, false><<<grid, kThreads, 0, s>>>(L, D);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_depth(const SrcDesc* src, int n, int color_bytes, const DstDesc& D,
                         cudaStream_t s)
{
    if (D.W <= 0 || D.H <= 0) return cudaSuccess;
    if (n <= 16) return depth_n<16>(src, n, color_bytes, D, s);
    if (n <= 64) return depth_n<64>(src, n, color_bytes, D, s);
    return depth_n<EC_MAX_SOURCES>(src, n, color_bytes, D, s);
}

cudaError_t launch_alpha_fwd(const SrcDesc* src, int n, bool f16, const DstDesc& D,
                             cudaStream_t s)
{
    if (D.W <= 0 || D.H <= 0) return cudaSuccess;
    if (n <= 16) return alpha_n<16>(src, n, f16, D, s);
    if (n <= 64) return alpha_n<64>(src, n, f16, D, s);
    return alpha_n<EC_MAX_SOURCES>(src, n, f16, D, s);
}

}  // namespace ec
