// k_fused.cu -- fused decode-and-composite for the stages of multi-stage
// compositing schedules (thesis 5.2.2 binary swap, 5.2.3 streaming
// compositing): a resource receives RLE-coded pieces (thesis 5.5.1) of another
// resource's partial frame and depth-merges them with its own image
// (thesis 5.2.1) without writing the decoded pieces to memory first.
//
// One CTA of eight warps per work unit.  A decode unit is one 4096-element
// chunk of a received piece: warps 0-3 decode the colour stream's four byte
// planes and warps 4-7 the depth stream's into shared memory (the decoder of
// the RLE kernels, including its validation), then every thread transposes
// four elements of each back from planes, reads the local input at the same
// frame pixels and writes the merge.  A fill unit covers output pixels no
// piece reaches: the local input (or the background) is written there.
//
// The merge of a front and a back partial: the front is first merged with the
// cleared background (depth not below 1.0, or NaN, gives the background), then
// the back replaces it where its depth is strictly smaller.  A partial that is
// already a composite is unchanged by the first step, a raw source image is
// made one, and ties stay with the front, the lower source indices.
#include "ec_internal.cuh"
#include "rle_codec.cuh"

namespace ec {
namespace {

constexpr int kFT = 256;
constexpr int kChunk = rlec::kChunk;
constexpr uint32_t kBgDepth = 0x3F800000u;   // 1.0f

__device__ __forceinline__ bool below_one(uint32_t d) { return __uint_as_float(d) < 1.0f; }
__device__ __forceinline__ bool less(uint32_t a, uint32_t b) { return __uint_as_float(a) < __uint_as_float(b); }

// Merge one pixel: front (fc, fd) and back (bc, bd) as raw bits.
__device__ __forceinline__ void merge(uint32_t fc, uint32_t fd, uint32_t bc, uint32_t bd, uint32_t& oc, uint32_t& od)
{
    if (!below_one(fd)) { fc = 0u; fd = kBgDepth; }
    const bool b = less(bd, fd);
    oc = b ? bc : fc;
    od = b ? bd : fd;
}

// Four consecutive elements of a rectangle of width w starting at element q:
// frame pixels (x0 + x, y0 + y) with (x, y) stepping along the rows.
struct Run4 {
    int x, y;      // frame coordinates of the first element
    bool row;      // all four in one row
};

__device__ __forceinline__ void local4(const FusedStage& S, const Run4& r, int cnt, uint32_t* lc, uint32_t* ld,
                                       int w, int x0)
{
    const bool in_y = r.y >= S.r0y && r.y < S.r1y;
    if (r.row && cnt == 4 && in_y && r.x >= S.r0x && r.x + 3 < S.r1x) {
        const size_t e = (size_t)(r.y - S.ly) * S.lpitch + (r.x - S.lx);
        if (S.lvec && (e & 3) == 0) {
            const uint4 c = __ldcs(reinterpret_cast<const uint4*>(S.lc + e));
            const uint4 d = __ldcs(reinterpret_cast<const uint4*>(S.ld + e));
            lc[0] = c.x; lc[1] = c.y; lc[2] = c.z; lc[3] = c.w;
            ld[0] = d.x; ld[1] = d.y; ld[2] = d.z; ld[3] = d.w;
            return;
        }
    }
    int x = r.x, y = r.y;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        lc[k] = 0u;
        ld[k] = kBgDepth;
        if (k < cnt && y >= S.r0y && y < S.r1y && x >= S.r0x && x < S.r1x) {
            const size_t e = (size_t)(y - S.ly) * S.lpitch + (x - S.lx);
            lc[k] = __ldcs(S.lc + e);
            ld[k] = __ldcs(reinterpret_cast<const uint32_t*>(S.ld) + e);
        }
        if (++x == x0 + w) { x = x0; ++y; }
    }
}

__device__ __forceinline__ void store4(const FusedStage& S, const Run4& r, int cnt, const uint32_t* oc,
                                       const uint32_t* od, int w, int x0)
{
    if (r.row && cnt == 4) {
        const size_t e = (size_t)(r.y - S.oy) * S.opitch + (r.x - S.ox);
        if (S.ovec && (e & 3) == 0) {
            st_stream(reinterpret_cast<uint4*>(S.oc + e), make_uint4(oc[0], oc[1], oc[2], oc[3]));
            st_stream(reinterpret_cast<uint4*>(S.od) + e / 4, make_uint4(od[0], od[1], od[2], od[3]));
            return;
        }
    }
    int x = r.x, y = r.y;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (k < cnt) {
            const size_t e = (size_t)(y - S.oy) * S.opitch + (x - S.ox);
            S.oc[e] = oc[k];
            reinterpret_cast<uint32_t*>(S.od)[e] = od[k];
        }
        if (++x == x0 + w) { x = x0; ++y; }
    }
}

__global__ void __launch_bounds__(kFT)
k_fused_depth(const FusedStage* __restrict__ stages, const FusedUnit* __restrict__ units, uint32_t* status)
{
    __shared__ __align__(16) uint8_t planes[8][kChunk];
    __shared__ uint8_t s_hdr[2][rlec::kHdrBytes];
    __shared__ uint32_t s_beg[2][5];
    __shared__ int s_mode[2];
    __shared__ int s_fail;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const FusedUnit u = units[blockIdx.x];
    const FusedStage S = stages[u.stage];
    const uint32_t n = (uint32_t)u.w * (uint32_t)u.h;
    const uint32_t q0 = u.chunk * (uint32_t)kChunk;
    const int len = (int)min((uint32_t)kChunk, n - q0);
    const bool coded = u.cs != nullptr;

    if (coded) {
        const uint32_t nc = (n + kChunk - 1) / kChunk;
        const uint64_t csz = *u.csize, dsz = *u.dsize;
        if (tid < rlec::kHdrBytes) s_hdr[0][tid] = rlec::header_byte(u.cs, csz, nc, u.chunk, tid);
        else if (tid >= 64 && tid < 64 + rlec::kHdrBytes)
            s_hdr[1][tid - 64] = rlec::header_byte(u.ds, dsz, nc, u.chunk, tid - 64);
        if (tid == 0) s_fail = 0;
        __syncthreads();
        if (tid == 0 || tid == 32) {
            const int k = tid >> 5;
            if (rlec::check_header(s_hdr[k], k ? dsz : csz, (uint32_t)u.w, (uint32_t)u.h, nc, u.chunk,
                                   s_beg[k], &s_mode[k]))
                s_fail = 1;
        }
        __syncthreads();
        if (s_fail) {
            if (tid == 0) set_status(status, EC_ERR_CORRUPT);
            return;
        }
        const int k = warp >> 2, p = warp & 3;
        const uint8_t* payload = (k ? u.ds : u.cs) + 32 + 16ull * nc;
        if (rlec::decode_plane(payload, (int)s_beg[k][p], (int)s_beg[k][p + 1], len, planes[warp], lane) &&
            lane == 0)
            s_fail = 1;
        __syncthreads();
        if (s_fail) {
            if (tid == 0) set_status(status, EC_ERR_CORRUPT);
            return;
        }
    }

    const bool csw = coded && s_mode[0] == 2, dsw = coded && s_mode[1] == 2;
    const int w = u.w;
    for (int g = tid; 4 * g < len; g += kFT) {
        const uint32_t q = q0 + 4u * (uint32_t)g;
        Run4 r;
        const int yy = (int)(q / (uint32_t)w), xx = (int)(q - (uint32_t)yy * (uint32_t)w);
        r.x = u.x + xx;
        r.y = u.y + yy;
        r.row = xx + 3 < w;
        const int cnt = min(4, len - 4 * g);
        uint32_t lc[4], ld[4], oc[4], od[4];
        local4(S, r, cnt, lc, ld, w, u.x);
        if (coded) {
            const uint4 C = rlec::transpose4(reinterpret_cast<const uint32_t*>(planes[0])[g],
                                             reinterpret_cast<const uint32_t*>(planes[1])[g],
                                             reinterpret_cast<const uint32_t*>(planes[2])[g],
                                             reinterpret_cast<const uint32_t*>(planes[3])[g]);
            const uint4 D = rlec::transpose4(reinterpret_cast<const uint32_t*>(planes[4])[g],
                                             reinterpret_cast<const uint32_t*>(planes[5])[g],
                                             reinterpret_cast<const uint32_t*>(planes[6])[g],
                                             reinterpret_cast<const uint32_t*>(planes[7])[g]);
            uint32_t ic[4] = {C.x, C.y, C.z, C.w}, id[4] = {D.x, D.y, D.z, D.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (csw) ic[k] = rlec::swizzle(ic[k]);
                if (dsw) id[k] = rlec::swizzle(id[k]);
                if (S.front) merge(ic[k], id[k], lc[k], ld[k], oc[k], od[k]);
                else merge(lc[k], ld[k], ic[k], id[k], oc[k], od[k]);
            }
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const bool keep = below_one(ld[k]);
                oc[k] = keep ? lc[k] : 0u;
                od[k] = keep ? ld[k] : kBgDepth;
            }
        }
        store4(S, r, cnt, oc, od, w, u.x);
    }
}

}  // namespace

cudaError_t launch_fused_depth(const FusedStage* stages, const FusedUnit* units, int n_units,
                               uint32_t* status, cudaStream_t s)
{
    if (n_units <= 0) return cudaSuccess;
    k_fused_depth<<<n_units, kFT, 0, s>>>(stages, units, status);
    return cudaGetLastError();
}

}  // namespace ec
