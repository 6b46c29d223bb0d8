// k_rle.cu -- run-length pixel codec kernels for sm_103a (thesis 5.5.1:
// per-component RLE, bit-swizzle preconditioner, data decomposition).
//
// Compress: a pipeline of kernels with no waits between warps.
//   1. Coding (persistent warps, a chunk of 4096 elements at a time from an
//      atomic ticket): the chunk streams through shared memory and its change
//      points are listed; a chunk with few of them (sparse) is coded at once
//      from the list into a scratch pool, the others (dense) are listed.
//      Modes 1, 2: element change points, four byte planes (mode 2 swizzled;
//      the swizzle permutes bits, so it commutes with the comparison); runs of
//      three or more bytes become repeat tokens, maximal spans of shorter runs
//      literal tokens.  Mode 0 (basic RLE): change points of 8-byte units,
//      one stream; runs of two or more units repeat, single units literal.
//   2. Sizing of the dense chunks from the image: all four planes classified
//      at once with byte-SIMD masks (a byte is part of a repeat iff one of the
//      three windows of 3 around it is constant), warp max- and sum-scans over
//      8 steps of 512 positions; in mode 0 a CTA per chunk with block scans.
//   3. A scan of each job's chunk sizes: the chunks' offsets, the header and
//      the stream size.
//   4. Placing: the pooled chunks copied to their place with their end-table
//      entries; the dense chunks coded again, straight to their place.
// Every wait (the copies into shared memory) is bounded (EC_ERR_TIMEOUT).
//
// Decompress: one CTA of four warps per chunk.  The header and the chunk's
// end-table entries are fetched in one round trip and validated.  Warp p
// decodes plane p in windows of 32 stream bytes: the jump from each byte to
// the token after one starting there is composed by doubling, so lane t holds
// the window's t-th token; a warp scan places the tokens, each is checked
// against its stream and chunk bounds, lanes write the unaligned ends of their
// repeat tokens and short aligned bodies, the warp a long body per store.  The four
// planes are then transposed back into elements with byte permutes.
#include "ec_internal.cuh"
#include "rle_codec.cuh"

#include <algorithm>
#include <atomic>

namespace ec {
namespace {

constexpr int kChunk = EC_RLE_CHUNK;                 // 4096 elements
constexpr int kT = 256;                              // threads per mode-0 CTA
constexpr uint32_t kMagic = 0x31524345u;             // "ECR1"
constexpr int kSpinLimit = 1 << 20;            // tries of a bounded mbarrier wait

using rlec::swizzle;
using rlec::transpose4;
using rlec::bcast8;

template <int N>
__device__ __forceinline__ int find_job(const RleJobList<N>& J, uint32_t unit)
{
    int lo = 0, hi = J.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (J.j[mid].first_unit <= unit) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void put_u32(uint8_t* p, uint32_t v)
{
    p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); p[2] = (uint8_t)(v >> 16); p[3] = (uint8_t)(v >> 24);
}


// Element q of a job's image.
__device__ __forceinline__ size_t elem_off(const RleJobDesc& jb, uint32_t q)
{
    const uint32_t y = q / (uint32_t)jb.w;
    return (size_t)y * jb.pitch + (q - y * (uint32_t)jb.w);
}

__device__ void write_header(uint8_t* d, const RleJobDesc& jb)
{
    put_u32(d + 0, kMagic);
    d[4] = 1; d[5] = 0;                               // version
    d[6] = (uint8_t)jb.mode; d[7] = 0;
    put_u32(d + 8, (uint32_t)jb.w);
    put_u32(d + 12, (uint32_t)jb.h);
    put_u32(d + 16, 4u);
    put_u32(d + 20, (uint32_t)kChunk);
    put_u32(d + 24, jb.n_chunks);
    put_u32(d + 28, jb.mode == 0 ? 1u : 4u);       // streams per chunk
}

// ------------------------------------------------------------- compress ----

// Copy n stage bytes (src 4-byte aligned) to o, threads t, t+nt, ...: byte
// stores up to o's first word boundary and after its last, word stores of
// funnel-shifted stage words between.  The two buffers never overlap, and a
// thread's loads (eight words at a time, and its head and tail bytes) are all
// issued before its stores.  Reads up to one word past src + n.
__device__ __forceinline__ void copy_out(uint8_t* __restrict__ o, const uint8_t* __restrict__ src, uint32_t n,
                                         uint32_t t, uint32_t nt)
{
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(o), a1 = a0 + n;
    const uintptr_t w0 = (a0 + 3) & ~(uintptr_t)3, w1 = a1 & ~(uintptr_t)3;
    if (w0 >= w1) {
        for (uint32_t i = t; i < n; i += nt) o[i] = src[i];
        return;
    }
    const uint32_t head = (uint32_t)(w0 - a0), tail0 = (uint32_t)(w1 - a0);   // head, n - tail0 < 4 <= nt
    const bool hh = t < head, th = tail0 + t < n;
    const uint8_t hb = hh ? src[t] : 0, tb = th ? src[tail0 + t] : 0;
    const uint32_t nw = (uint32_t)((w1 - w0) >> 2);
    const uint32_t* __restrict__ s32 = reinterpret_cast<const uint32_t*>(src);
    const uint32_t sh = 8u * head;
    uint32_t* __restrict__ o32 = reinterpret_cast<uint32_t*>(w0);
    for (uint32_t k0 = t; k0 < nw; k0 += 8u * nt) {
        uint32_t v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            // bytes [head + 4k, head + 4k + 4), head < 4
            const uint32_t k = k0 + (uint32_t)j * nt;
            v[j] = k < nw ? __funnelshift_r(s32[k], s32[k + 1], sh) : 0u;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t k = k0 + (uint32_t)j * nt;
            if (k < nw) o32[k] = v[j];
        }
    }
    if (hh) o[t] = hb;
    if (th) o[tail0 + t] = tb;
}

// ---- compressor: one warp per chunk ---------------------------------------
// Every warp of the coding kernel works alone, chunk after chunk.  It streams
// each chunk through a ring of two 2 KB quarter buffers in shared memory,
// filled by asynchronous copies (bulk copies of row segments, or 4-byte copies
// where rows are not 16-byte aligned) that complete on the buffer's mbarrier;
// a buffer is refilled with the next quarter (of this chunk or the next) as
// soon as it has been read.  Reading a chunk, the warp lists its change
// points: the positions where the element differs from its predecessor, with
// the element there.  A byte plane can change only where the element does, so
// each plane's runs are the change points where that plane's byte differs
// from the previous change point's, and every run's value is the byte at its
// start: the sparse path codes the chunk's streams from the change list alone,
// into the warp's stage, and leaves them in a scratch pool.  Chunks with more
// change points than the list holds are dense: a recoding kernel sizes them
// from the image.  A scan over each job's chunk sizes gives every chunk its
// offset; a placing kernel copies the pooled chunks to their place and the
// recoding kernel writes the dense ones there (coded again from the image,
// partly from L2).  No kernel waits for another's warps.
constexpr int kWPB = 2;                       // warps per CTA
constexpr int kCap = 128;                     // change points the sparse path takes
constexpr int kQ = 512;                       // elements per quarter buffer
constexpr int kQPC = kChunk / kQ;             // quarters per chunk
constexpr int kSlots = 2;                     // quarter buffers per warp

// Each plane of a sparse chunk has at most kCap runs and codes to at most
// 3 kCap + kChunk / 64 bytes (a repeat run of length L to 2 ceil(L / 128) <=
// 2 + L / 64 bytes, a literal span of k short runs to at most 3k bytes).
constexpr int kStagePlane = 3 * kCap + kChunk / 64;
constexpr uint32_t kRecode = 0xFFFFFFFFu;      // record: coded again when placed

// One warp's shared memory.  Quarter s of the warp's sequence of quarters
// (4 per chunk) goes to buf[s % kSlots].
struct WarpRing {
    uint32_t buf[kSlots][kQ + 4];   // + 16 guard bytes before each quarter
    uint64_t full[kSlots];
    uint64_t pad[4 - kSlots];       // (keeps what follows 16-byte aligned)
    uint8_t stage[4 * kStagePlane]; // the chunk's plane streams (plane p at p * kStagePlane)
    uint32_t ce[kCap];              // the chunk being read: element at each change point
    uint16_t cq[kCap];              // (swizzled in mode 2) and its position
    uint8_t rl[4][kCap];            // the planes' runs: index of the change point starting each
};
static_assert((kQ + 4) * 4 % 16 == 0 && sizeof(WarpRing) % 16 == 0, "16-byte aligned buffers");

// A coded chunk, as the coding kernel leaves it for the placing kernels: its
// four plane stream sizes, where its streams wait in the pool (kRecode: not
// kept, coded again from the image when placed), and its offset inside the
// stream's payload (written by the scan).
struct ChunkRec {
    uint16_t T[4];
    uint32_t pool;
    uint32_t off;
};
static_assert(sizeof(ChunkRec) == 16, "chunk record");
constexpr size_t kCompressSmem = kWPB * sizeof(WarpRing);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t* b, uint32_t bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
                 ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

// One try of a wait for the phase of the given parity; the thread may sleep
// in it (up to about a microsecond) until the phase completes.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_u32(b)), "r"(parity), "r"(1000u) : "memory");
    return ok != 0u;
}

// Wait for the phase of the given parity to complete; gives up after
// kSpinLimit tries (recording EC_ERR_TIMEOUT) instead of spinning forever.
__device__ __forceinline__ void mbar_wait(uint64_t* b, uint32_t parity, uint32_t* status)
{
    for (int i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(b, parity)) return;
    set_status(status, EC_ERR_TIMEOUT);
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from
// global to shared memory, completing on mbarrier b.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* b)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(b)) : "memory");
}

// Elements [q, q + 4) of a chunk that starts at element q0 (q a multiple of
// 4; zeros past len).  16-byte loads where the image allows them (the four
// elements then lie in one row), else one load per element.
__device__ __forceinline__ uint4 load_elems(const RleJobDesc& jb, uint32_t q0, int len, int q)
{
    if (q >= len) return make_uint4(0u, 0u, 0u, 0u);
    const uint32_t w = (uint32_t)jb.w;
    if (jb.vec) {
        size_t e = q0 + (uint32_t)q;
        if (jb.pitch != jb.w) {
            const uint32_t y = (q0 + (uint32_t)q) / w;
            e = (size_t)y * jb.pitch + (q0 + (uint32_t)q - y * w);
        }
        return __ldg(reinterpret_cast<const uint4*>(jb.src + e));
    }
    uint32_t v[4];
    uint32_t y = (q0 + (uint32_t)q) / w, x = q0 + (uint32_t)q - y * w;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = q + k < len ? __ldg(jb.src + (size_t)y * jb.pitch + x) : 0u;
        if (++x == w) { x = 0u; ++y; }
    }
    return make_uint4(v[0], v[1], v[2], v[3]);
}

// Asynchronous 4-byte copy from global to shared memory, and the arrival on
// mbarrier b once all of this thread's earlier such copies have landed (the
// barrier's pending count is raised by one now and lowered by the arrival).
__device__ __forceinline__ void cp_async4(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_arrive(uint64_t* b)
{
    asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(smem_u32(b)) : "memory");
}

// Start the copy of quarter qi of chunk `unit` into W.buf[slot].  Images whose
// rows are 16-byte aligned: lane 0 sets the expected bytes, every lane copies
// row segments with bulk copies.  Other images: every lane copies elements
// lane, lane + 32, ... with 4-byte asynchronous copies, and the barrier
// completes once all of them have landed.  Quarters with nothing to copy (past
// the image's end, an empty image) just arrive.
__device__ void issue_quarter(const RleJobDesc& jb, uint32_t unit, int qi, int slot, WarpRing& W)
{
    const int lane = threadIdx.x & 31;
    int qlen = 0;
    uint32_t qs = 0u;
    if (jb.n_chunks > 0) {
        const uint32_t q0 = (unit - jb.first_unit) * (uint32_t)kChunk;
        const int len = (int)min((uint32_t)kChunk, (uint32_t)jb.w * (uint32_t)jb.h - q0);
        qlen = min(max(len - kQ * qi, 0), kQ);
        qs = q0 + (uint32_t)(kQ * qi);
    }
    if (qlen == 0) {
        if (lane == 0) mbar_arrive(&W.full[slot]);
        return;
    }
    uint32_t* dst = W.buf[slot] + 4;
    const uint32_t w = (uint32_t)jb.w;
    if (!jb.vec) {
        uint32_t y = (qs + (uint32_t)lane) / w, x = qs + (uint32_t)lane - y * w;
        for (int i = lane; i < qlen; i += 32) {
            cp_async4(dst + i, jb.src + (size_t)y * jb.pitch + x);
            x += 32u;
            while (x >= w) { x -= w; ++y; }
        }
        cp_async_arrive(&W.full[slot]);
        __syncwarp();                                  // every lane's pending count is in
        if (lane == 0) mbar_arrive(&W.full[slot]);
        return;
    }
    if (lane == 0) mbar_arrive_tx(&W.full[slot], 4u * (uint32_t)qlen);
    __syncwarp();
    if (jb.pitch == jb.w) {
        if (lane == 0) bulk_load(dst, jb.src + qs, 4u * (uint32_t)qlen, &W.full[slot]);
        return;
    }
    const uint32_t y0 = qs / w, y1 = (qs + (uint32_t)qlen - 1u) / w;
    for (uint32_t y = y0 + (uint32_t)lane; y <= y1; y += 32) {
        const uint32_t a = y == y0 ? qs - y0 * w : 0u;                   // first column of the segment
        const uint32_t b = min(w, qs + (uint32_t)qlen - y * w);          // its end column
        bulk_load(dst + (y * w + a - qs), jb.src + (size_t)y * jb.pitch + a, 4u * (b - a), &W.full[slot]);
    }
}

// Append the change points among positions [kQ qi, kQ qi + kQ) of the chunk
// to W.ce / W.cq (the quarter's elements in shared memory at `data`).  carry:
// the element before the quarter (updated to the quarter's last).  Every lane
// flags the changes among its four elements of each of the G groups of 128
// positions; one warp scan of the four groups' per-lane counts, packed in the
// bytes of a word (a group has at most 128 changes, so no byte carries into
// the next), places every change point in position order at once.  Returns
// false once the chunk has more than kCap change points.
__device__ bool detect_quarter(const uint32_t* data, int len, int qi, WarpRing& W, int& m, uint32_t& carry)
{
    const int lane = threadIdx.x & 31;
    constexpr int G = kQ / 128;
    static_assert(G == 4, "four groups' counts in the bytes of one word");
    uint4 vv[G];
    uint32_t pv[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        vv[g] = *reinterpret_cast<const uint4*>(data + 128 * g + 4 * lane);
        pv[g] = data[128 * g + 4 * lane - 1];             // g = lane = 0 reads the guard word
    }
    if (lane == 0) pv[0] = qi == 0 ? ~vv[0].x : carry;    // position 0 is always listed
    carry = __shfl_sync(0xffffffffu, vv[G - 1].w, 31);   // (used only when the quarter is full)
    const int qend = min(len - kQ * qi, kQ);              // positions of this quarter
    uint32_t f[G], packed = 0u;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const uint4 v = vv[g];
        f[g] = (uint32_t)(v.x != pv[g]) | ((uint32_t)(v.y != v.x) << 1) | ((uint32_t)(v.z != v.y) << 2) |
               ((uint32_t)(v.w != v.z) << 3);
    }
    if (qend < kQ) {                                      // the chunk's last quarter: positions past len
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int q = 128 * g + 4 * lane;
            if (q + 4 > qend) f[g] &= q >= qend ? 0u : (1u << (qend - q)) - 1u;
        }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) packed |= (uint32_t)__popc(f[g]) << (8 * g);
    uint32_t inc = packed;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    const uint32_t tot = __shfl_sync(0xffffffffu, inc, 31), exc = inc - packed;
    const int cnt = (int)((tot & 0xFFu) + ((tot >> 8) & 0xFFu) + ((tot >> 16) & 0xFFu) + (tot >> 24));
    if (m + cnt > kCap) return false;
    int base = m;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        if (f[g]) {
            const uint4 v = vv[g];
            const int qq = kQ * qi + 128 * g + 4 * lane;
            int o = base + (int)((exc >> (8 * g)) & 0xFFu);
            if (f[g] & 1u) { W.cq[o] = (uint16_t)qq; W.ce[o] = v.x; ++o; }
            if (f[g] & 2u) { W.cq[o] = (uint16_t)(qq + 1); W.ce[o] = v.y; ++o; }
            if (f[g] & 4u) { W.cq[o] = (uint16_t)(qq + 2); W.ce[o] = v.z; ++o; }
            if (f[g] & 8u) { W.cq[o] = (uint16_t)(qq + 3); W.ce[o] = v.w; }
        }
        base += (int)((tot >> (8 * g)) & 0xFFu);
    }
    m += cnt;
    return true;
}

// The change lists a sparse coder reads: element (swizzled in mode 2) and
// position of each change point, in order; rl is its scratch.
struct Lists {
    uint32_t* ce;
    uint16_t* cq;
    uint8_t (*rl)[kCap];
};

// Sparse path, fast case: at most 32 change points and every run of every
// plane at least 3 bytes long (so every run is repeat tokens).  Lane i holds
// change point i; for each plane the lanes that start a run are found with
// one ballot, each run's end is the next such lane's position (a shuffle) or
// the chunk's end, and one scan over the four planes (16-bit halves) places
// the tokens.  Returns false, writing nothing, when the case does not apply.
__device__ bool code_sparse_fast(const Lists& W, int m, int len, uint32_t* T, uint8_t* stage)
{
    const int lane = threadIdx.x & 31;
    if (m > 32) return false;
    __syncwarp();                                     // the change list is complete
    const bool valid = lane < m;
    const uint32_t e = valid ? W.ce[lane] : 0u;
    const int q = valid ? (int)W.cq[lane] : 0;
    uint32_t diff = e ^ __shfl_up_sync(0xffffffffu, e, 1);
    if (lane == 0) diff = 0xFFFFFFFFu;                // change point 0 starts a run in every plane
    const uint32_t above = lane == 31 ? 0u : ~((2u << lane) - 1u);
    uint32_t cost[4], K[4];
    int L[4];
    bool bad = false;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const bool keep = valid && ((diff >> (8 * p)) & 0xFFu) != 0u;
        K[p] = __ballot_sync(0xffffffffu, keep);
        const uint32_t nm = K[p] & above;
        const int qn = __shfl_sync(0xffffffffu, q, nm ? __ffs(nm) - 1 : 0);
        L[p] = keep ? (nm ? qn : len) - q : 0;
        bad |= keep && L[p] < 3;
        cost[p] = keep ? 2u * (uint32_t)((L[p] + 127) >> 7) : 0u;
    }
    if (__any_sync(0xffffffffu, bad)) return false;
    const uint32_t a = cost[0] | (cost[1] << 16), b = cost[2] | (cost[3] << 16);
    uint32_t ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t ya = __shfl_up_sync(0xffffffffu, ia, o), yb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) { ia += ya; ib += yb; }
    }
    const uint32_t ta = __shfl_sync(0xffffffffu, ia, 31), tb = __shfl_sync(0xffffffffu, ib, 31);
    const uint32_t ea = ia - a, eb = ib - b;
    const uint32_t ex[4] = {ea & 0xFFFFu, ea >> 16, eb & 0xFFFFu, eb >> 16};
    T[0] = ta & 0xFFFFu; T[1] = ta >> 16; T[2] = tb & 0xFFFFu; T[3] = tb >> 16;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        if (!((K[p] >> lane) & 1u) || ex[p] + cost[p] > (uint32_t)kStagePlane) continue;
        uint8_t* ob = stage + p * kStagePlane + ex[p];
        const uint8_t v = (uint8_t)(e >> (8 * p));
        for (int rr = L[p]; rr > 0; rr -= 128) {
            ob[0] = (uint8_t)(127 + min(rr, 128));
            ob[1] = v;
            ob += 2;
        }
    }
    return true;
}

// Sparse path, the four planes together (their chains of shuffles and shared
// memory accesses overlap).  Runs of plane p: change point i starts one iff
// its plane-p byte differs from change point i-1's (point 0 always does);
// rl[p][0, n_p) lists those change points.  Then the runs are coded 32 at a
// time, a run per lane: a run of three or more bytes becomes repeat tokens; a
// shorter one belongs to a literal span (a maximal sequence of short runs),
// whose start a warp max-scan finds (four planes in the bytes of one word).
// A short run at byte offset b of its span writes its bytes, the control
// byte of a token that starts among them, and, if it holds a token's last
// byte, that token's control byte (127 for a full token; the span's last run
// knows the span's length).  Plane p's stream goes to stage + p * kStagePlane
// (as far as it fits); its size to T[p].
__device__ void code_sparse(const Lists& W, int m, int len, uint32_t* T, uint8_t* stage)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    __syncwarp();                                     // the change list is complete
    int n[4] = {0, 0, 0, 0};
    uint32_t preve = 0u;
    for (int r = 0; r < m; r += 32) {
        const int i = r + lane;
        const bool valid = i < m;
        const uint32_t e = valid ? W.ce[i] : 0u;
        uint32_t ep = __shfl_up_sync(0xffffffffu, e, 1);
        if (lane == 0) ep = preve;
        const uint32_t diff = e ^ ep;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const bool keep = valid && (i == 0 || ((diff >> (8 * p)) & 0xFFu) != 0u);
            const uint32_t K = __ballot_sync(0xffffffffu, keep);
            if (keep) W.rl[p][n[p] + __popc(K & lt)] = (uint8_t)i;
            n[p] += __popc(K);
        }
        preve = __shfl_sync(0xffffffffu, e, 31);
    }
    __syncwarp();
    uint32_t carry[4] = {0u, 0u, 0u, 0u};
    uint32_t sscarry = 0u;                            // byte p: 1 + the last span start of plane p so far
    uint32_t prevshort = 0u;                          // bit p: the previous block's last run was short
    const int nmax = max(max(n[0], n[1]), max(n[2], n[3]));
    for (int r = 0; r < nmax; r += 32) {
        const int i = r + lane;
        int s[4], L[4];
        uint32_t shm = 0u, nshm = 0u, stv = 0u;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const uint8_t* R = W.rl[p];
            const int np = n[p];
            s[p] = 0;
            L[p] = 0;
            if (i < np) {
                s[p] = (int)W.cq[R[i]];
                L[p] = (i + 1 < np ? (int)W.cq[R[i + 1]] : len) - s[p];
                if (L[p] < 3) shm |= 1u << p;
            }
        }
        uint32_t prevm = __shfl_up_sync(0xffffffffu, shm, 1);
        if (lane == 0) prevm = prevshort;
        nshm = __shfl_down_sync(0xffffffffu, shm, 1);
        if (lane == 31) {                             // the next block's first runs
            nshm = 0u;
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const uint8_t* R = W.rl[p];
                const int np = n[p];
                if (i + 1 < np) {
                    const int ln = (i + 2 < np ? (int)W.cq[R[i + 2]] : len) - (int)W.cq[R[i + 1]];
                    if (ln < 3) nshm |= 1u << p;
                }
            }
        }
#pragma unroll
        for (int p = 0; p < 4; ++p)
            if (((shm & ~prevm) >> p) & 1u) stv |= (uint32_t)(i + 1) << (8 * p);
        uint32_t ss = stv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, ss, o);
            if (lane >= o) ss = __vmaxu4(ss, y);
        }
        ss = __vmaxu4(ss, sscarry);
        sscarry = __shfl_sync(0xffffffffu, ss, 31);
        prevshort = __shfl_sync(0xffffffffu, shm, 31);
        uint32_t cost[4], B[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            cost[p] = 0u;
            B[p] = 0u;
            if (i >= n[p]) continue;
            if (!((shm >> p) & 1u)) {
                cost[p] = 2u * (uint32_t)((L[p] + 127) >> 7);
            } else {
                const int ssi = (int)((ss >> (8 * p)) & 0xFFu) - 1;
                const uint32_t b = (uint32_t)(s[p] - (int)W.cq[W.rl[p][ssi]]);   // offset in the span
                B[p] = b;
                cost[p] = (uint32_t)L[p] + (((b + (uint32_t)L[p] + 127u) >> 7) - ((b + 127u) >> 7));
            }
        }
        // four scans at once: planes 0,1 and 2,3 in 16-bit halves
        const uint32_t a = cost[0] | (cost[1] << 16), bb = cost[2] | (cost[3] << 16);
        uint32_t ia = a, ib = bb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t ya = __shfl_up_sync(0xffffffffu, ia, o), yb = __shfl_up_sync(0xffffffffu, ib, o);
            if (lane >= o) { ia += ya; ib += yb; }
        }
        const uint32_t ta = __shfl_sync(0xffffffffu, ia, 31), tb = __shfl_sync(0xffffffffu, ib, 31);
        const uint32_t ea = ia - a, eb = ib - bb;
        const uint32_t ex[4] = {ea & 0xFFFFu, ea >> 16, eb & 0xFFFFu, eb >> 16};
        const uint32_t tot[4] = {ta & 0xFFFFu, ta >> 16, tb & 0xFFFFu, tb >> 16};
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const uint32_t o = carry[p] + ex[p];
            carry[p] += tot[p];
            if (i >= n[p] || o + cost[p] > (uint32_t)kStagePlane) continue;   // (never exceeds: kStagePlane)
            uint8_t* ob = stage + p * kStagePlane;
            const uint8_t v = (uint8_t)(W.ce[W.rl[p][i]] >> (8 * p));
            if (!((shm >> p) & 1u)) {
                uint32_t q = o;
                for (int rr = L[p]; rr > 0; rr -= 128) {
                    ob[q] = (uint8_t)(127 + min(rr, 128));
                    ob[q + 1] = v;
                    q += 2;
                }
            } else {
                const uint32_t b = B[p];
                const uint32_t so = o - b - ((b + 127u) >> 7);   // the span's first control byte
                for (uint32_t x = b; x < b + (uint32_t)L[p]; ++x) {
                    ob[so + x + (x >> 7) + 1u] = v;
                    if ((x & 127u) == 127u) ob[so + 129u * (x >> 7)] = 127u;
                }
                if (!((nshm >> p) & 1u)) {            // the span's last run: its last token
                    const uint32_t last = b + (uint32_t)L[p] - 1u;
                    ob[so + 129u * (last >> 7)] = (uint8_t)(last & 127u);
                }
            }
        }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) T[p] = carry[p];
}

// Four 16-bit lanes in two words (planes 0,1 | planes 2,3).
struct P4 { uint32_t a, b; };

template <bool MAX>
__device__ __forceinline__ P4 combine(P4 x, P4 y)
{
    if (MAX) return {__vmaxu2(x.a, y.a), __vmaxu2(x.b, y.b)};
    return {x.a + y.a, x.b + y.b};   // lanes never carry: every sum < 65536
}

__device__ __forceinline__ uint32_t lane16(P4 v, int p)
{
    const uint32_t w = p < 2 ? v.a : v.b;
    return (p & 1) ? (w >> 16) : (w & 0xFFFFu);
}

// Warp-wide exclusive scan of P4 values; *total receives the warp's total.
template <bool MAX>
__device__ __forceinline__ P4 warp_scan4(P4 v, int lane, P4* total)
{
    P4 inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        P4 y;
        y.a = __shfl_up_sync(0xffffffffu, inc.a, o);
        y.b = __shfl_up_sync(0xffffffffu, inc.b, o);
        if (lane >= o) inc = combine<MAX>(inc, y);
    }
    total->a = __shfl_sync(0xffffffffu, inc.a, 31);
    total->b = __shfl_sync(0xffffffffu, inc.b, 31);
    P4 ex;
    ex.a = __shfl_up_sync(0xffffffffu, inc.a, 1);
    ex.b = __shfl_up_sync(0xffffffffu, inc.b, 1);
    if (lane == 0) ex = {0u, 0u};
    return ex;
}

// The most significant bit of each byte of w, gathered into bits 0..3.
__device__ __forceinline__ uint32_t byte_msbs(uint32_t w)
{
    return ((w & 0x80808080u) * 0x00204081u) >> 28;
}

// 4-bit mask of the bytes of a and b that are equal (bit i = byte i).
__device__ __forceinline__ uint32_t eq_bytes(uint32_t a, uint32_t b)
{
    const uint32_t x = a ^ b;                                   // zero byte <=> equal
    const uint32_t t = ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x | 0x7F7F7F7Fu);
    return byte_msbs(t);
}

// Bits [lo, hi) set (0 <= lo, hi <= 31).
__device__ __forceinline__ uint32_t bit_range(int lo, int hi)
{
    lo = max(lo, 0);
    hi = min(hi, 31);
    return hi > lo ? ((1u << hi) - 1u) & ~((1u << lo) - 1u) : 0u;
}

// Elements [q, q + 4) of the chunk (q a multiple of 4), swizzled in mode 2.
__device__ __forceinline__ uint4 load4(const RleJobDesc& jb, uint32_t q0, int len, int q, bool sw)
{
    uint4 v = load_elems(jb, q0, len, q);
    if (sw) { v.x = swizzle(v.x); v.y = swizzle(v.y); v.z = swizzle(v.z); v.w = swizzle(v.w); }
    return v;
}

// Dense path, a CTA of 8 warps per chunk: every position is classified with
// byte-SIMD bit masks, all four planes at once.  Warp k takes positions
// [512 k, 512 k + 512): lane l holds positions [P0, P0 + 16), P0 = 16 (32 k +
// l), in registers, and the bytes just before and after them come from its
// neighbours (shuffles; lane 0 and lane 31 load the neighbouring words).  A
// byte lies in a repeat iff one of the three windows of 3 around it is
// constant.  A max-scan of segment starts (warp scans, then the warps' totals
// through shared memory) cuts tokens every 128 bytes of a segment, and a
// sum-scan of output bytes (likewise) places them.  Without EMIT the plane
// stream sizes are returned in T; with EMIT (T holding them) the streams are
// written to out.  xw: 16 P4 of shared memory.
template <bool EMIT>
__device__ void dense_chunk(const RleJobDesc& jb, uint32_t q0, int len, bool sw, uint32_t* T, uint8_t* out, P4* xw)
{
    const int lane = threadIdx.x & 31, k = threadIdx.x >> 5;
    const bool act = 512 * k < len;                          // (uniform in the warp)
    uint32_t pbase[4] = {0u, 0u, 0u, 0u};
    if (EMIT) {
        pbase[1] = T[0];
        pbase[2] = T[0] + T[1];
        pbase[3] = T[0] + T[1] + T[2];
    }
    const int P0 = 16 * (32 * k + lane);
    uint32_t REP[4] = {0u, 0u, 0u, 0u}, SEG[4] = {0u, 0u, 0u, 0u};
    uint4 bytes[4];
    uint32_t VALID = 0u;
    P4 mine = {0u, 0u};
    if (act) {
        uint4 t[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint4 g = load4(jb, q0, len, P0 + 4 * i, sw);
            t[i] = transpose4(g.x, g.y, g.z, g.w);              // t[i] word b = plane b of 4 positions
        }
        uint4 tn = make_uint4(0u, 0u, 0u, 0u), tp = make_uint4(0u, 0u, 0u, 0u);
        if (lane == 31) {
            const uint4 g = load4(jb, q0, len, P0 + 16, sw);
            tn = transpose4(g.x, g.y, g.z, g.w);
        }
        if (lane == 0 && P0 > 0) {
            const uint4 g = load4(jb, q0, len, P0 - 4, sw);
            tp = transpose4(g.x, g.y, g.z, g.w);
        }
        const uint32_t VQ = bit_range(4 - P0, len - P0 + 4);          // 0 <= q < len
        const uint32_t VEQ = bit_range(5 - P0, len - P0 + 4);         // 1 <= q < len
        const uint32_t HIGH = bit_range(len - P0 + 4, 24);            // q >= len
        const uint32_t Q0 = P0 == 0 ? (1u << 4) : 0u;                 // q == 0
        VALID = (VQ >> 4) & 0xFFFFu;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            auto pw = [&](const uint4& x) { return b == 0 ? x.x : b == 1 ? x.y : b == 2 ? x.z : x.w; };
            const uint4 v = make_uint4(pw(t[0]), pw(t[1]), pw(t[2]), pw(t[3]));
            uint32_t wm = __shfl_up_sync(0xffffffffu, v.w, 1);
            if (lane == 0) wm = pw(tp);
            uint32_t wp = __shfl_down_sync(0xffffffffu, v.x, 1);
            if (lane == 31) wp = pw(tn);
            bytes[b] = v;
            // eq bit i: byte at position P0-4+i equals its predecessor
            uint32_t EQ = eq_bytes(wm, wm << 8);
            EQ |= eq_bytes(v.x, __funnelshift_l(wm, v.x, 8)) << 4;
            EQ |= eq_bytes(v.y, __funnelshift_l(v.x, v.y, 8)) << 8;
            EQ |= eq_bytes(v.z, __funnelshift_l(v.y, v.z, 8)) << 12;
            EQ |= eq_bytes(v.w, __funnelshift_l(v.z, v.w, 8)) << 16;
            EQ |= eq_bytes(wp, __funnelshift_l(v.w, wp, 8)) << 20;
            EQ &= VEQ & ~1u;                                          // bit 0 has no predecessor here
            const uint32_t T3 = EQ & (EQ << 1);                       // positions i-2, i-1, i equal
            const uint32_t R = (T3 | (T3 >> 1) | (T3 >> 2)) & VQ;     // byte lies in a run >= 3
            const uint32_t Sg = (((R & ~EQ) | (~R & (R << 1))) & VQ) | HIGH | Q0;
            REP[b] = (R >> 4) & 0xFFFFu;
            SEG[b] = (Sg >> 4) & 0x1FFFFu;                            // bit 16: position P0+16
        }
        // last segment start in each lane's range (position + 1)
        uint32_t l[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const uint32_t m = SEG[b] & 0xFFFFu;
            l[b] = m ? (uint32_t)(P0 + 31 - __clz(m) + 1) : 0u;
        }
        mine.a = l[0] | (l[1] << 16);
        mine.b = l[2] | (l[3] << 16);
    }
    // max-scan over the chunk: in the warp, then over the warps before
    P4 tmax = {0u, 0u}, smax = {0u, 0u};
    if (act) smax = warp_scan4<true>(mine, lane, &tmax);
    if (lane == 0) xw[k] = tmax;
    __syncthreads();
    P4 before = smax;
    for (int j = 0; j < k; ++j) before = combine<true>(before, xw[j]);
    // piece starts (tokens hold <= 128 bytes) and output sizes
    uint32_t PSV[4], PE[4], LIT[4], cost[4];
    int sbin[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const uint32_t seg16 = SEG[b] & 0xFFFFu;
        const int sb_in = (int)lane16(before, b) - 1;            // -1 only for position 0
        sbin[b] = sb_in;
        uint32_t PS = seg16;
        const int first = seg16 ? __ffs(seg16) - 1 : 16;
        if (sb_in >= 0) {                                        // continuing segment
            const int r = (P0 - sb_in) & 127;
            const int d = r ? 128 - r : 0;
            if (d < first) PS |= 1u << d;
        }
        const int sb15 = seg16 ? P0 + 31 - __clz(seg16) : sb_in;
        const uint32_t next = ((SEG[b] >> 16) & 1u) | (((P0 + 16 - sb15) & 127) == 0 ? 1u : 0u);
        PSV[b] = PS & VALID;
        PE[b] = ((PS | (next << 16)) >> 1) & VALID;
        LIT[b] = ~REP[b] & VALID;
        cost[b] = __popc(LIT[b]) + __popc(PSV[b]) + __popc(PSV[b] & REP[b]);
    }
    P4 tsum = {0u, 0u}, ssum = {0u, 0u};
    if (act) ssum = warp_scan4<false>(P4{cost[0] | (cost[1] << 16), cost[2] | (cost[3] << 16)}, lane, &tsum);
    if (lane == 0) xw[8 + k] = tsum;
    __syncthreads();
    P4 off0 = ssum, total = {0u, 0u};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const P4 x = xw[8 + j];
        if (j < k) off0 = combine<false>(off0, x);
        total = combine<false>(total, x);
    }
    __syncthreads();                                         // xw is reused by the next chunk
#pragma unroll
    for (int b = 0; b < ((EMIT && act) ? 4 : 0); ++b) {
        uint8_t* o = out + pbase[b];
        const uint32_t off = lane16(off0, b);
        const uint32_t lit = LIT[b], psv = PSV[b], psr = PSV[b] & REP[b], seg16 = SEG[b] & 0xFFFFu;
        const uint4 v = bytes[b];
        auto byte_at = [&](int i) -> uint8_t {
            const uint32_t wd = i < 8 ? (i < 4 ? v.x : v.y) : (i < 12 ? v.z : v.w);
            return (uint8_t)(wd >> (8 * (i & 3)));
        };
        auto inc_at = [&](int i) -> uint32_t {
            const uint32_t le = (2u << i) - 1u;
            return off + __popc(lit & le) + __popc(psv & le) + __popc(psr & le);
        };
        for (uint32_t m = lit; m; m &= m - 1u) {
            const int i = __ffs(m) - 1;
            o[inc_at(i) - 1] = byte_at(i);
        }
        for (uint32_t m = PE[b]; m; m &= m - 1u) {
            const int i = __ffs(m) - 1;
            const uint32_t inc = inc_at(i);
            const uint32_t h = seg16 & ((2u << i) - 1u);
            const int sbk = h ? P0 + 31 - __clz(h) : sbin[b];
            const uint32_t jj = (uint32_t)(P0 + i - sbk) & 127u;
            if ((REP[b] >> i) & 1u) {
                o[inc - 2] = (uint8_t)(0x80u + jj);
                o[inc - 1] = byte_at(i);
            } else {
                o[inc - 2 - jj] = (uint8_t)jj;
            }
        }
    }
    if (!EMIT)
#pragma unroll
        for (int b = 0; b < 4; ++b) T[b] = lane16(total, b);
}

// ---- basic RLE (mode 0) on the same pipeline --------------------------------
// Thesis 5.5.1's basic RLE codes 8-byte units (element pairs) in one stream
// per chunk.  The coding kernel lists the chunk's unit change points (units
// that differ from their predecessor) as it lists element change points for
// the four-plane modes; a run of one unit is literal, maximal spans of literal
// units become literal tokens and longer runs repeat tokens, both at most 128
// units per token, full tokens first.  Chunks with more change points than the
// list holds are coded by a CTA per chunk from the image (code0_block).
constexpr int kU = kChunk / 2;                       // units per chunk
constexpr int kUPer = kU / kT;                       // 8 per thread of a CTA
constexpr int kStage0 = 8 * kU + kU / 128 + 32;      // worst case + room for copy_out's read-ahead

__device__ __forceinline__ void put8(uint8_t* p, uint32_t lo, uint32_t hi)
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        p[k] = (uint8_t)(lo >> (8 * k));
        p[4 + k] = (uint8_t)(hi >> (8 * k));
    }
}

// Append the unit change points among units [kQ/2 qi, kQ/2 qi + kQ/2) of the
// chunk (unit k = elements 2k, 2k + 1) to W.cq (the unit's index) and W.ce /
// the second list `ch` (its two elements), as detect_quarter does for
// elements: a lane's 16-byte group holds two units.  carry: the unit before
// the quarter (updated to the quarter's last).  Returns false once the chunk
// has more than kCap change points.
__device__ bool detect_quarter0(const uint32_t* data, int len, int qi, WarpRing& W, uint32_t* ch, int& m,
                                uint2& carry)
{
    const int lane = threadIdx.x & 31;
    constexpr int G = kQ / 128;
    static_assert(G == 4, "four groups' counts in the bytes of one word");
    uint4 vv[G];
    uint2 pv[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        vv[g] = *reinterpret_cast<const uint4*>(data + 128 * g + 4 * lane);
        pv[g] = *reinterpret_cast<const uint2*>(data + 128 * g + 4 * lane - 2);   // g = lane = 0: guard words
    }
    if (lane == 0) pv[0] = qi == 0 ? make_uint2(~vv[0].x, vv[0].y) : carry;     // unit 0 is always listed
    carry = make_uint2(__shfl_sync(0xffffffffu, vv[G - 1].z, 31), __shfl_sync(0xffffffffu, vv[G - 1].w, 31));
    const int uend = min(len / 2 - kQ / 2 * qi, kQ / 2);                         // units of this quarter
    uint32_t f[G], packed = 0u;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const uint4 v = vv[g];
        const int u = 64 * g + 2 * lane;                  // within the quarter
        f[g] = (uint32_t)(v.x != pv[g].x || v.y != pv[g].y) | ((uint32_t)(v.z != v.x || v.w != v.y) << 1);
        if (u + 2 > uend) f[g] &= u >= uend ? 0u : 1u;
        packed |= (uint32_t)__popc(f[g]) << (8 * g);
    }
    // one warp scan of the four groups' per-lane counts (bytes of a word)
    uint32_t inc = packed;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    const uint32_t tot = __shfl_sync(0xffffffffu, inc, 31), exc = inc - packed;
    const int cnt = (int)((tot & 0xFFu) + ((tot >> 8) & 0xFFu) + ((tot >> 16) & 0xFFu) + (tot >> 24));
    if (m + cnt > kCap) return false;
    int base = m;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        if (f[g]) {
            const uint4 v = vv[g];
            const int uu = kQ / 2 * qi + 64 * g + 2 * lane;
            int o = base + (int)((exc >> (8 * g)) & 0xFFu);
            if (f[g] & 1u) { W.cq[o] = (uint16_t)uu; W.ce[o] = v.x; ch[o] = v.y; ++o; }
            if (f[g] & 2u) { W.cq[o] = (uint16_t)(uu + 1); W.ce[o] = v.z; ch[o] = v.w; }
        }
        base += (int)((tot >> (8 * g)) & 0xFFu);
    }
    m += cnt;
    return true;
}

// Mode 0, sparse path: the tokens of a chunk of nu units from its m <= 128
// unit change points (run i starts at unit cq[i], its unit is (ce[i], ch[i]),
// and it ends where run i + 1 starts, or at nu).  Lane l takes runs 4l .. 4l+3.
// A warp max-scan gives every literal run the start of its span, a sum-scan
// the place of its bytes; a repeat run writes its tokens, a literal unit its
// 8 bytes, and the unit that ends a literal token the token's control byte.
// Returns the bytes written.
__device__ uint32_t code_sparse0(const uint32_t* ce, const uint32_t* ch, const uint16_t* cq, int m, int nu,
                                 uint8_t* out)
{
    const int lane = threadIdx.x & 31;
    const int i0 = 4 * lane;
    int s[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) s[k] = i0 + k < m ? (int)cq[i0 + k] : nu;
    uint32_t lit = 0u;                                    // bit k: run i0 + k is one unit
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (i0 + k < m && s[k + 1] - s[k] == 1) lit |= 1u << k;
    const uint32_t litn = __shfl_down_sync(0xffffffffu, lit, 1);
    const uint32_t litp = __shfl_up_sync(0xffffffffu, lit, 1);
    const uint32_t lx = lit | ((lane < 31 ? (litn & 1u) : 0u) << 4);   // bit 4: the next lane's first run
    const uint32_t pre = (lit << 1) | (lane > 0 ? ((litp >> 3) & 1u) : 0u);   // bit k: run i0 + k - 1 literal
    const uint32_t starts = lit & ~pre;                   // literal runs that start a span
    // the last span start up to each lane (index + 1; 0: none)
    uint32_t last = starts ? (uint32_t)(i0 + 32 - __clz(starts)) : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, last, o);
        if (lane >= o) last = max(last, y);
    }
    uint32_t S0 = __shfl_up_sync(0xffffffffu, last, 1);
    if (lane == 0) S0 = 0u;
    uint32_t sz = 0u, S = S0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (i0 + k >= m) break;
        if ((starts >> k) & 1u) S = (uint32_t)(i0 + k + 1);
        if ((lit >> k) & 1u) sz += ((uint32_t)(i0 + k) - (S - 1u)) % 128u == 0u ? 9u : 8u;
        else sz += 9u * (((uint32_t)(s[k + 1] - s[k]) + 127u) / 128u);
    }
    uint32_t inc = sz;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
    uint32_t P = inc - sz;
    S = S0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = i0 + k;
        if (i >= m) break;
        const uint32_t lo = ce[i], hi = ch[i];
        if ((starts >> k) & 1u) S = (uint32_t)(i + 1);
        if ((lit >> k) & 1u) {
            const uint32_t p = ((uint32_t)i - (S - 1u)) % 128u;   // place in its token
            const uint32_t ts = p == 0u ? 1u : 0u;
            put8(out + P + ts, lo, hi);
            P += 8u + ts;
            if (p == 127u || !((lx >> (k + 1)) & 1u)) out[P - 8u * (p + 1u) - 1u] = (uint8_t)p;
        } else {
            for (uint32_t L = (uint32_t)(s[k + 1] - s[k]); L > 0u;) {
                const uint32_t piece = min(L, 128u);
                out[P] = (uint8_t)(127u + piece);
                put8(out + P + 1u, lo, hi);
                P += 9u;
                L -= piece;
            }
        }
    }
    return total;
}

// Exclusive block scan (sum, or max with identity 0) of one value per thread;
// *total receives the reduction over the block.
template <bool MAX>
__device__ __forceinline__ uint32_t block_excl(uint32_t v, uint32_t* wt, uint32_t* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc = MAX ? max(inc, y) : inc + y;
    }
    if (lane == 31) wt[warp] = inc;
    __syncthreads();
    uint32_t pre = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kT / 32; ++w) {
        const uint32_t t = wt[w];
        if (w < warp) pre = MAX ? max(pre, t) : pre + t;
        tot = MAX ? max(tot, t) : tot + t;
    }
    uint32_t ex = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) ex = 0u;
    *total = tot;
    __syncthreads();                                  // wt is reused by the next scan
    return MAX ? max(pre, ex) : pre + ex;
}

// Mode 0, dense path: one CTA of kT threads codes chunk [q0, q0 + len) of the
// job into stage and returns its size (the odd tail element included).  The
// chunk's elements go to e in shared memory; each thread reads its 8
// consecutive units and the two on either side into registers once (16-byte
// reads).  A unit equal to a neighbour belongs to a repeat run, the others form
// literal spans; a block max-scan gives every unit its segment's start (a run,
// or a maximal span of single units), a block sum-scan the place of its bytes,
// and the unit that ends a token writes the token's control byte.
__device__ uint32_t code0_block(const RleJobDesc& jb, uint32_t q0, int len, uint32_t* e, uint8_t* stage,
                                uint32_t* wt)
{
    const int tid = threadIdx.x;
    for (int t = tid; 4 * t < len; t += kT)
        *reinterpret_cast<uint4*>(e + 4 * t) = load_elems(jb, q0, len, 4 * t);
    __syncthreads();
    const int nu = len / 2;
    const int k0 = tid * kUPer;
    uint32_t ul[kUPer + 4], uh[kUPer + 4];           // [0,1] = k0-2, k0-1; [2..9] = k0..k0+7; [10,11] = k0+8, k0+9
    {
        const uint4* e4 = reinterpret_cast<const uint4*>(e);
        const uint4 m = tid > 0 ? e4[4 * tid - 1] : make_uint4(0u, 0u, 0u, 0u);
        ul[0] = m.x; uh[0] = m.y; ul[1] = m.z; uh[1] = m.w;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const uint4 v = e4[4 * tid + g];
            ul[2 + 2 * g] = v.x; uh[2 + 2 * g] = v.y; ul[3 + 2 * g] = v.z; uh[3 + 2 * g] = v.w;
        }
        const uint4 n = tid + 1 < kT ? e4[4 * tid + 4] : make_uint4(0u, 0u, 0u, 0u);
        ul[10] = n.x; uh[10] = n.y; ul[11] = n.z; uh[11] = n.w;
    }
    // eqp bit i: unit k0-2+i equals its predecessor (both exist), i = 0 .. 11
    uint32_t eqp = 0u;
#pragma unroll
    for (int i = 1; i < kUPer + 4; ++i) {
        const int k = k0 - 2 + i;
        if (k >= 1 && k < nu && ul[i] == ul[i - 1] && uh[i] == uh[i - 1]) eqp |= 1u << i;
    }
    // lit bit i, i = 1 .. 10: unit k0-2+i exists and equals neither neighbour
    uint32_t lit = 0u;
#pragma unroll
    for (int i = 1; i < kUPer + 3; ++i) {
        const int k = k0 - 2 + i;
        if (k >= 0 && k < nu && !((eqp >> i) & 1u) && !((eqp >> (i + 1)) & 1u)) lit |= 1u << i;
    }
    // seg bit i, i = 2 .. 10: unit k0-2+i starts a run or a span
    uint32_t seg = 0u;
#pragma unroll
    for (int i = 2; i < kUPer + 3; ++i) {
        const int k = k0 - 2 + i;
        if (k >= nu) continue;
        const bool l = (lit >> i) & 1u, lp = (lit >> (i - 1)) & 1u;
        if (k == 0 || l != lp || (!l && !((eqp >> i) & 1u))) seg |= 1u << i;
    }
    uint32_t smax = 0, ssum = 0, tot = 0;
#pragma unroll
    for (int j = 0; j < kUPer; ++j)
        if (k0 + j < nu && ((seg >> (j + 2)) & 1u)) smax = (uint32_t)(k0 + j);
    const uint32_t carry = block_excl<true>(smax, wt, &tot);
    uint32_t S = carry;
#pragma unroll
    for (int j = 0; j < kUPer; ++j) {
        const int k = k0 + j;
        if (k >= nu) break;
        if ((seg >> (j + 2)) & 1u) S = (uint32_t)k;
        const bool ts = ((uint32_t)k - S) % 128u == 0u;
        ssum += ((lit >> (j + 2)) & 1u) ? 8u + (ts ? 1u : 0u) : (ts ? 9u : 0u);
    }
    uint32_t body = 0;
    uint32_t P = block_excl<false>(ssum, wt, &body);
    S = carry;
#pragma unroll
    for (int j = 0; j < kUPer; ++j) {
        const int k = k0 + j;
        if (k >= nu) break;
        if ((seg >> (j + 2)) & 1u) S = (uint32_t)k;
        const bool l = (lit >> (j + 2)) & 1u;
        const uint32_t pos = (uint32_t)k - S;
        const bool ts = pos % 128u == 0u;
        const uint32_t sz = l ? 8u + (ts ? 1u : 0u) : (ts ? 9u : 0u);
        const bool te = k + 1 == nu || ((seg >> (j + 3)) & 1u) || ((uint32_t)k + 1u - S) % 128u == 0u;
        const uint32_t L = pos % 128u + 1u;          // units of the token so far
        if (l) {
            put8(stage + P + (ts ? 1u : 0u), ul[j + 2], uh[j + 2]);
            if (te) stage[P + sz - 1u - 8u * L] = (uint8_t)(L - 1u);
        } else {
            if (ts) put8(stage + P + 1u, ul[j + 2], uh[j + 2]);
            if (te) stage[P + sz - 9u] = (uint8_t)(128u + L - 1u);
        }
        P += sz;
    }
    if ((len & 1) && tid == 0) {
        const uint32_t v = e[len - 1];
#pragma unroll
        for (int k = 0; k < 4; ++k) stage[body + k] = (uint8_t)(v >> (8 * k));
    }
    __syncthreads();                                  // the stage is complete
    return body + ((len & 1) ? 4u : 0u);
}

// Coding kernel.  Per chunk a warp: takes its next ticket; reads the chunk's
// eight quarters, refilling each slot as soon as it has been read (with the
// next quarter of this chunk or of the next one); sizes the plane streams;
// and leaves the chunk's record and, for a sparse chunk, its streams in the
// pool (space from the warp's slab, a fresh slab taken with one atomic on the
// pool cursor when the chunk does not fit, or from the cursor chunk by chunk
// when slab is 0; a chunk that finds the pool full is coded again when
// placed, like a dense one; such chunks are listed for the recoding kernel).
// No warp waits for another.  M0: basic RLE (mode 0), from unit change points.
template <int N, bool M0>
__global__ void __launch_bounds__(32 * kWPB, 16)
k_rle_compress(const __grid_constant__ RleJobList<N> J, ChunkRec* rec, uint32_t* recode, uint8_t* pool,
               uint32_t pool_bytes, uint32_t slab, uint32_t* ticket, uint32_t* status)
{
    extern __shared__ __align__(16) uint8_t smem[];
    WarpRing& W = reinterpret_cast<WarpRing*>(smem)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const uint32_t T = J.total_units;
    unsigned long long* cursor = reinterpret_cast<unsigned long long*>(ticket + 2);   // pool bytes taken
    if (lane == 0) {
        for (int q = 0; q < kSlots; ++q) mbar_init(&W.full[q], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    uint32_t sb = 0u, sl = 0u;                          // lane 0: the warp's pool slab (base, bytes left)
    uint32_t cur = 0u;
    if (lane == 0) cur = atomicAdd(ticket, 1u);
    cur = __shfl_sync(0xffffffffu, cur, 0);
    int ji = cur < T ? find_job(J, cur) : 0;            // job of the current chunk
    if (cur < T)
        for (int q = 0; q < kSlots; ++q) issue_quarter(J.j[ji], cur, q, q, W);
    for (uint32_t seq = 0; cur < T; ++seq) {
        uint32_t nxt = 0u;
        if (lane == 0) nxt = atomicAdd(ticket, 1u);
        nxt = __shfl_sync(0xffffffffu, nxt, 0);
        const RleJobDesc& jb = J.j[ji];
        const int jn = nxt < T ? find_job(J, nxt) : 0;
        const uint32_t nc = jb.n_chunks;
        const uint32_t q0 = nc ? (cur - jb.first_unit) * (uint32_t)kChunk : 0u;
        const int len = nc ? (int)min((uint32_t)kChunk, (uint32_t)jb.w * (uint32_t)jb.h - q0) : 0;
        int m = 0;
        uint32_t carry = 0u;
        uint2 carry2 = make_uint2(0u, 0u);
        uint32_t* ch = reinterpret_cast<uint32_t*>(W.rl);    // mode 0: second element of each listed unit
        bool fits = true;
        for (int q = 0; q < kQPC; ++q) {
            const uint32_t qs = (uint32_t)kQPC * seq + (uint32_t)q;   // the warp's quarter sequence number
            const int slot = (int)(qs % kSlots);
            mbar_wait(&W.full[slot], (qs / kSlots) & 1u, status);
            if (fits && kQ * q < len)
                fits = M0 ? detect_quarter0(W.buf[slot] + 4, len, q, W, ch, m, carry2)
                          : detect_quarter(W.buf[slot] + 4, len, q, W, m, carry);
            // the quarter's values have all been consumed (compared, voted on) by
            // now, so its reads are complete before the refill below starts
            __syncwarp();
            // refill the slot with quarter qs + kSlots: of this chunk or of the next
            const int qn = q + kSlots;
            if (qn < kQPC) issue_quarter(jb, cur, qn, slot, W);
            else if (nxt < T) issue_quarter(J.j[jn], nxt, qn - kQPC, slot, W);
        }
        if (nc > 0) {
            const bool sw = jb.mode == 2;
            uint32_t Ts[4] = {0u, 0u, 0u, 0u};          // (a dense chunk is sized by the recoding kernels)
            if (fits && M0) {
                __syncwarp();
                Ts[0] = code_sparse0(W.ce, ch, W.cq, m, len / 2, W.stage);
                if (len & 1) {                            // the odd last element follows the tokens
                    if (lane == 0) put_u32(W.stage + Ts[0], __ldg(jb.src + elem_off(jb, q0 + (uint32_t)len - 1u)));
                    Ts[0] += 4u;
                }
            } else if (fits) {
                __syncwarp();
                if (sw)
                    for (int i = lane; i < m; i += 32) W.ce[i] = swizzle(W.ce[i]);
                const Lists L{W.ce, W.cq, W.rl};
                if (!code_sparse_fast(L, m, len, Ts, W.stage)) code_sparse(L, m, len, Ts, W.stage);
            }
            const uint32_t total = Ts[0] + Ts[1] + Ts[2] + Ts[3];
            uint32_t po = kRecode;
            if (fits && lane == 0) {
                // (+ 4: the copy-out reads up to one word past a chunk's bytes)
                const uint32_t need = (total + 3u) & ~3u;
                if (slab == 0u) {                         // small pools: space per chunk
                    const unsigned long long a = atomicAdd(cursor, (unsigned long long)need);
                    if (a + total + 4u <= pool_bytes) po = (uint32_t)a;
                } else {
                    // space from the warp's own slab, one atomic per slab (a
                    // sparse chunk codes to at most 4 kStagePlane <= slab bytes)
                    if (need > sl) {
                        const unsigned long long a = atomicAdd(cursor, (unsigned long long)slab);
                        sl = a + slab + 4u <= pool_bytes ? slab : 0u;
                        sb = (uint32_t)a;
                    }
                    if (need <= sl) { po = sb; sb += need; sl -= need; }
                }
            }
            po = __shfl_sync(0xffffffffu, po, 0);
            __syncwarp();
            if (po != kRecode) {                      // the four streams, back to back
                const uint32_t e1 = Ts[0], e2 = e1 + Ts[1], e3 = e2 + Ts[2];
                for (uint32_t i = lane; i < total; i += 32) {
                    const int p = (i >= e1) + (i >= e2) + (i >= e3);
                    const uint32_t b = p == 0 ? 0u : p == 1 ? e1 : p == 2 ? e2 : e3;
                    pool[po + i] = W.stage[p * kStagePlane + (i - b)];
                }
            }
            if (lane == 0) {
                ChunkRec r;
                r.T[0] = (uint16_t)Ts[0]; r.T[1] = (uint16_t)Ts[1]; r.T[2] = (uint16_t)Ts[2]; r.T[3] = (uint16_t)Ts[3];
                r.pool = po;
                r.off = 0u;
                rec[cur] = r;
                if (po == kRecode) recode[atomicAdd(ticket + 1, 1u)] = cur;   // coded again when placed
            }
            __syncwarp();
        }
        cur = nxt;
        ji = jn;
    }
}

// Scan kernel: one CTA per job.  The exclusive prefix of the job's chunk sizes
// gives every chunk its offset in the payload (written to its record); the
// job's header and stream size are written here too.
template <int N>
__global__ void __launch_bounds__(1024)
k_rle_scan(const __grid_constant__ RleJobList<N> J, ChunkRec* rec)
{
    __shared__ uint32_t wsum[32];
    const RleJobDesc& jb = J.j[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint8_t* dst = reinterpret_cast<uint8_t*>(jb.dst);
    const uint32_t nc = jb.n_chunks;
    if (nc == 0) {                                    // empty image: header only
        if (tid == 0) {
            write_header(dst, jb);
            *jb.d_size = 32u;
        }
        return;
    }
    ChunkRec* R = rec + jb.first_unit;
    const uint32_t per = (nc + blockDim.x - 1) / blockDim.x;   // contiguous chunks per thread
    const uint32_t c0 = min(nc, tid * per), c1 = min(nc, c0 + per);
    uint32_t mine = 0u;
    for (uint32_t c = c0; c < c1; ++c) mine += (uint32_t)R[c].T[0] + R[c].T[1] + R[c].T[2] + R[c].T[3];
    uint32_t inc = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    uint32_t base = inc - mine;
    for (int k = 0; k < warp; ++k) base += wsum[k];
    for (uint32_t c = c0; c < c1; ++c) {
        R[c].off = base;
        base += (uint32_t)R[c].T[0] + R[c].T[1] + R[c].T[2] + R[c].T[3];
    }
    if (tid == (int)blockDim.x - 1) {                 // its base is now the job's total
        write_header(dst, jb);
        *jb.d_size = 32ull + (jb.mode == 0 ? 4ull : 16ull) * nc + base;
    }
}

// Placing kernel: kPlaceLanes lanes (a quarter-warp) per chunk copy its
// streams from the pool to their place and write its end-table entries (four;
// one in mode 0), so a warp's four chunks have their loads in flight together.
// Chunks to be coded again are left to the recoding kernel.
constexpr int kPlaceLanes = 8;
template <int N>
__global__ void __launch_bounds__(128)
k_rle_place(const __grid_constant__ RleJobList<N> J, const ChunkRec* rec, const uint8_t* pool)
{
    const int lane = (int)threadIdx.x % kPlaceLanes;
    const uint32_t unit = blockIdx.x * (128u / kPlaceLanes) + threadIdx.x / kPlaceLanes;
    if (unit >= J.total_units) return;
    const ChunkRec r = rec[unit];                     // (in flight during the job search)
    const RleJobDesc& jb = J.j[find_job(J, unit)];
    const uint32_t nc = jb.n_chunks;
    if (nc == 0) return;                              // header written by the scan
    if (r.pool == kRecode) return;
    const uint32_t c = unit - jb.first_unit;
    const uint32_t T0 = r.T[0], T1 = r.T[1], T2 = r.T[2], T3 = r.T[3];
    const uint32_t total = T0 + T1 + T2 + T3;
    uint8_t* dst = reinterpret_cast<uint8_t*>(jb.dst);
    if (jb.mode == 0) {                               // one stream, one end-table entry
        copy_out(dst + 32 + 4ull * nc + r.off, pool + r.pool, total, lane, kPlaceLanes);
        if (lane == 0) put_u32(dst + 32 + 4ull * c, r.off + total);
        return;
    }
    copy_out(dst + 32 + 16ull * nc + r.off, pool + r.pool, total, lane, kPlaceLanes);
    const uint32_t mine = lane == 0 ? T0 : lane == 1 ? T0 + T1 : lane == 2 ? T0 + T1 + T2 : total;
    if (lane < 4) put_u32(dst + 32 + 16ull * c + 4u * lane, r.off + mine);
}

// Recoding kernels: the listed chunks (dense, or sparse ones that found the
// pool full) are coded from the image, a CTA of 8 warps per listed chunk over
// a persistent grid.  Before the scan (EMIT false) the dense ones are sized,
// their sizes written to their records; after it (EMIT true) every listed
// chunk is written straight to its place with its four end-table entries.
template <int N, bool EMIT>
__global__ void __launch_bounds__(256)
k_rle_recode(const __grid_constant__ RleJobList<N> J, ChunkRec* rec, const uint32_t* recode, const uint32_t* count)
{
    __shared__ P4 xw[16];
    const uint32_t n = *count;
    for (uint32_t i = blockIdx.x; i < n; i += gridDim.x) {
        const uint32_t unit = recode[i];
        const RleJobDesc& jb = J.j[find_job(J, unit)];
        const uint32_t nc = jb.n_chunks, c = unit - jb.first_unit;
        const ChunkRec r = rec[unit];
        uint32_t T[4] = {r.T[0], r.T[1], r.T[2], r.T[3]};
        const uint32_t total = T[0] + T[1] + T[2] + T[3];
        uint8_t* dst = reinterpret_cast<uint8_t*>(jb.dst);
        const uint32_t q0 = c * (uint32_t)kChunk;
        const int len = (int)min((uint32_t)kChunk, (uint32_t)jb.w * (uint32_t)jb.h - q0);
        if (!EMIT) {
            if (total != 0u) continue;                    // sized already (a sparse chunk)
            dense_chunk<false>(jb, q0, len, jb.mode == 2, T, nullptr, xw);
            if (threadIdx.x == 0)
#pragma unroll
                for (int p = 0; p < 4; ++p) rec[unit].T[p] = (uint16_t)T[p];
            continue;
        }
        dense_chunk<true>(jb, q0, len, jb.mode == 2, T, dst + 32 + 16ull * nc + r.off, xw);
        const uint32_t t = threadIdx.x;
        const uint32_t mine = t == 0 ? T[0] : t == 1 ? T[0] + T[1] : t == 2 ? T[0] + T[1] + T[2] : total;
        if (t < 4) put_u32(dst + 32 + 16ull * c + 4u * t, r.off + mine);
    }
}

// Mode-0 recoding kernels: as k_rle_recode, with one CTA per listed chunk
// (code0_block).  Before the scan (EMIT false) the dense chunks are sized;
// after it (EMIT true) every listed chunk is written to its place with its
// end-table entry.
template <int N, bool EMIT>
__global__ void __launch_bounds__(kT)
k_rle0_recode(const __grid_constant__ RleJobList<N> J, ChunkRec* rec, const uint32_t* recode, const uint32_t* count)
{
    __shared__ __align__(16) uint32_t e[kChunk];
    __shared__ __align__(16) uint8_t stage[kStage0];
    __shared__ uint32_t wt[kT / 32];
    const int tid = threadIdx.x;
    const uint32_t n = *count;
    for (uint32_t i = blockIdx.x; i < n; i += gridDim.x) {
        const uint32_t unit = recode[i];
        const RleJobDesc& jb = J.j[find_job(J, unit)];
        const uint32_t nc = jb.n_chunks, c = unit - jb.first_unit;
        const ChunkRec r = rec[unit];
        if (!EMIT && r.T[0] != 0u) continue;              // sized already (a sparse chunk)
        const uint32_t q0 = c * (uint32_t)kChunk;
        const int len = (int)min((uint32_t)kChunk, (uint32_t)jb.w * (uint32_t)jb.h - q0);
        const uint32_t total = code0_block(jb, q0, len, e, stage, wt);
        if (!EMIT) {
            if (tid == 0) rec[unit].T[0] = (uint16_t)total;
        } else {
            uint8_t* dst = reinterpret_cast<uint8_t*>(jb.dst);
            copy_out(dst + 32 + 4ull * nc + r.off, stage, total, tid, kT);
            if (tid == 0) put_u32(dst + 32 + 4ull * c, r.off + total);
        }
        __syncthreads();                                  // e and stage are reused
    }
}

// Self-test of the bounded waits: a warp waits on an mbarrier that nothing
// arrives on; the wait gives up after its try limit, records EC_ERR_TIMEOUT
// and the kernel returns.
__global__ void k_selftest_wait(uint32_t* status)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    mbar_wait(&bar, 0u, status);
}

// ----------------------------------------------------------- decompress ----

constexpr int kDT = 128;        // decoder CTA: one warp per byte plane


// Mode 0 (basic 64-bit RLE): the chunk's one stream [b, e) of the payload is
// staged in shared memory.  Then, up to kTok0 tokens at a time, one thread
// walks the tokens (control byte, size, bounds) and lists each token's first
// unit and stream offset in tok, and the four warps write the listed tokens,
// one token per warp and a unit per lane (8-byte stores of the unit's two
// elements where the image allows).  A unit's 8 stream bytes are funnel-
// shifted out of three aligned shared-memory words.
constexpr int kTok0 = 256;

__device__ void decode_mode0(const RleJobDesc& jb, const uint8_t* pay, uint32_t b, uint32_t e, uint32_t q0,
                             int len, uint8_t* sbuf, uint32_t* tok, uint32_t* status)
{
    __shared__ uint32_t s_ntok, s_i, s_o, s_bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t w0 = b >> 2, wl = e >> 2;          // whole words [w0, wl), then bytes [4 wl, e)
    uint32_t* st = reinterpret_cast<uint32_t*>(sbuf);
    const uint32_t* p32 = reinterpret_cast<const uint32_t*>(pay);
    for (uint32_t i = tid; w0 + i < wl; i += kDT) st[i] = __ldg(p32 + w0 + i);
    if (tid < (int)(e - 4u * wl) && wl >= w0) sbuf[4u * (wl - w0) + tid] = __ldg(pay + 4u * wl + tid);
    if (tid == 0) { s_i = b; s_o = 0u; s_bad = 0u; }
    __syncthreads();
    const uint8_t* sb = sbuf - 4u * w0;                // stream byte i at sb[i]
    const uint32_t* sw = st - w0;                      // stream word j (bytes 4j .. 4j+3) at sw[j]
    uint32_t* dst = reinterpret_cast<uint32_t*>(jb.dst);
    const bool pairs = jb.vec != 0u;                   // rows 16-byte aligned: a unit never straddles rows
    const bool dense = jb.pitch == jb.w;
    const uint32_t nu = (uint32_t)len / 2u;
    for (;;) {
        if (tid == 0) {
            uint32_t i = s_i, o = s_o, k = 0u, bad = 0u;
            while (o < nu && k < (uint32_t)kTok0) {
                if (i >= e) { bad = 1u; break; }
                const uint32_t ctl = sb[i];
                const uint32_t m = ctl < 128u ? ctl + 1u : ctl - 127u;
                const uint32_t need = ctl < 128u ? 1u + 8u * m : 9u;
                if (o + m > nu || i + need > e) { bad = 1u; break; }
                tok[k++] = o | ((i - b) << 12);
                i += need;
                o += m;
            }
            s_ntok = k; s_i = i; s_o = o; s_bad = bad;
        }
        __syncthreads();
        const uint32_t ntok = s_ntok;
        for (uint32_t t = (uint32_t)warp; t < ntok; t += kDT / 32) {
            const uint32_t r = tok[t], o = r & 0xFFFu, i = b + (r >> 12);
            const uint32_t ctl = sb[i];
            const bool lit = ctl < 128u;
            const uint32_t m = lit ? ctl + 1u : ctl - 127u;
            for (uint32_t k = (uint32_t)lane; k < m; k += 32u) {
                const uint32_t x = i + 1u + (lit ? 8u * k : 0u);   // the unit's first stream byte
                const uint32_t sh = 8u * (x & 3u), j = x >> 2;
                const uint32_t a0 = sw[j], a1 = sw[j + 1], a2 = sw[j + 2];
                const uint32_t lo = __funnelshift_r(a0, a1, sh), hi = __funnelshift_r(a1, a2, sh);
                const uint32_t q = q0 + 2u * (o + k);
                if (pairs) {
                    size_t eo = q;
                    if (!dense) {
                        const uint32_t y = q / (uint32_t)jb.w;
                        eo = (size_t)y * jb.pitch + (q - y * (uint32_t)jb.w);
                    }
                    __stcs(reinterpret_cast<uint2*>(dst + eo), make_uint2(lo, hi));
                } else {
                    dst[elem_off(jb, q)] = lo;
                    dst[elem_off(jb, q + 1u)] = hi;
                }
            }
        }
        const bool done = s_bad != 0u || s_o >= nu;
        __syncthreads();                              // tok and the shared words are reused
        if (done) break;
    }
    if (tid != 0) return;
    uint32_t i = s_i;
    bool bad = s_bad != 0u;
    if (!bad && (len & 1)) {
        if (i + 4u > e) bad = true;
        else {
            dst[elem_off(jb, q0 + (uint32_t)len - 1u)] =
                (uint32_t)sb[i] | ((uint32_t)sb[i + 1] << 8) | ((uint32_t)sb[i + 2] << 16) | ((uint32_t)sb[i + 3] << 24);
            i += 4u;
        }
    }
    if (!bad && i != e) bad = true;
    if (bad) set_status(status, EC_ERR_CORRUPT);
}

// Run path of the decoder (few runs): the chunk's elements are constant
// between the union of the four planes' run starts, so each such segment's
// element is assembled once (one byte per plane, found by the rank of the
// segment's start among that plane's run starts) and written with 16-byte
// stores of constant groups.  bm: the planes' run-start bitmaps [4][128];
// val: their run bytes [4][256]; work: shared scratch of kRunArea bytes
// (bitmaps included).
constexpr int kRunCap = 255;                        // runs per plane the run path takes
constexpr int kRunArea = 2048 + 3 * 512;            // bitmaps, union, two prefix arrays

__device__ void fill_segments(const RleJobDesc& jb, uint32_t q0, int len, bool sw, const uint32_t* bm,
                              const uint8_t* val, uint8_t* work, uint32_t* dstp)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t* U = reinterpret_cast<uint32_t*>(work + 2048);      // [128] union of run starts
    uint32_t* PU = U + 128;                                       // [128] segments before word i
    uint32_t* wt = PU + 128;                                      // per-warp totals (scan)
    uint32_t* SV = reinterpret_cast<uint32_t*>(work + kRunArea + 1024);   // segment elements
    // word tid of every bitmap; exclusive prefixes of their bit counts
    const uint32_t b0 = bm[tid], b1 = bm[128 + tid], b2 = bm[256 + tid], b3 = bm[384 + tid];
    const uint32_t u = b0 | b1 | b2 | b3;
    const uint32_t cu = __popc(u);
    const uint32_t cb = __popc(b0) | (__popc(b1) << 8) | (__popc(b2) << 16) | ((uint32_t)__popc(b3) << 24);
    uint32_t iu = cu, ib = cb;                   // (each plane has <= 255 runs: its byte never carries)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t yu = __shfl_up_sync(0xffffffffu, iu, o), yb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) { iu += yu; ib += yb; }
    }
    if (lane == 31) { wt[2 * warp] = iu; wt[2 * warp + 1] = ib; }
    __syncthreads();
    uint32_t eu = iu - cu, eb = ib - cb;
    for (int k = 0; k < warp; ++k) { eu += wt[2 * k]; eb += wt[2 * k + 1]; }
    U[tid] = u;
    PU[tid] = eu;
    // the element of every segment starting in word tid
    for (uint32_t m = u; m; m &= m - 1u) {
        const int b = __ffs(m) - 1;
        const uint32_t le = (2u << b) - 1u;      // bits 0..b
        const uint32_t r0 = ((eb >> 0) & 0xFFu) + __popc(b0 & le) - 1u;
        const uint32_t r1 = ((eb >> 8) & 0xFFu) + __popc(b1 & le) - 1u;
        const uint32_t r2 = ((eb >> 16) & 0xFFu) + __popc(b2 & le) - 1u;
        const uint32_t r3 = (eb >> 24) + __popc(b3 & le) - 1u;
        uint32_t e = (uint32_t)val[r0] | ((uint32_t)val[256 + r1] << 8) | ((uint32_t)val[512 + r2] << 16) |
                     ((uint32_t)val[768 + r3] << 24);
        if (sw) e = swizzle(e);
        SV[eu + __popc(u & (le >> 1))] = e;
    }
    __syncthreads();
    const uint32_t w = (uint32_t)jb.w;
    const bool dense = jb.pitch == jb.w;
    for (int g = tid; 4 * g < len; g += kDT) {
        const uint32_t uw = U[g >> 3];
        const int bb = (g & 7) << 2;
        const uint32_t k0 = PU[g >> 3] + __popc(uw & ((2u << bb) - 1u)) - 1u;
        const uint32_t in = (uw >> (bb + 1)) & 7u;                // segments starting inside the group
        const uint32_t k1 = k0 + (in & 1u), k2 = k1 + ((in >> 1) & 1u), k3 = k2 + (in >> 2);
        const uint32_t v0 = SV[k0];
        const uint4 v = in ? make_uint4(v0, SV[k1], SV[k2], SV[k3]) : make_uint4(v0, v0, v0, v0);
        const uint32_t q = q0 + 4u * (uint32_t)g;
        if (jb.vec) {
            size_t e = q;
            if (!dense) {
                const uint32_t y = q / w;
                e = (size_t)y * jb.pitch + (q - y * w);
            }
            st_stream(reinterpret_cast<uint4*>(dstp + e), v);
        } else {
            const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (4 * g + j < len) dstp[elem_off(jb, q + (uint32_t)j)] = vv[j];
        }
    }
}

template <int N>
__global__ void __launch_bounds__(kDT)
k_rle_decompress(const __grid_constant__ RleJobList<N> J, uint32_t* status)
{
    // the four decoded planes; a mode-0 chunk's stream (at most 8 * 2048 + 16
    // bytes) is staged here instead
    __shared__ __align__(16) uint8_t sbuf[4 * kChunk + 64];
    uint8_t (*planes)[kChunk] = reinterpret_cast<uint8_t (*)[kChunk]>(sbuf);
    __shared__ uint32_t s_beg[5];
    __shared__ int s_fail, s_over, s_mode;
    __shared__ uint8_t s_hdr[rlec::kHdrBytes];
    __shared__ uint32_t s_tok[kTok0];                 // mode 0: listed tokens

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t unit = blockIdx.x;
    // the run bitmaps start empty; nothing else uses sbuf before they are filled
#pragma unroll
    for (int i = 0; i < 4; ++i) reinterpret_cast<uint32_t*>(sbuf)[tid + kDT * i] = 0u;
    if (tid == 0) s_over = 0;
    const RleJobDesc& jb = J.j[find_job(J, unit)];
    const uint8_t* src = reinterpret_cast<const uint8_t*>(jb.src);
    const uint64_t size = jb.capacity;
    const uint32_t nc = jb.n_chunks;
    const uint32_t c = unit - jb.first_unit;

    // header (32 bytes) and this chunk's end-table entries 4c-1 .. 4c+3 (20 bytes),
    // fetched in one round trip by 52 threads
    if (tid < rlec::kHdrBytes) s_hdr[tid] = rlec::header_byte(src, size, nc, c, tid);
    __syncthreads();
    if (tid == 0) {
        const int bad = rlec::check_header(s_hdr, size, (uint32_t)jb.w, (uint32_t)jb.h, nc, c, s_beg, &s_mode, true);
        s_fail = bad;
        if (bad) set_status(status, EC_ERR_CORRUPT);
    }
    __syncthreads();
    if (s_fail || nc == 0) return;

    const uint32_t n = (uint32_t)jb.w * (uint32_t)jb.h;
    const uint32_t q0 = c * (uint32_t)kChunk;
    const int len = (int)min((uint32_t)kChunk, n - q0);
    if (s_mode == 0) {
        decode_mode0(jb, src + 32 + 4ull * nc, s_beg[0], s_beg[1], q0, len, sbuf, s_tok, status);
        return;
    }
    const uint8_t* payload = src + 32 + 16ull * nc;
    uint32_t* dstp = reinterpret_cast<uint32_t*>(jb.dst);
    const uint32_t w = (uint32_t)jb.w;
    const bool sw = s_mode == 2;

    // Runs first: warp p walks plane p's tokens, marking where each run starts
    // (every repeat token, every literal byte) and keeping its byte.
    {
        uint32_t* bm = reinterpret_cast<uint32_t*>(sbuf);          // [4][128] run starts per plane
        uint8_t* val = sbuf + kRunArea;                             // [4][256] run bytes per plane
        int nr = 0;
        const int r = rlec::decode_plane_runs(rlec::GlobalBytes{payload}, (int)s_beg[warp], (int)s_beg[warp + 1],
                                              len, bm + 128 * warp, val + 256 * warp, kRunCap, &nr, lane);
        if (lane == 0 && r == 1) s_fail = 1;
        if (lane == 0 && r == 2) s_over = 1;
        __syncthreads();
        if (s_fail) {
            if (tid == 0) set_status(status, EC_ERR_CORRUPT);
            return;
        }
        if (!s_over) {
            fill_segments(jb, q0, len, sw, bm, val, sbuf, dstp);
            return;
        }
    }

    // many runs: warp p decodes byte plane p into shared memory
    if (rlec::decode_plane(rlec::GlobalBytes{payload}, (int)s_beg[warp], (int)s_beg[warp + 1], len, planes[warp],
                           lane) &&
        lane == 0)
        s_fail = 1;
    __syncthreads();
    if (s_fail) {
        if (tid == 0) set_status(status, EC_ERR_CORRUPT);
        return;
    }

    // transpose planes back into elements, 16 per thread; groups of four
    // equal elements (each plane word one repeated byte) are un-swizzled once
    if (jb.vec) {
        const bool dense = jb.pitch == jb.w;
        for (int g16 = tid; 16 * g16 < len; g16 += kDT) {
            const uint4 A = *reinterpret_cast<const uint4*>(&planes[0][16 * g16]);
            const uint4 B = *reinterpret_cast<const uint4*>(&planes[1][16 * g16]);
            const uint4 C = *reinterpret_cast<const uint4*>(&planes[2][16 * g16]);
            const uint4 D = *reinterpret_cast<const uint4*>(&planes[3][16 * g16]);
            const uint32_t a4[4] = {A.x, A.y, A.z, A.w}, b4[4] = {B.x, B.y, B.z, B.w};
            const uint32_t c4[4] = {C.x, C.y, C.z, C.w}, d4[4] = {D.x, D.y, D.z, D.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int g = 4 * g16 + k;
                if (4 * g >= len) break;
                const uint32_t a = a4[k], bb = b4[k], c = c4[k], d = d4[k];
                uint4 v;
                if (a == bcast8(a) && bb == bcast8(bb) && c == bcast8(c) && d == bcast8(d)) {
                    uint32_t e = __byte_perm(__byte_perm(a, bb, 0x0040), __byte_perm(c, d, 0x0040), 0x5410);
                    if (sw) e = swizzle(e);
                    v = make_uint4(e, e, e, e);
                } else {
                    v = transpose4(a, bb, c, d);              // planes -> elements
                    if (sw) { v.x = swizzle(v.x); v.y = swizzle(v.y); v.z = swizzle(v.z); v.w = swizzle(v.w); }
                }
                const uint32_t q = q0 + 4u * g;
                size_t e = q;
                if (!dense) {
                    const uint32_t y = q / w;
                    e = (size_t)y * jb.pitch + (q - y * w);
                }
                st_stream(reinterpret_cast<uint4*>(dstp + e), v);
            }
        }
    } else {
        for (int t = tid; t < len; t += kDT) {
            uint32_t v = (uint32_t)planes[0][t] | ((uint32_t)planes[1][t] << 8) |
                         ((uint32_t)planes[2][t] << 16) | ((uint32_t)planes[3][t] << 24);
            if (sw) v = swizzle(v);
            const uint32_t q = q0 + t, y = q / w, x = q - y * w;
            dstp[(size_t)y * jb.pitch + x] = v;
        }
    }
}

template <int N>
RleJobList<N> make_jobs(const RleJobDesc* jobs, int n, uint32_t total)
{
    RleJobList<N> J;
    J.n = n;
    J.total_units = total;
    J.pad[0] = J.pad[1] = 0;
    for (int i = 0; i < n; ++i) J.j[i] = jobs[i];
    return J;
}

}  // namespace

namespace {

// Persistent grid: as many coding CTAs as fit on the device at once.
template <int N, bool M0>
cudaError_t compress_grid(int* grid)
{
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < kMaxDev && (*grid = cache[dev].load(std::memory_order_relaxed)) > 0) return cudaSuccess;
    e = cudaFuncSetAttribute(k_rle_compress<N, M0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCompressSmem);
    if (e != cudaSuccess) return e;
    // the persistent grid is sized for the largest shared-memory carveout:
    // ask for it, so that every CTA of the grid is resident at once
    e = cudaFuncSetAttribute(k_rle_compress<N, M0>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rle_compress<N, M0>, 32 * kWPB, kCompressSmem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    *grid = std::max(1, per_sm) * sms;
    if (dev < kMaxDev) cache[dev].store(*grid, std::memory_order_relaxed);
    return cudaSuccess;
}

// Code (persistent warps), size the dense chunks, scan the sizes (a CTA per
// job), place (a warp per chunk), write the dense chunks.  M0: basic RLE.
template <int N, bool M0>
cudaError_t compress_n(const RleJobDesc* jobs, int n, uint32_t total_units, void* scratch, size_t scratch_bytes,
                       uint32_t* status, cudaStream_t s)
{
    int grid = 0;
    cudaError_t e = compress_grid<N, M0>(&grid);
    if (e != cudaSuccess) return e;
    grid = (int)std::min<uint32_t>((uint32_t)grid, (total_units + kWPB - 1) / kWPB);
    uint32_t* ticket = reinterpret_cast<uint32_t*>(scratch);     // [0] ticket, [1] chunks to recode
    ChunkRec* rec = reinterpret_cast<ChunkRec*>(reinterpret_cast<char*>(scratch) + 16);
    uint32_t* recode = reinterpret_cast<uint32_t*>(rec + total_units);
    uint8_t* pool = reinterpret_cast<uint8_t*>(recode + ((total_units + 3u) & ~3u));
    const size_t used = rle_compress_scratch_bytes(total_units, 0);
    const uint32_t pool_bytes = (uint32_t)std::min<size_t>(scratch_bytes - used, 0xFFFFFFF0u);
    // pool space is taken in slabs of up to 16 KB per warp where the pool
    // has room for eight slabs per warp of the grid (their unused tails are
    // then at most an eighth of it), else chunk by chunk
    uint32_t slab = std::min<uint32_t>(pool_bytes / (8u * (uint32_t)grid * kWPB), 16384u) & ~255u;
    if (slab < 4u * kStagePlane) slab = 0u;
    const RleJobList<N> J = make_jobs<N>(jobs, n, total_units);
    int sms = 0;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int rgrid = std::max(1, sms) * 4;
    k_rle_compress<N, M0><<<grid, 32 * kWPB, kCompressSmem, s>>>(J, rec, recode, pool, pool_bytes, slab, ticket,
                                                                 status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (M0) k_rle0_recode<N, false><<<rgrid, kT, 0, s>>>(J, rec, recode, ticket + 1);
    else k_rle_recode<N, false><<<rgrid, 256, 0, s>>>(J, rec, recode, ticket + 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_rle_scan<N><<<n, 1024, 0, s>>>(J, rec);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_rle_place<N><<<(total_units + 128 / kPlaceLanes - 1) / (128 / kPlaceLanes), 128, 0, s>>>(J, rec, pool);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (M0) k_rle0_recode<N, true><<<rgrid, kT, 0, s>>>(J, rec, recode, ticket + 1);
    else k_rle_recode<N, true><<<rgrid, 256, 0, s>>>(J, rec, recode, ticket + 1);
    return cudaGetLastError();
}

}  // namespace

size_t rle_compress_scratch_bytes(uint32_t units, size_t pool_per_unit)
{
    const size_t u = std::max<uint32_t>(units, 1);
    return 16 + sizeof(ChunkRec) * u + 4 * ((u + 3) & ~(size_t)3) + pool_per_unit * u;
}

cudaError_t launch_rle_compress(const RleJobDesc* jobs, int n, uint32_t total_units,
                                void* scratch, size_t scratch_bytes, uint32_t* status, cudaStream_t s)
{
    if (n <= 0 || total_units == 0) return cudaSuccess;
    if (scratch_bytes < rle_compress_scratch_bytes(total_units, 0)) return cudaErrorInvalidValue;
    const cudaError_t e = cudaMemsetAsync(scratch, 0, 16, s);   // ticket, recode count, pool cursor
    if (e != cudaSuccess) return e;
    if (jobs[0].mode == 0) {                      // (one launch codes one mode family)
        if (n <= 8) return compress_n<8, true>(jobs, n, total_units, scratch, scratch_bytes, status, s);
        if (n <= 64) return compress_n<64, true>(jobs, n, total_units, scratch, scratch_bytes, status, s);
        return compress_n<kRleJobsPerLaunch, true>(jobs, n, total_units, scratch, scratch_bytes, status, s);
    }
    if (n <= 8) return compress_n<8, false>(jobs, n, total_units, scratch, scratch_bytes, status, s);
    if (n <= 64) return compress_n<64, false>(jobs, n, total_units, scratch, scratch_bytes, status, s);
    return compress_n<kRleJobsPerLaunch, false>(jobs, n, total_units, scratch, scratch_bytes, status, s);
}

cudaError_t launch_selftest_wait(uint32_t* status, cudaStream_t s)
{
    k_selftest_wait<<<1, 32, 0, s>>>(status);
    return cudaGetLastError();
}

cudaError_t launch_rle_decompress(const RleJobDesc* jobs, int n, uint32_t total_units,
                                  uint32_t* status, cudaStream_t s)
{
    if (n <= 0 || total_units == 0) return cudaSuccess;
    if (n <= 8) k_rle_decompress<8><<<total_units, kDT, 0, s>>>(make_jobs<8>(jobs, n, total_units), status);
    else if (n <= 64) k_rle_decompress<64><<<total_units, kDT, 0, s>>>(make_jobs<64>(jobs, n, total_units), status);
    else k_rle_decompress<kRleJobsPerLaunch><<<total_units, kDT, 0, s>>>(make_jobs<kRleJobsPerLaunch>(jobs, n, total_units), status);
    return cudaGetLastError();
}

}  // namespace ec
