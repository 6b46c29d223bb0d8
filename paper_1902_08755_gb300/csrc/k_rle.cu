// k_rle.cu -- run-length pixel codec kernels for sm_103a (thesis 5.5.1:
// per-component RLE, bit-swizzle preconditioner, data decomposition).
//
// Compress: persistent CTAs (four per SM) take 4096-element chunks from an
// atomic ticket and pipeline them: while chunk j+1 is copied in (cp.async),
// chunk j is coded and its size published, then chunk j-1's offset is found
// by a decoupled look-back and its bytes are copied out.
//   1. Changes: every thread compares its 16 elements with their predecessors
//      (one XOR per element; the swizzle is a bit permutation, so it commutes
//      with the XOR) and records, per byte plane, which positions start a new
//      run of equal bytes.
//   2. Sparse path (at most 512 runs in the chunk, the common case for frames
//      with flat regions): warp p lists plane p's run starts from the change
//      masks with a warp scan and codes them 32 at a time: runs of three or
//      more become repeat tokens, the first short run of a literal span codes
//      the whole span; each plane is written to its own stage region.
//   3. Dense path: each thread classifies its 16 positions for all four planes
//      with byte-SIMD compares on a plane-major copy (a byte is part of a
//      repeat iff one of the three windows of 3 around it is constant); a
//      block max-scan of segment starts splits tokens at 128 bytes and a block
//      sum-scan of per-position output sizes places every byte.
//   4. The chunk's offset inside the stream comes from the look-back over the
//      job's preceding chunks; a chunk waits only for lower tickets, which
//      running CTAs code before any higher one, and every wait is bounded
//      (EC_ERR_TIMEOUT).  Chunk 0 writes the header, every chunk its four
//      end-table entries, the last chunk the stream size.
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
constexpr int kT = 256;                              // threads per CTA
constexpr int kPer = kChunk / kT;                    // 16 positions per thread
constexpr int kPlaneCap = kChunk + kChunk / 128;     // worst-case stream bytes
constexpr int kStage = 4 * kPlaneCap;                // 16512
constexpr uint32_t kMagic = 0x31524345u;             // "ECR1"
constexpr uint64_t kAgg = 1ull << 62, kInc = 2ull << 62, kVal = (1ull << 62) - 1;
constexpr int kSpinLimit = 1 << 22;

using rlec::swizzle;
using rlec::get_u32;
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

// Two 32-bit words holding four 16-bit lanes (planes 0,1 | planes 2,3).
struct P4 { uint32_t a, b; };

template <bool MAX>
__device__ __forceinline__ P4 combine(P4 x, P4 y)
{
    if (MAX) return {__vmaxu2(x.a, y.a), __vmaxu2(x.b, y.b)};
    return {x.a + y.a, x.b + y.b};   // lanes never carry: every sum < 65536
}

// Block-wide exclusive scan of P4 values; *total receives the block total.
template <bool MAX>
__device__ __forceinline__ P4 block_scan(P4 v, P4* warp_tot, P4* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    P4 inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        P4 y;
        y.a = __shfl_up_sync(0xffffffffu, inc.a, o);
        y.b = __shfl_up_sync(0xffffffffu, inc.b, o);
        if (lane >= o) inc = combine<MAX>(inc, y);
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    P4 pre = {0u, 0u}, tot = {0u, 0u};
#pragma unroll
    for (int w = 0; w < kT / 32; ++w) {
        const P4 t = warp_tot[w];
        if (w < warp) pre = combine<MAX>(pre, t);
        tot = combine<MAX>(tot, t);
    }
    P4 ex;
    ex.a = __shfl_up_sync(0xffffffffu, inc.a, 1);
    ex.b = __shfl_up_sync(0xffffffffu, inc.b, 1);
    if (lane == 0) ex = {0u, 0u};
    *total = tot;
    return combine<MAX>(pre, ex);
}

__device__ __forceinline__ uint32_t lane16(P4 v, int p)
{
    const uint32_t w = p < 2 ? v.a : v.b;
    return (p & 1) ? (w >> 16) : (w & 0xFFFFu);
}

// ------------------------------------------------------------- compress ----

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

__device__ __forceinline__ uint64_t warp_sum(uint64_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int kSparseMax = 512;               // most segments (all planes) the sparse path takes
constexpr int kCPerSM = 4;                    // resident compress CTAs per SM
// Element buffer: 4096 elements; the dense path later reuses it for the plane-
// major copy and then as its output stage (<= kStage bytes + 16 of slack).
constexpr int kRawBytes = kStage + 16;
// Sparse stage: plane p's stream gets a region of sp_region(n_p) bytes (see
// sparse_plane), at most 3 * kSparseMax + 4 * (kChunk / 64 + 3) in all, + slack.
constexpr int kSpBytes = 3 * kSparseMax + 4 * (kChunk / 64) + 64;
constexpr int kSegBytes = 2 * kSparseMax;     // segment starts of the sparse path
constexpr int kChmBytes = 4 * kT * 2;         // one 16-bit change mask per thread and plane
constexpr size_t kCompressSmem = 3ull * kRawBytes + 2ull * kSpBytes + kSegBytes + kChmBytes;
constexpr uint32_t kNone = 0xFFFFFFFFu;
static_assert(kRawBytes % 16 == 0 && kSpBytes % 16 == 0 && kSegBytes % 16 == 0, "16-byte aligned regions");
static_assert(3 * kSparseMax + 4 * (kChunk / 64 + 3) + 16 <= kSpBytes, "sparse stage bound");

// Element q of a chunk sits at word raw_idx(q) of its buffer.  The 16-byte
// groups are permuted inside every 128 bytes (XOR with bits 3..5 of the group
// index), so that a quarter warp reading 16 consecutive elements per thread
// touches all 32 banks.
__device__ __forceinline__ int raw_idx(int q) { return (((q >> 2) ^ ((q >> 5) & 7)) << 2) | (q & 3); }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int K>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory"); }

// The chunk-size flags carry their own value, so relaxed accesses suffice.
__device__ __forceinline__ void st_flag(uint64_t* p, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t ld_flag(const uint64_t* p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Start the copy of work unit `unit`'s elements into `raw` (positions past the
// chunk's end are left as they are and never used).
__device__ void load_chunk(const RleJobDesc& jb, uint32_t unit, uint32_t* raw)
{
    const uint32_t c = unit - jb.first_unit;
    if (c >= jb.n_chunks) return;                     // empty image
    const uint32_t n = (uint32_t)jb.w * (uint32_t)jb.h, q0 = c * (uint32_t)kChunk;
    const int len = (int)min((uint32_t)kChunk, n - q0);
    const uint32_t w = (uint32_t)jb.w;
    const int tid = threadIdx.x;
    if (jb.vec) {                                     // groups of 4 never straddle a row
        const bool dense = jb.pitch == jb.w;
#pragma unroll
        for (int k = 0; k < kChunk / 4 / kT; ++k) {
            const int q = 4 * (tid + k * kT);
            if (q < len) {
                size_t e = q0 + q;
                if (!dense) {
                    const uint32_t y = (q0 + q) / w;
                    e = (size_t)y * jb.pitch + (q0 + q - y * w);
                }
                cp_async16(raw + raw_idx(q), jb.src + e);
            }
        }
    } else {
        for (int t = tid; t < len; t += kT) {
            const uint32_t q = q0 + t, y = q / w;
            cp_async4(raw + raw_idx(t), jb.src + (size_t)y * jb.pitch + (q - y * w));
        }
    }
}

// Exclusive prefix of work unit `unit`'s output inside its job's payload: the
// sizes of the preceding chunks of the job, summed 32 flags at a time back to
// one that holds its inclusive prefix; then this chunk's inclusive prefix is
// published.  Run by one warp; every wait is bounded.
__device__ uint64_t look_back(uint64_t* flags, uint32_t unit, uint32_t first_unit, uint64_t total,
                              uint32_t* status)
{
    const int lane = threadIdx.x & 31;
    if (unit == first_unit) return 0;                 // published inclusive when coded
    uint64_t acc = 0;
    int64_t hi = (int64_t)unit - 1;
    int spins = 0;
    for (;;) {
        const int64_t k = hi - lane;
        const uint64_t v = k >= (int64_t)first_unit ? ld_flag(flags + k) : kInc;
        const uint32_t st = (uint32_t)(v >> 62);
        const uint32_t incm = __ballot_sync(0xffffffffu, st == 2u);
        const uint32_t zerom = __ballot_sync(0xffffffffu, st == 0u);
        const uint32_t upto = incm ? ((incm & (0u - incm)) << 1) - 1u : 0xffffffffu;
        if (zerom & upto) {
            if (++spins > kSpinLimit) {
                if (lane == 0) set_status(status, EC_ERR_TIMEOUT);
                break;
            }
            __nanosleep(64);
            continue;
        }
        acc += warp_sum(((upto >> lane) & 1u) ? (v & kVal) : 0ull);
        if (incm) break;
        hi -= 32;
    }
    if (lane == 0) st_flag(flags + unit, kInc | (acc + total));
    return acc;
}

// What the finishing step needs of a coded chunk.
struct ChunkMeta {
    uint32_t unit, job, total, dense;
    uint32_t pend[4];        // end of plane p's stream inside the chunk's output
    uint32_t roff[4];        // sparse path: plane p's region in the stage
};

// Shared state of one compress CTA.
struct CState {
    P4 wt_a[kT / 32], wt_b[kT / 32];
    uint32_t tk[3], tj[3];   // ticket ring: work unit and its job
    uint4 wcnt[kT / 32];     // change counts per warp and plane
    uint32_t ptot[4];        // sparse path: stream size per plane
    ChunkMeta meta[2];
    uint64_t off;
};

// Publish the chunk's size: inclusive for the job's first chunk, else an
// aggregate that the look-back of later chunks may sum.
__device__ __forceinline__ void publish(uint64_t* flags, uint32_t unit, uint32_t first_unit, uint32_t total)
{
    st_flag(flags + unit, (unit == first_unit ? kInc : kAgg) | (uint64_t)total);
}

// Bytes reserved for a plane stream of n segments on the sparse path: a
// repeat segment of length L codes to 2 * ceil(L / 128) <= 2 + L / 64 bytes
// and a literal span of k short runs to at most 3k bytes, so a plane codes
// to at most 3n + kChunk / 64 bytes.
__device__ __forceinline__ uint32_t sp_region(uint32_t n) { return (3u * n + kChunk / 64 + 3u) & ~3u; }

// Sparse path, one warp per plane: the plane's segments (maximal runs of one
// byte value) are listed by start position from the change masks, then coded
// 32 at a time.  Runs of three or more become repeat tokens; the first short
// run of a literal span walks to the span's end and codes the whole span.
// Writes the stream to `out` and returns its size.
__device__ uint32_t sparse_plane(int p, const uint32_t* raw, const uint16_t* chm, uint16_t* seg,
                                 uint8_t* out, uint32_t n, int len, bool sw)
{
    const int lane = threadIdx.x & 31;
    // masks of threads 8l .. 8l+7 = positions 128l .. 128l+127, 32 per word
    const uint4 mm = *reinterpret_cast<const uint4*>(chm + p * kT + 8 * lane);
    const uint32_t c = __popc(mm.x) + __popc(mm.y) + __popc(mm.z) + __popc(mm.w);
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    uint32_t at = incl - c;
    const uint32_t wd[4] = {mm.x, mm.y, mm.z, mm.w};
#pragma unroll
    for (int k = 0; k < 4; ++k)
        for (uint32_t m = wd[k]; m; m &= m - 1u) seg[at++] = (uint16_t)(128 * lane + 32 * k + __ffs(m) - 1);
    __syncwarp();

    const int sh = 8 * p;
    uint32_t carry = 0;
    for (uint32_t r = 0; r < n; r += 32) {
        const uint32_t i = r + lane;
        uint32_t cost = 0, kind = 0;
        int s = 0, L = 0;
        if (i < n) {
            s = seg[i];
            const int e = i + 1 < n ? (int)seg[i + 1] : len;
            L = e - s;
            if (L >= 3) {
                kind = 1;
                cost = 2u * (uint32_t)((L + 127) >> 7);
            } else if (i == 0 || s - (int)seg[i - 1] >= 3) {
                int end = e;                              // first short run: find the span's end
                for (uint32_t j = i + 1; j < n; ++j) {
                    const int en = j + 1 < n ? (int)seg[j + 1] : len;
                    if (en - end >= 3) break;
                    end = en;
                }
                L = end - s;
                kind = 2;
                cost = (uint32_t)(L + ((L + 127) >> 7));
            }
        }
        uint32_t inc = cost;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        uint32_t o = carry + inc - cost;
        carry += __shfl_sync(0xffffffffu, inc, 31);
        if (kind == 1u) {
            uint32_t e = raw[raw_idx(s)];
            if (sw) e = swizzle(e);
            const uint8_t v = (uint8_t)(e >> sh);
            for (int rr = L; rr > 0; rr -= 128) {
                out[o] = (uint8_t)(127 + min(rr, 128));
                out[o + 1] = v;
                o += 2;
            }
        } else if (kind == 2u) {
            for (int d = 0; d < L; d += 128) {
                const int m = min(L - d, 128);
                out[o++] = (uint8_t)(m - 1);
                for (int t = 0; t < m; ++t) {
                    uint32_t e = raw[raw_idx(s + d + t)];
                    if (sw) e = swizzle(e);
                    out[o++] = (uint8_t)(e >> sh);
                }
            }
        }
    }
    return carry;
}

// Dense path: every position is classified with byte-SIMD bit masks on a
// plane-major copy of the chunk (pl[b * kChunk + q] = plane b of element q),
// which lies in the element buffer; once classified, that buffer becomes the
// stage.
__device__ void dense_chunk(uint8_t* pl, CState& S, ChunkMeta& M, int len,
                            uint64_t* flags, uint32_t unit, uint32_t first_unit)
{
    const int tid = threadIdx.x;
    // classify this thread's 16 positions of every plane with bit masks.
    // Bit i of the 24-bit masks stands for position P0 - 4 + i.
    const int P0 = tid * kPer;
    const uint32_t VQ = bit_range(4 - P0, len - P0 + 4);          // 0 <= q < len
    const uint32_t VEQ = bit_range(5 - P0, len - P0 + 4);         // 1 <= q < len
    const uint32_t HIGH = bit_range(len - P0 + 4, 24);            // q >= len
    const uint32_t Q0 = P0 == 0 ? (1u << 4) : 0u;                 // q == 0
    uint32_t REP[4], SEG[4];
    uint4 bytes[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const uint8_t* base = pl + b * kChunk + P0;
        const uint4 v = *reinterpret_cast<const uint4*>(base);
        // neighbours outside the chunk only feed masked-off bits
        const uint32_t wm = P0 > 0 ? *reinterpret_cast<const uint32_t*>(base - 4) : 0u;
        const uint32_t wp = P0 + kPer < kChunk ? *reinterpret_cast<const uint32_t*>(base + 16) : 0u;
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
    const uint32_t VALID = (VQ >> 4) & 0xFFFFu;

    // last segment start before each thread (max-scan of position + 1)
    P4 mine;
    {
        uint32_t l[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const uint32_t m = SEG[b] & 0xFFFFu;
            l[b] = m ? (uint32_t)(P0 + 31 - __clz(m) + 1) : 0u;
        }
        mine.a = l[0] | (l[1] << 16);
        mine.b = l[2] | (l[3] << 16);
    }
    P4 tot_max;
    const P4 before = block_scan<true>(mine, S.wt_a, &tot_max);   // (barrier inside: pl is dead after it)

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
    P4 tot;
    const P4 off0 = block_scan<false>(P4{cost[0] | (cost[1] << 16), cost[2] | (cost[3] << 16)},
                                      S.wt_b, &tot);
    uint32_t pbase[4], total = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        pbase[b] = total;
        total += lane16(tot, b);
    }
    if (tid < 4) {
        uint32_t e = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) e += b <= tid ? lane16(tot, b) : 0u;
        M.pend[tid] = e;
    }
    if (tid == 0) {
        publish(flags, unit, first_unit, total);
        M.total = total;
        M.dense = 1u;
    }

    // emit bytes and control codes into the stage
    uint8_t* stage = pl;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        uint8_t* out = stage + pbase[b];
        const uint32_t off = lane16(off0, b);
        const uint32_t lit = LIT[b], psv = PSV[b], psr = PSV[b] & REP[b], seg16 = SEG[b] & 0xFFFFu;
        const uint4 v = bytes[b];
        auto byte_at = [&](int k) -> uint8_t {
            const uint32_t wd = k < 8 ? (k < 4 ? v.x : v.y) : (k < 12 ? v.z : v.w);
            return (uint8_t)(wd >> (8 * (k & 3)));
        };
        auto inc_at = [&](int k) -> uint32_t {
            const uint32_t le = (2u << k) - 1u;
            return off + __popc(lit & le) + __popc(psv & le) + __popc(psr & le);
        };
        for (uint32_t m = lit; m; m &= m - 1u) {
            const int k = __ffs(m) - 1;
            out[inc_at(k) - 1] = byte_at(k);
        }
        for (uint32_t m = PE[b]; m; m &= m - 1u) {
            const int k = __ffs(m) - 1;
            const uint32_t inc = inc_at(k);
            const uint32_t h = seg16 & ((2u << k) - 1u);
            const int sbk = h ? P0 + 31 - __clz(h) : sbin[b];
            const uint32_t jj = (uint32_t)(P0 + k - sbk) & 127u;
            if ((REP[b] >> k) & 1u) {
                out[inc - 2] = (uint8_t)(0x80u + jj);
                out[inc - 1] = byte_at(k);
            } else {
                out[inc - 2 - jj] = (uint8_t)jj;
            }
        }
    }
}

// Code one chunk into its stage and publish its size: find where every byte
// plane changes value, count the segments, then take the sparse or the dense
// path.  `raw` holds the chunk's elements (raw_idx layout).
__device__ void code_chunk(const RleJobDesc& jb, uint32_t unit, ChunkMeta& M, uint32_t* raw, uint8_t* sp,
                           uint16_t* seg, uint16_t* chm, CState& S, uint64_t* flags)
{
    const int tid = threadIdx.x;
    const uint32_t nc = jb.n_chunks;
    if (nc == 0) return;                             // empty image: header only, when finished
    const uint32_t c = unit - jb.first_unit;
    const uint32_t n = (uint32_t)jb.w * (uint32_t)jb.h;
    const int len = (int)min((uint32_t)kChunk, n - c * (uint32_t)kChunk);
    const bool sw = jb.mode == 2;

    // 1. value changes: bit i of CH[p] is set when plane p of element P0+i
    // differs from element P0+i-1 (the swizzle permutes bits, so it commutes
    // with the XOR); position 0 starts a segment in every plane
    const int P0 = tid * kPer;
    uint32_t e[kPer];
#pragma unroll
    for (int k = 0; k < kPer / 4; ++k) {
        const uint4 v = *reinterpret_cast<const uint4*>(raw + raw_idx(P0 + 4 * k));
        e[4 * k] = v.x; e[4 * k + 1] = v.y; e[4 * k + 2] = v.z; e[4 * k + 3] = v.w;
    }
    const uint32_t prev = P0 > 0 ? raw[raw_idx(P0 - 1)] : e[0];
    const int nv = min(max(len - P0, 0), kPer);
    uint32_t nzm = 0u;
#pragma unroll
    for (int i = 0; i < kPer; ++i) nzm |= (e[i] != (i ? e[i - 1] : prev) ? 1u : 0u) << i;
    nzm &= (1u << nv) - 1u;
    uint32_t CH[4] = {0u, 0u, 0u, 0u};
    for (uint32_t m = nzm; m; m &= m - 1u) {
        const int i = __ffs(m) - 1;
        uint32_t x = raw[raw_idx(P0 + i)] ^ raw[raw_idx(P0 + i - 1)];
        if (sw) x = swizzle(x);
#pragma unroll
        for (int p = 0; p < 4; ++p) CH[p] |= ((x >> (8 * p)) & 0xFFu ? 1u : 0u) << i;
    }
    if (P0 == 0) {
#pragma unroll
        for (int p = 0; p < 4; ++p) CH[p] |= 1u;
    }

    // 2. segment counts per plane; masks to shared memory for the sparse path
    const int lane = tid & 31, warp = tid >> 5;
    uint32_t wc[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        chm[p * kT + tid] = (uint16_t)CH[p];
        wc[p] = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(CH[p]));
    }
    if (lane == 0) S.wcnt[warp] = make_uint4(wc[0], wc[1], wc[2], wc[3]);
    __syncthreads();                                 // (also: every thread has read its elements)
    uint32_t n0 = 0, n1 = 0, n2 = 0, n3 = 0;
#pragma unroll
    for (int w = 0; w < kT / 32; ++w) {
        const uint4 v = S.wcnt[w];
        n0 += v.x; n1 += v.y; n2 += v.z; n3 += v.w;
    }

    if (n0 + n1 + n2 + n3 <= (uint32_t)kSparseMax) {
        // plane p: segments at seg[lb_p ..), stream at sp + ro_p
        const uint32_t r0 = 0, r1 = sp_region(n0), r2 = r1 + sp_region(n1), r3 = r2 + sp_region(n2);
        if (warp < 4) {
            const uint32_t np = warp == 0 ? n0 : warp == 1 ? n1 : warp == 2 ? n2 : n3;
            const uint32_t lb = warp == 0 ? 0u : warp == 1 ? n0 : warp == 2 ? n0 + n1 : n0 + n1 + n2;
            const uint32_t ro = warp == 0 ? r0 : warp == 1 ? r1 : warp == 2 ? r2 : r3;
            const uint32_t t = sparse_plane(warp, raw, chm, seg + lb, sp + ro, np, len, sw);
            if (lane == 0) S.ptot[warp] = t;
        }
        __syncthreads();
        if (tid == 0) {
            const uint32_t e0 = S.ptot[0], e1 = e0 + S.ptot[1], e2 = e1 + S.ptot[2], e3 = e2 + S.ptot[3];
            publish(flags, unit, jb.first_unit, e3);
            M.total = e3;
            M.dense = 0u;
            M.pend[0] = e0; M.pend[1] = e1; M.pend[2] = e2; M.pend[3] = e3;
            M.roff[0] = r0; M.roff[1] = r1; M.roff[2] = r2; M.roff[3] = r3;
        }
    } else {
        // plane-major copy, written over the element buffer
        uint8_t* pl = reinterpret_cast<uint8_t*>(raw);
#pragma unroll
        for (int k = 0; k < kPer / 4; ++k) {
            uint32_t a = e[4 * k], b = e[4 * k + 1], cc = e[4 * k + 2], d = e[4 * k + 3];
            if (sw) { a = swizzle(a); b = swizzle(b); cc = swizzle(cc); d = swizzle(d); }
            const uint4 t = transpose4(a, b, cc, d);
            *reinterpret_cast<uint32_t*>(pl + 0 * kChunk + P0 + 4 * k) = t.x;
            *reinterpret_cast<uint32_t*>(pl + 1 * kChunk + P0 + 4 * k) = t.y;
            *reinterpret_cast<uint32_t*>(pl + 2 * kChunk + P0 + 4 * k) = t.z;
            *reinterpret_cast<uint32_t*>(pl + 3 * kChunk + P0 + 4 * k) = t.w;
        }
        __syncthreads();
        dense_chunk(pl, S, M, len, flags, unit, jb.first_unit);
    }
}

// Copy n stage bytes (src 4-byte aligned) to o, threads t, t+nt, ...: byte
// stores up to o's first word boundary and after its last, word stores of
// funnel-shifted stage words between.
__device__ __forceinline__ void copy_out(uint8_t* o, const uint8_t* src, uint32_t n, uint32_t t, uint32_t nt)
{
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(o), a1 = a0 + n;
    const uintptr_t w0 = (a0 + 3) & ~(uintptr_t)3, w1 = a1 & ~(uintptr_t)3;
    if (w0 >= w1) {
        for (uint32_t i = t; i < n; i += nt) o[i] = src[i];
        return;
    }
    const uint32_t head = (uint32_t)(w0 - a0), tail0 = (uint32_t)(w1 - a0);
    if (t < head) o[t] = src[t];
    for (uint32_t i = tail0 + t; i < n; i += nt) o[i] = src[i];
    const uint32_t nw = (uint32_t)((w1 - w0) >> 2);
    const uint32_t* s32 = reinterpret_cast<const uint32_t*>(src);
    const uint32_t sh = 8u * head;
    uint32_t* o32 = reinterpret_cast<uint32_t*>(w0);
    for (uint32_t k = t; k < nw; k += nt) {
        // bytes [head + 4k, head + 4k + 4), head < 4
        o32[k] = __funnelshift_r(s32[k], s32[k + 1], sh);
    }
}

// Place a coded chunk in its stream and copy it out: look back for its
// offset (warp 0), then write the payload bytes, the chunk's four end-table
// entries, the header (chunk 0) and the stream size (last chunk).
__device__ void finish_chunk(const RleJobDesc& jb, const ChunkMeta& M, const uint8_t* stage, CState& S,
                             uint64_t* flags, uint32_t* status)
{
    const int tid = threadIdx.x;
    uint8_t* dst = reinterpret_cast<uint8_t*>(jb.dst);
    const uint32_t nc = jb.n_chunks;
    if (nc == 0) {                                   // empty image: header only
        if (tid == 0) {
            write_header(dst, jb);
            *jb.d_size = 32u;
        }
        return;
    }
    const uint32_t c = M.unit - jb.first_unit;
    const uint32_t total = M.total;
    if (tid < 32) {
        const uint64_t acc = look_back(flags, M.unit, jb.first_unit, total, status);
        if (tid == 0) S.off = acc;
    }
    __syncthreads();
    const uint64_t G = S.off;
    uint8_t* o = dst + 32 + 16ull * nc + G;
    if (M.dense) {
        copy_out(o, stage, total, tid, kT);
    } else if (tid < 128) {                           // one warp per plane
        const int p = tid >> 5;
        const uint32_t b = p ? M.pend[p - 1] : 0u;
        copy_out(o + b, stage + M.roff[p], M.pend[p] - b, tid & 31, 32);
    }
    if (tid < 4) put_u32(dst + 32 + 16ull * c + 4u * tid, (uint32_t)(G + M.pend[tid]));
    if (tid == 0) {
        if (c == 0) write_header(dst, jb);
        if (c == nc - 1) *jb.d_size = 32ull + 16ull * nc + G + total;
    }
}

// Persistent compressor.  Each CTA takes work units (chunks) from an atomic
// ticket and runs a three-stage pipeline over them: while the copy of chunk
// j+1 is in flight, it codes chunk j and publishes its size, then looks back
// for chunk j-1's offset and copies that chunk out.  A chunk's size is thus
// published before its CTA waits on anything, and a look-back waits only for
// chunks with lower tickets, whose CTAs code them before any higher one.
template <int N>
__global__ void __launch_bounds__(kT, kCPerSM)
k_rle_compress(const __grid_constant__ RleJobList<N> J, uint64_t* flags, uint32_t* ticket,
               uint32_t* status)
{
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ CState S;
    const int tid = threadIdx.x;
    const uint32_t T = J.total_units;
    // dynamic shared memory: three element buffers, two sparse stages, the
    // sparse segment list and the change masks
    auto rawb = [&](int j) { return reinterpret_cast<uint32_t*>(smem + (j % 3) * kRawBytes); };
    auto spb = [&](int j) { return smem + 3 * kRawBytes + (j & 1) * kSpBytes; };
    uint16_t* seg = reinterpret_cast<uint16_t*>(smem + 3 * kRawBytes + 2 * kSpBytes);
    uint16_t* chm = reinterpret_cast<uint16_t*>(smem + 3 * kRawBytes + 2 * kSpBytes + kSegBytes);
    auto take = [&](int slot) {                       // thread 0
        const uint32_t u = atomicAdd(ticket, 1u);
        S.tk[slot] = u;
        S.tj[slot] = u < T ? (uint32_t)find_job(J, u) : 0u;
    };

    if (tid == 0) { take(0); take(1); }
    __syncthreads();
    uint32_t cur = S.tk[0], nxt = S.tk[1], prev = kNone;
    if (cur < T) load_chunk(J.j[S.tj[0]], cur, rawb(0));
    cp_async_commit();
    if (nxt < T) load_chunk(J.j[S.tj[1]], nxt, rawb(1));
    cp_async_commit();
    for (int j = 0; cur < T || prev != kNone; ++j) {
        cp_async_wait<1>();                           // this thread's copies of chunk j landed
        __syncthreads();
        if (cur < T) {
            ChunkMeta& M = S.meta[j & 1];
            const RleJobDesc& jb = J.j[S.tj[j % 3]];
            if (tid == 0) { M.unit = cur; M.job = S.tj[j % 3]; }
            code_chunk(jb, cur, M, rawb(j), spb(j), seg, chm, S, flags);
            __syncthreads();
        }
        if (prev != kNone) {
            const ChunkMeta& M = S.meta[(j + 1) & 1];
            const uint8_t* stage = M.dense ? reinterpret_cast<const uint8_t*>(rawb(j + 2)) : spb(j + 1);
            finish_chunk(J.j[M.job], M, stage, S, flags, status);
        }
        if (tid == 0) take((j + 2) % 3);
        __syncthreads();                              // chunk j-1's buffers are free
        const uint32_t nn = S.tk[(j + 2) % 3];
        if (nn < T) load_chunk(J.j[S.tj[(j + 2) % 3]], nn, rawb(j + 2));
        cp_async_commit();
        prev = cur < T ? cur : kNone;
        cur = nxt;
        nxt = nn;
    }
    cp_async_wait<0>();
}

// ------------------------------------------------- basic RLE, mode 0 ------
// Thesis 5.5.1's basic RLE: 8-byte units (element pairs) in one stream per
// chunk.  One CTA per chunk, taken in ticket order.  The chunk's elements are
// loaded into shared memory; each thread reads its 8 consecutive units and
// the two on either side into registers once (16-byte reads).  A unit
// equal to a neighbour belongs to a repeat run; the others form literal
// spans.  A block max-scan gives every unit its segment's start (a run, or a
// maximal span of single units), a block sum-scan the position of its bytes,
// and the unit that ends a token (at most 128 units) writes the token's
// control byte in front of it.  The chunk's offset comes from the same
// decoupled look-back as the four-plane modes.
constexpr int kU = kChunk / 2;                       // units per chunk
constexpr int kUPer = kU / kT;                       // 8 per thread
constexpr int kStage0 = 8 * kU + kU / 128 + 32;      // worst case + room for copy_out's read-ahead

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

__device__ __forceinline__ void put8(uint8_t* p, uint32_t lo, uint32_t hi)
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        p[k] = (uint8_t)(lo >> (8 * k));
        p[4 + k] = (uint8_t)(hi >> (8 * k));
    }
}

template <int N>
__global__ void __launch_bounds__(kT, 5)
k_rle0_compress(const __grid_constant__ RleJobList<N> J, uint64_t* flags, uint32_t* ticket, uint32_t* status)
{
    __shared__ __align__(16) uint32_t e[kChunk];
    __shared__ __align__(16) uint8_t stage[kStage0];
    __shared__ uint32_t wt[kT / 32];
    __shared__ uint32_t s_unit;
    __shared__ uint64_t s_off;
    const int tid = threadIdx.x;
    if (tid == 0) s_unit = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t unit = s_unit;
    const RleJobDesc& jb = J.j[find_job(J, unit)];
    const uint32_t nc = jb.n_chunks, c = unit - jb.first_unit;
    uint8_t* dst = reinterpret_cast<uint8_t*>(jb.dst);
    if (c >= nc) {                                    // empty image: header only
        if (tid == 0) {
            write_header(dst, jb);
            *jb.d_size = 32u;
        }
        return;
    }
    const uint32_t w = (uint32_t)jb.w, n = w * (uint32_t)jb.h, q0 = c * (uint32_t)kChunk;
    const int len = (int)min((uint32_t)kChunk, n - q0);
    for (int t = tid; t < len; t += kT) {
        const uint32_t q = q0 + (uint32_t)t, y = q / w;
        e[t] = __ldg(jb.src + (size_t)y * jb.pitch + (q - y * w));
    }
    __syncthreads();

    // this thread's 8 units, the two before and the two after, read once
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
    // eqp[i]: unit k0-2+i equals its predecessor (both exist), i = 0 .. 11
    uint32_t eqp = 0u;
#pragma unroll
    for (int i = 1; i < kUPer + 4; ++i) {
        const int k = k0 - 2 + i;
        if (k >= 1 && k < nu && ul[i] == ul[i - 1] && uh[i] == uh[i - 1]) eqp |= 1u << i;
    }
    // lit[i], i = 1 .. 10: unit k0-2+i exists and equals neither neighbour
    uint32_t lit = 0u;
#pragma unroll
    for (int i = 1; i < kUPer + 3; ++i) {
        const int k = k0 - 2 + i;
        if (k >= 0 && k < nu && !((eqp >> i) & 1u) && !((eqp >> (i + 1)) & 1u)) lit |= 1u << i;
    }
    // seg[i], i = 2 .. 10: unit k0-2+i starts a run or a span
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
    const uint32_t total = body + ((len & 1) ? 4u : 0u);
    if ((len & 1) && tid == 0) {
        const uint32_t v = e[len - 1];
#pragma unroll
        for (int k = 0; k < 4; ++k) stage[body + k] = (uint8_t)(v >> (8 * k));
    }
    if (tid == 0) publish(flags, unit, jb.first_unit, total);
    __syncthreads();
    if (tid < 32) {
        const uint64_t acc = look_back(flags, unit, jb.first_unit, total, status);
        if (tid == 0) s_off = acc;
    }
    __syncthreads();
    const uint64_t G = s_off;
    copy_out(dst + 32 + 4ull * nc + G, stage, total, tid, kT);
    if (tid == 0) {
        put_u32(dst + 32 + 4ull * c, (uint32_t)(G + total));
        if (c == 0) write_header(dst, jb);
        if (c == nc - 1) *jb.d_size = 32ull + 4ull * nc + G + total;
    }
}

// Self-test of the bounded waits: unit 1 looks back for unit 0, which never
// publishes its size (flags[0] stays 0); the wait gives up after its poll
// limit, records EC_ERR_TIMEOUT and the kernel returns.
__global__ void k_selftest_lookback(uint64_t* flags, uint32_t* status)
{
    if (threadIdx.x < 32) look_back(flags, 1u, 0u, 0u, status);
}

// ----------------------------------------------------------- decompress ----

constexpr int kDT = 128;        // decoder CTA: one warp per byte plane

// Element q of a job's image.
__device__ __forceinline__ size_t elem_off(const RleJobDesc& jb, uint32_t q)
{
    const uint32_t y = q / (uint32_t)jb.w;
    return (size_t)y * jb.pitch + (q - y * (uint32_t)jb.w);
}

// Mode 0 (basic 64-bit RLE): the chunk's one stream [b, e) of the payload is
// staged in shared memory, then warp 0 walks its tokens in order, every lane
// reading each control byte, and writes each token's units with its lanes.
__device__ void decode_mode0(const RleJobDesc& jb, const uint8_t* pay, uint32_t b, uint32_t e, uint32_t q0,
                             int len, uint8_t* sbuf, uint32_t* status)
{
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t w0 = b >> 2, wl = e >> 2;          // whole words [w0, wl), then bytes [4 wl, e)
    uint32_t* st = reinterpret_cast<uint32_t*>(sbuf);
    const uint32_t* p32 = reinterpret_cast<const uint32_t*>(pay);
    for (uint32_t i = tid; w0 + i < wl; i += kDT) st[i] = __ldg(p32 + w0 + i);
    if (tid < (int)(e - 4u * wl) && wl >= w0) sbuf[4u * (wl - w0) + tid] = __ldg(pay + 4u * wl + tid);
    __syncthreads();
    if (tid >= 32) return;
    const uint8_t* sb = sbuf - 4u * w0;                // stream byte i at sb[i]
    auto u32_at = [&](uint32_t i) {
        return (uint32_t)sb[i] | ((uint32_t)sb[i + 1] << 8) | ((uint32_t)sb[i + 2] << 16) | ((uint32_t)sb[i + 3] << 24);
    };
    uint32_t* dst = reinterpret_cast<uint32_t*>(jb.dst);
    const int nu = len / 2;
    uint32_t i = b;
    int o = 0, bad = 0;
    while (o < nu) {
        if (i >= e) { bad = 1; break; }
        const uint32_t ctl = sb[i];
        const int m = ctl < 128u ? (int)ctl + 1 : (int)ctl - 127;
        const uint32_t need = ctl < 128u ? 1u + 8u * (uint32_t)m : 9u;
        if (o + m > nu || i + need > e) { bad = 1; break; }
        for (int k = lane; k < m; k += 32) {
            const uint32_t v = ctl < 128u ? i + 1u + 8u * (uint32_t)k : i + 1u;
            const uint32_t q = q0 + 2u * (uint32_t)(o + k);
            dst[elem_off(jb, q)] = u32_at(v);
            dst[elem_off(jb, q + 1u)] = u32_at(v + 4u);
        }
        i += need;
        o += m;
    }
    if (!bad && (len & 1)) {
        if (i + 4u > e) bad = 1;
        else {
            if (lane == 0) dst[elem_off(jb, q0 + (uint32_t)len - 1u)] = u32_at(i);
            i += 4u;
        }
    }
    if (!bad && i != e) bad = 1;
    if (bad && lane == 0) set_status(status, EC_ERR_CORRUPT);
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
    __shared__ int s_fail, s_mode;
    __shared__ uint8_t s_hdr[rlec::kHdrBytes];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t unit = blockIdx.x;
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
        decode_mode0(jb, src + 32 + 4ull * nc, s_beg[0], s_beg[1], q0, len, sbuf, status);
        return;
    }
    const uint8_t* payload = src + 32 + 16ull * nc;

    // warp p decodes byte plane p
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
    uint32_t* dstp = reinterpret_cast<uint32_t*>(jb.dst);
    const uint32_t w = (uint32_t)jb.w;
    const bool sw = s_mode == 2;
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

// Persistent grid: as many compress CTAs as fit on the device at once (the
// kernel's dynamic shared memory attribute is set on first use per device).
template <int N>
cudaError_t compress_grid(int* grid)
{
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < kMaxDev && (*grid = cache[dev].load(std::memory_order_relaxed)) > 0) return cudaSuccess;
    e = cudaFuncSetAttribute(k_rle_compress<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCompressSmem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rle_compress<N>, kT, kCompressSmem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    *grid = std::max(1, per_sm) * sms;
    if (dev < kMaxDev) cache[dev].store(*grid, std::memory_order_relaxed);
    return cudaSuccess;
}

template <int N>
cudaError_t compress_n(const RleJobDesc* jobs, int n, uint32_t total_units, uint64_t* flags,
                       uint32_t* ticket, uint32_t* status, cudaStream_t s)
{
    int grid = 0;
    const cudaError_t e = compress_grid<N>(&grid);
    if (e != cudaSuccess) return e;
    grid = (int)std::min<uint32_t>((uint32_t)grid, total_units);
    k_rle_compress<N><<<grid, kT, kCompressSmem, s>>>(make_jobs<N>(jobs, n, total_units), flags, ticket, status);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rle_compress(const RleJobDesc* jobs, int n, uint32_t total_units,
                                void* scratch, uint32_t* status, cudaStream_t s)
{
    if (n <= 0 || total_units == 0) return cudaSuccess;
    uint32_t* ticket = reinterpret_cast<uint32_t*>(scratch);
    uint64_t* flags = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(scratch) + 16);
    cudaError_t e = cudaMemsetAsync(scratch, 0, 16 + 8ull * total_units, s);
    if (e != cudaSuccess) return e;
    if (jobs[0].mode == 0) {                      // basic RLE: one CTA per chunk
        if (n <= 8) k_rle0_compress<8><<<total_units, kT, 0, s>>>(make_jobs<8>(jobs, n, total_units), flags, ticket, status);
        else if (n <= 64) k_rle0_compress<64><<<total_units, kT, 0, s>>>(make_jobs<64>(jobs, n, total_units), flags, ticket, status);
        else k_rle0_compress<kRleJobsPerLaunch><<<total_units, kT, 0, s>>>(make_jobs<kRleJobsPerLaunch>(jobs, n, total_units), flags, ticket, status);
        return cudaGetLastError();
    }
    if (n <= 8) return compress_n<8>(jobs, n, total_units, flags, ticket, status, s);
    if (n <= 64) return compress_n<64>(jobs, n, total_units, flags, ticket, status, s);
    return compress_n<kRleJobsPerLaunch>(jobs, n, total_units, flags, ticket, status, s);
}

cudaError_t launch_selftest_lookback(void* scratch, uint32_t* status, cudaStream_t s)
{
    const cudaError_t e = cudaMemsetAsync(scratch, 0, 16, s);
    if (e != cudaSuccess) return e;
    k_selftest_lookback<<<1, 32, 0, s>>>(reinterpret_cast<uint64_t*>(scratch), status);
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
