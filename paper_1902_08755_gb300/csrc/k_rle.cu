// k_rle.cu -- run-length pixel codec kernels for sm_103a (thesis 5.5.1:
// per-component RLE, bit-swizzle preconditioner, data decomposition).
//
// Compress: one CTA per 4096-element chunk, single pass over the input.
//   1. 16-byte loads of the chunk into shared memory (swizzled in registers for
//      mode 2).  The layout pads 4 words after every 32 so that each thread's
//      16 consecutive words read back without bank conflicts.
//   2. Each thread classifies its 16 positions for all four byte planes at once
//      with byte-SIMD compares (one 32-bit word = the four planes of an
//      element): a byte is part of a repeat iff one of the three windows of 3
//      around it is constant, which needs only +-2 neighbours.
//   3. Token boundaries need each position's offset inside its run or literal
//      span (tokens hold at most 128 bytes): a block-wide max-scan of segment
//      starts, two planes per word as 16-bit lanes (__vmaxu2).
//   4. A block-wide sum-scan of per-position output sizes (again 16-bit lanes)
//      gives every byte its output offset; bytes and control codes are
//      scattered into a shared-memory stage.
//   5. The chunk's offset inside the stream comes from a decoupled look-back
//      over preceding chunks (chunk order from an atomic ticket, so every
//      chunk waited on belongs to a CTA that is already running); every wait
//      is bounded and records EC_ERR_TIMEOUT if it gives up.
//   6. The stage is copied out with word stores; chunk 0 writes the header,
//      every chunk its four end-table entries, the last chunk the size.
//
// Decompress: one CTA per chunk.  The header and the chunk's end-table entries
// are validated, the chunk's compressed bytes are staged in shared memory, one
// walker thread per plane parses token headers into a list (bounds-checked,
// in rounds of kTok tokens) while all warps expand the listed tokens, and the
// four planes are transposed back into elements with byte permutes.
#include "ec_internal.cuh"

namespace ec {
namespace {

constexpr int kChunk = EC_RLE_CHUNK;                 // 4096 elements
constexpr int kT = 256;                              // threads per CTA
constexpr int kPer = kChunk / kT;                    // 16 positions per thread
constexpr int kPlaneCap = kChunk + kChunk / 128;     // worst-case stream bytes
constexpr int kStage = 4 * kPlaneCap;                // 16512
constexpr int kSmemWords = kChunk + (kChunk / 32) * 4;
constexpr uint32_t kMagic = 0x31524345u;             // "ECR1"
constexpr uint64_t kAgg = 1ull << 62, kInc = 2ull << 62, kVal = (1ull << 62) - 1;
constexpr int kSpinLimit = 1 << 22;
constexpr int kTok = 256;                            // tokens per plane per round

__device__ __forceinline__ int pidx(int q) { return q + ((q >> 5) << 2); }

// Bit-swizzle: byte k of the result gathers bit pair (7-2k, 6-2k) of the four
// components, component 0 (R) in the top pair.  This is a transpose of the 4x4
// matrix of 2-bit cells, done as two delta swaps; it is its own inverse.
__device__ __forceinline__ uint32_t swizzle(uint32_t x)
{
    uint32_t t = ((x >> 20) ^ x) & 0x00000F0Fu;
    x ^= t ^ (t << 20);
    t = ((x >> 10) ^ x) & 0x00330033u;
    x ^= t ^ (t << 10);
    return x;
}

__device__ __forceinline__ void st_release(uint64_t* p, uint64_t v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t ld_acquire(const uint64_t* p)
{
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

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

__device__ __forceinline__ uint32_t get_u32(const uint8_t* p)
{
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
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
    put_u32(d + 28, 4u);
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

template <int N>
__global__ void __launch_bounds__(kT)
k_rle_compress(const __grid_constant__ RleJobList<N> J, uint64_t* flags, uint32_t* ticket,
               uint32_t* status)
{
    __shared__ __align__(16) uint32_t se[kSmemWords];
    __shared__ __align__(16) uint8_t stage[kStage + 16];
    __shared__ P4 wt_max[kT / 32], wt_sum[kT / 32];
    __shared__ uint32_t s_unit;
    __shared__ uint64_t s_off;

    const int tid = threadIdx.x;
    if (tid == 0) s_unit = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t unit = s_unit;
    if (unit >= J.total_units) return;               // cannot happen: one ticket per CTA
    const RleJobDesc& jb = J.j[find_job(J, unit)];
    uint8_t* dst = reinterpret_cast<uint8_t*>(jb.dst);
    const uint32_t nc = jb.n_chunks;
    if (nc == 0) {                                   // empty image: header only
        if (tid == 0) {
            write_header(dst, jb);
            *jb.d_size = 32u;
        }
        return;
    }
    const uint32_t c = unit - jb.first_unit;
    const uint32_t n = (uint32_t)jb.w * (uint32_t)jb.h;
    const uint32_t q0 = c * (uint32_t)kChunk;
    const int len = (int)min((uint32_t)kChunk, n - q0);
    const uint32_t w = (uint32_t)jb.w;

    // 1. load
    if (jb.vec) {
        for (int g = tid; 4 * g < len; g += kT) {
            const uint32_t q = q0 + 4u * g, y = q / w, x = q - y * w;
            uint4 v = ld_stream(reinterpret_cast<const uint4*>(jb.src + (size_t)y * jb.pitch + x));
            if (jb.mode == 2) { v.x = swizzle(v.x); v.y = swizzle(v.y); v.z = swizzle(v.z); v.w = swizzle(v.w); }
            *reinterpret_cast<uint4*>(se + pidx(4 * g)) = v;
        }
    } else {
        for (int t = tid; t < len; t += kT) {
            const uint32_t q = q0 + t, y = q / w, x = q - y * w;
            uint32_t v = __ldcs(jb.src + (size_t)y * jb.pitch + x);
            if (jb.mode == 2) v = swizzle(v);
            se[pidx(t)] = v;
        }
    }
    __syncthreads();

    // 2. classify positions P0-3 .. P0+19 (i = p - P0 + 3)
    const int P0 = tid * kPer;
    constexpr int NV = kPer + 7;
    uint32_t val[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        const int p = P0 - 3 + i;
        val[i] = (p >= 0 && p < len) ? se[pidx(p)] : 0u;
    }
    uint32_t eq[NV];
    eq[0] = 0u;
#pragma unroll
    for (int i = 1; i < NV; ++i) {
        const int p = P0 - 3 + i;
        eq[i] = (p >= 1 && p < len) ? __vcmpeq4(val[i], val[i - 1]) : 0u;
    }
    uint32_t t3[NV];
    t3[0] = t3[1] = 0u;
#pragma unroll
    for (int i = 2; i < NV; ++i) t3[i] = eq[i] & eq[i - 1];
    // rep[i] for i in [2, NV-2): the byte lies in a run of >= 3
    uint32_t rep[NV];
#pragma unroll
    for (int i = 2; i < NV - 2; ++i) rep[i] = t3[i] | t3[i + 1] | t3[i + 2];
    // segment starts at p in [P0, P0+16); positions >= len count as starts.
    // Mlo holds planes 0 (bits 0-15) and 1 (bits 16-31), Mhi planes 2 and 3.
    uint32_t Mlo = 0u, Mhi = 0u;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int i = k + 3, p = P0 + k;
        uint32_t seg;
        if (p >= len) {
            seg = 0xFFFFFFFFu;
        } else {
            const uint32_t rs = rep[i] & ~eq[i];
            const uint32_t ls = ~rep[i] & (p == 0 ? 0xFFFFFFFFu : rep[i - 1]);
            seg = rs | ls;
        }
        Mlo |= ((seg >> 7) & 1u) << k | ((seg >> 15) & 1u) << (k + 16);
        Mhi |= ((seg >> 23) & 1u) << k | ((seg >> 31) & 1u) << (k + 16);
    }
    // 16-bit mask of segment starts at positions P0..P0+15 of one plane
    auto mask_of = [&](int pl) -> uint32_t {
        const uint32_t m = pl < 2 ? Mlo : Mhi;
        return (pl & 1) ? (m >> 16) : (m & 0xFFFFu);
    };
    // whether position P0+16 starts a segment, per plane
    uint32_t next_seg[4];
    {
        const int p = P0 + kPer;
        uint32_t seg;
        if (p >= len) {
            seg = 0xFFFFFFFFu;
        } else {
            const int i = kPer + 3;
            const uint32_t rs = rep[i] & ~eq[i];
            const uint32_t ls = ~rep[i] & rep[i - 1];
            seg = rs | ls;
        }
#pragma unroll
        for (int pl = 0; pl < 4; ++pl) next_seg[pl] = (seg >> (8 * pl + 7)) & 1u;
    }

    // 3. last segment start before this thread (max-scan of position + 1)
    P4 mine;
    {
        uint32_t l[4];
#pragma unroll
        for (int pl = 0; pl < 4; ++pl) {
            const uint32_t m = mask_of(pl);
            l[pl] = m ? (uint32_t)(P0 + 31 - __clz(m) + 1) : 0u;
        }
        mine.a = l[0] | (l[1] << 16);
        mine.b = l[2] | (l[3] << 16);
    }
    P4 tot_max;
    const P4 before = block_scan<true>(mine, wt_max, &tot_max);

    // 4. output sizes: repeat piece start 2, literal piece start 2, literal 1
    uint32_t cost[4];
#pragma unroll
    for (int pl = 0; pl < 4; ++pl) {
        const uint32_t m = mask_of(pl);
        int sb = (int)lane16(before, pl) - 1;
        uint32_t sum = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int p = P0 + k;
            if (p < len) {
                if ((m >> k) & 1u) sb = p;
                const bool ps = ((p - sb) & 127) == 0;
                const bool isrep = (rep[k + 3] >> (8 * pl)) & 0xFFu;
                sum += isrep ? (ps ? 2u : 0u) : (ps ? 2u : 1u);
            }
        }
        cost[pl] = sum;
    }
    P4 tot;
    const P4 off0 = block_scan<false>(P4{cost[0] | (cost[1] << 16), cost[2] | (cost[3] << 16)},
                                      wt_sum, &tot);
    uint32_t ptot[4], pbase[4], total = 0;
#pragma unroll
    for (int pl = 0; pl < 4; ++pl) {
        ptot[pl] = lane16(tot, pl);
        pbase[pl] = total;
        total += ptot[pl];
    }

    // 5. chunk offset: decoupled look-back (thread 0), bounded waits
    if (tid == 0) {
        uint64_t* f = flags + unit;
        if (c == 0) {
            st_release(f, kInc | (uint64_t)total);
            s_off = 0;
        } else {
            st_release(f, kAgg | (uint64_t)total);
            uint64_t acc = 0;
            uint32_t k = unit - 1;
            int spins = 0;
            for (;;) {
                const uint64_t v = ld_acquire(flags + k);
                if ((v & ~kVal) == 0) {
                    if (++spins > kSpinLimit) {
                        set_status(status, EC_ERR_TIMEOUT);
                        break;
                    }
                    __nanosleep(64);
                    continue;
                }
                acc += v & kVal;
                if ((v & ~kVal) == kInc || k == jb.first_unit) break;
                --k;
            }
            st_release(f, kInc | (acc + total));
            s_off = acc;
        }
    }

    // emit into the stage
#pragma unroll
    for (int pl = 0; pl < 4; ++pl) {
        const uint32_t m = mask_of(pl) | (next_seg[pl] << kPer);
        int sb = (int)lane16(before, pl) - 1;
        uint32_t off = lane16(off0, pl);
        uint8_t* out = stage + pbase[pl];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int p = P0 + k;
            if (p < len) {
                if ((m >> k) & 1u) sb = p;
                const int j = p - sb;
                const bool ps = (j & 127) == 0;
                const bool isrep = (rep[k + 3] >> (8 * pl)) & 0xFFu;
                off += isrep ? (ps ? 2u : 0u) : (ps ? 2u : 1u);
                const bool last = ((m >> (k + 1)) & 1u) || ((j + 1) & 127) == 0;
                const uint8_t byte = (uint8_t)(val[k + 3] >> (8 * pl));
                if (isrep) {
                    if (last) {
                        out[off - 2] = (uint8_t)(0x80 + (j & 127));
                        out[off - 1] = byte;
                    }
                } else {
                    out[off - 1] = byte;
                    if (last) out[off - 2 - (j & 127)] = (uint8_t)(j & 127);
                }
            }
        }
    }
    __syncthreads();

    // 6. copy out
    const uint64_t G = s_off;
    uint8_t* payload = dst + 32 + 16ull * nc;
    uint8_t* o = payload + G;
    {
        const uintptr_t a0 = reinterpret_cast<uintptr_t>(o), a1 = a0 + total;
        const uintptr_t w0 = (a0 + 3) & ~(uintptr_t)3, w1 = a1 & ~(uintptr_t)3;
        if (w0 >= w1) {
            for (uint32_t i = tid; i < total; i += kT) o[i] = stage[i];
        } else {
            const uint32_t head = (uint32_t)(w0 - a0), tail0 = (uint32_t)(w1 - a0);
            if (tid < head) o[tid] = stage[tid];
            for (uint32_t i = tail0 + tid; i < total; i += kT) o[i] = stage[i];
            const uint32_t nw = (uint32_t)((w1 - w0) >> 2);
            const uint32_t* s32 = reinterpret_cast<const uint32_t*>(stage);
            const uint32_t sh = 8u * (head & 3u);
            uint32_t* o32 = reinterpret_cast<uint32_t*>(w0);
            for (uint32_t k = tid; k < nw; k += kT) {
                // stage bytes [head + 4k, head + 4k + 4): head < 4
                const uint32_t lo = s32[k + (head >> 2)], hi = s32[k + (head >> 2) + 1];
                o32[k] = __funnelshift_r(lo, hi, sh);
            }
        }
    }
    if (tid < 4) put_u32(dst + 32 + 16ull * c + 4u * tid, (uint32_t)(G + pbase[tid] + ptot[tid]));
    if (tid == 0) {
        if (c == 0) write_header(dst, jb);
        if (c == nc - 1) *jb.d_size = 32ull + 16ull * nc + G + total;
    }
}

// ----------------------------------------------------------- decompress ----

template <int N>
__global__ void __launch_bounds__(kT)
k_rle_decompress(const __grid_constant__ RleJobList<N> J, uint32_t* status)
{
    __shared__ __align__(16) uint8_t sbuf[kStage + 16];
    __shared__ __align__(16) uint8_t planes[4][kChunk];
    __shared__ uint2 toks[4][kTok];
    __shared__ int ntok[4], pref[5];
    __shared__ uint32_t s_beg[5];
    __shared__ int s_fail, s_mode, s_live;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t unit = blockIdx.x;
    const RleJobDesc& jb = J.j[find_job(J, unit)];
    const uint8_t* src = reinterpret_cast<const uint8_t*>(jb.src);
    const uint64_t size = jb.capacity;
    const uint32_t nc = jb.n_chunks;
    const uint32_t c = unit - jb.first_unit;

    if (tid == 0) {
        int bad = 0;
        if (size < 32) bad = 1;
        else {
            const uint32_t mode = (uint32_t)src[6] | ((uint32_t)src[7] << 8);
            bad |= get_u32(src) != kMagic;
            bad |= (src[4] | (src[5] << 8)) != 1;
            bad |= mode != 1u && mode != 2u;
            bad |= get_u32(src + 8) != (uint32_t)jb.w || get_u32(src + 12) != (uint32_t)jb.h;
            bad |= get_u32(src + 16) != 4u || get_u32(src + 20) != (uint32_t)kChunk;
            bad |= get_u32(src + 24) != nc || get_u32(src + 28) != 4u;
            s_mode = (int)mode;
            if (!bad && size < 32ull + 16ull * nc) bad = 1;
            if (!bad && nc > 0) {
                const uint8_t* tab = src + 32;
                const uint64_t psize = size - 32ull - 16ull * nc;
                const uint32_t n = (uint32_t)jb.w * (uint32_t)jb.h;
                const uint32_t clen = min((uint32_t)kChunk, n - c * (uint32_t)kChunk);
                const uint32_t cap = clen + (clen + 127u) / 128u;   // all-literal coding
                s_beg[0] = c == 0 ? 0u : get_u32(tab + 4u * (4u * c - 1u));
                for (int p = 0; p < 4; ++p) {
                    s_beg[p + 1] = get_u32(tab + 4u * (4u * c + p));
                    bad |= s_beg[p + 1] < s_beg[p];
                    bad |= s_beg[p + 1] - s_beg[p] > cap;   // longer than any valid stream
                }
                bad |= (uint64_t)s_beg[4] > psize;
            }
        }
        s_fail = bad;
        if (bad) set_status(status, EC_ERR_CORRUPT);
    }
    __syncthreads();
    if (s_fail || nc == 0) return;

    const uint32_t n = (uint32_t)jb.w * (uint32_t)jb.h;
    const uint32_t q0 = c * (uint32_t)kChunk;
    const int len = (int)min((uint32_t)kChunk, n - q0);
    const uint8_t* payload = src + 32 + 16ull * nc;
    const uint32_t b0 = s_beg[0], nbytes = s_beg[4] - b0;
    for (uint32_t i = tid; i < nbytes; i += kT) sbuf[i] = payload[b0 + i];

    // token walk (lane 0 of warps 0..3, one plane each) + cooperative expansion
    int in = 0, in_end = 0, outp = 0;
    bool done = true;
    if (lane == 0 && warp < 4) {
        in = (int)(s_beg[warp] - b0);
        in_end = (int)(s_beg[warp + 1] - b0);
        done = false;
    }
    if (tid == 0) s_live = 4;
    __syncthreads();
    for (;;) {
        if (lane == 0 && warp < 4) {
            int cnt = 0;
            if (!done) {
                while (cnt < kTok && in < in_end) {
                    const int ctl = sbuf[in];
                    int m, next;
                    uint32_t rep;
                    if (ctl < 128) { m = ctl + 1; next = in + 1 + m; rep = 0; }
                    else { m = ctl - 127; next = in + 2; rep = 1; }
                    if (next > in_end || outp + m > len) { s_fail = 1; break; }
                    toks[warp][cnt++] = make_uint2((uint32_t)outp | ((uint32_t)(m - 1) << 16) | (rep << 31),
                                                   (uint32_t)(in + 1));
                    outp += m;
                    in = next;
                }
                if (in >= in_end && !s_fail) {
                    done = true;
                    if (outp != len) s_fail = 1;
                    atomicSub(&s_live, 1);
                }
            }
            ntok[warp] = cnt;
        }
        __syncthreads();
        if (s_fail) {
            if (tid == 0) set_status(status, EC_ERR_CORRUPT);
            return;
        }
        if (tid == 0) {
            pref[0] = 0;
            for (int p = 0; p < 4; ++p) pref[p + 1] = pref[p] + ntok[p];
        }
        __syncthreads();
        for (int t = warp; t < pref[4]; t += kT / 32) {
            const int p = t < pref[1] ? 0 : t < pref[2] ? 1 : t < pref[3] ? 2 : 3;
            const uint2 tk = toks[p][t - pref[p]];
            const int o = (int)(tk.x & 0xFFFFu), m = (int)((tk.x >> 16) & 0x7Fu) + 1;
            const int s0 = (int)tk.y;
            if (tk.x >> 31) {
                const uint8_t v = sbuf[s0];
                for (int i = lane; i < m; i += 32) planes[p][o + i] = v;
            } else {
                for (int i = lane; i < m; i += 32) planes[p][o + i] = sbuf[s0 + i];
            }
        }
        __syncthreads();
        if (s_live == 0) break;
    }

    // transpose planes back into elements
    uint32_t* dstp = reinterpret_cast<uint32_t*>(jb.dst);
    const uint32_t w = (uint32_t)jb.w;
    const bool sw = s_mode == 2;
    if (jb.vec) {
        for (int g = tid; 4 * g < len; g += kT) {
            const uint32_t A = *reinterpret_cast<const uint32_t*>(&planes[0][4 * g]);
            const uint32_t B = *reinterpret_cast<const uint32_t*>(&planes[1][4 * g]);
            const uint32_t C = *reinterpret_cast<const uint32_t*>(&planes[2][4 * g]);
            const uint32_t D = *reinterpret_cast<const uint32_t*>(&planes[3][4 * g]);
            const uint32_t ab_lo = __byte_perm(A, B, 0x5140), cd_lo = __byte_perm(C, D, 0x5140);
            const uint32_t ab_hi = __byte_perm(A, B, 0x7362), cd_hi = __byte_perm(C, D, 0x7362);
            uint4 v = make_uint4(__byte_perm(ab_lo, cd_lo, 0x5410), __byte_perm(ab_lo, cd_lo, 0x7632),
                                 __byte_perm(ab_hi, cd_hi, 0x5410), __byte_perm(ab_hi, cd_hi, 0x7632));
            if (sw) { v.x = swizzle(v.x); v.y = swizzle(v.y); v.z = swizzle(v.z); v.w = swizzle(v.w); }
            const uint32_t q = q0 + 4u * g, y = q / w, x = q - y * w;
            st_stream(reinterpret_cast<uint4*>(dstp + (size_t)y * jb.pitch + x), v);
        }
    } else {
        for (int t = tid; t < len; t += kT) {
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

cudaError_t launch_rle_compress(const RleJobDesc* jobs, int n, uint32_t total_units,
                                void* scratch, uint32_t* status, cudaStream_t s)
{
    if (n <= 0 || total_units == 0) return cudaSuccess;
    uint32_t* ticket = reinterpret_cast<uint32_t*>(scratch);
    uint64_t* flags = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(scratch) + 16);
    cudaError_t e = cudaMemsetAsync(scratch, 0, 16 + 8ull * total_units, s);
    if (e != cudaSuccess) return e;
    if (n <= 8) k_rle_compress<8><<<total_units, kT, 0, s>>>(make_jobs<8>(jobs, n, total_units), flags, ticket, status);
    else if (n <= 64) k_rle_compress<64><<<total_units, kT, 0, s>>>(make_jobs<64>(jobs, n, total_units), flags, ticket, status);
    else k_rle_compress<kRleJobsPerLaunch><<<total_units, kT, 0, s>>>(make_jobs<kRleJobsPerLaunch>(jobs, n, total_units), flags, ticket, status);
    return cudaGetLastError();
}

cudaError_t launch_rle_decompress(const RleJobDesc* jobs, int n, uint32_t total_units,
                                  uint32_t* status, cudaStream_t s)
{
    if (n <= 0 || total_units == 0) return cudaSuccess;
    if (n <= 8) k_rle_decompress<8><<<total_units, kT, 0, s>>>(make_jobs<8>(jobs, n, total_units), status);
    else if (n <= 64) k_rle_decompress<64><<<total_units, kT, 0, s>>>(make_jobs<64>(jobs, n, total_units), status);
    else k_rle_decompress<kRleJobsPerLaunch><<<total_units, kT, 0, s>>>(make_jobs<kRleJobsPerLaunch>(jobs, n, total_units), status);
    return cudaGetLastError();
}

}  // namespace ec
