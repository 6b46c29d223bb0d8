// rle_codec.cuh -- device pieces of the RLE container (thesis 5.5.1) shared by
// the decoder kernel and the fused decode-and-composite kernel: the swizzle,
// byte transposes, header and end-table validation, and the warp-wide decoder
// of one byte-plane stream.
#pragma once

#include "ec_internal.cuh"

namespace ec {
namespace rlec {

constexpr int kChunk = EC_RLE_CHUNK;                 // 4096 elements
constexpr uint32_t kMagic = 0x31524345u;             // "ECR1"
constexpr int kHdrBytes = 60;                        // header + 5 four-plane and 2 one-plane entries

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

__device__ __forceinline__ uint32_t get_u32(const uint8_t* p)
{
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

// 4x4 byte transpose: word b of the result holds byte b of e0..e3 (e0 lowest).
__device__ __forceinline__ uint4 transpose4(uint32_t e0, uint32_t e1, uint32_t e2, uint32_t e3)
{
    const uint32_t lo01 = __byte_perm(e0, e1, 0x5140), lo23 = __byte_perm(e2, e3, 0x5140);
    const uint32_t hi01 = __byte_perm(e0, e1, 0x7362), hi23 = __byte_perm(e2, e3, 0x7362);
    return make_uint4(__byte_perm(lo01, lo23, 0x5410), __byte_perm(lo01, lo23, 0x7632),
                      __byte_perm(hi01, hi23, 0x5410), __byte_perm(hi01, hi23, 0x7632));
}

__device__ __forceinline__ uint32_t bcast8(uint32_t w) { return 0x01010101u * (w & 0xFFu); }

// Byte i (0 <= i < 60) of what the validator reads for chunk c: the 32-byte
// header; end-table entries 4c-1 .. 4c+3 of a four-plane stream (modes 1, 2);
// entries c-1 and c of a one-plane stream (mode 0).  Entry -1 reads as 0 and
// bytes past `size` read as 0 (and fail validation).
__device__ __forceinline__ uint8_t header_byte(const uint8_t* src, uint64_t size, uint32_t nc,
                                               uint32_t c, int i)
{
    if (i < 32) return size >= 32 ? src[i] : 0;
    if (i < 52) {
        const int k = i - 32;
        const bool has_tab = nc > 0 && size >= 32ull + 16ull * nc;
        return (has_tab && !(c == 0 && k < 4)) ? src[32 + 16ull * c - 4 + k] : 0;
    }
    const int k = i - 52;
    const bool has_tab = nc > 0 && size >= 32ull + 4ull * nc;
    return (has_tab && !(c == 0 && k < 4)) ? src[32 + 4ull * c - 4 + k] : 0;
}

// Bytes of the end table: 16 per chunk for four-plane streams, 4 for mode 0.
__device__ __forceinline__ uint64_t table_bytes(int mode, uint32_t nc) { return (mode == 0 ? 4ull : 16ull) * nc; }

// Validate the header fields against the expected w x h and n_chunks, and
// chunk c's stream ends against the payload size and the all-literal bound.
// Four-plane streams (modes 1, 2) write beg[0..4], mode 0 (accepted only with
// allow0) beg[0..1]: stream offsets inside the payload.  Writes *mode.
// Returns nonzero for a malformed stream.
__device__ __forceinline__ int check_header(const uint8_t* h, uint64_t size, uint32_t w, uint32_t hgt,
                                            uint32_t nc, uint32_t c, uint32_t* beg, int* mode,
                                            bool allow0 = false)
{
    if (size < 32) return 1;
    int bad = 0;
    const uint32_t md = (uint32_t)h[6] | ((uint32_t)h[7] << 8);
    bad |= get_u32(h) != kMagic;
    bad |= (h[4] | (h[5] << 8)) != 1;
    bad |= md > 2u || (md == 0u && !allow0);
    bad |= get_u32(h + 8) != w || get_u32(h + 12) != hgt;
    bad |= get_u32(h + 16) != 4u || get_u32(h + 20) != (uint32_t)kChunk;
    bad |= get_u32(h + 24) != nc || get_u32(h + 28) != (md == 0u ? 1u : 4u);
    *mode = (int)md;
    const uint64_t tab = table_bytes((int)md, nc);
    if (!bad && nc > 0 && size < 32ull + tab) bad = 1;
    if (!bad && nc > 0) {
        const uint64_t psize = size - 32ull - tab;
        const uint32_t n = w * hgt;
        const uint32_t clen = min((uint32_t)kChunk, n - c * (uint32_t)kChunk);
        if (md == 0u) {
            const uint32_t u = clen / 2;
            const uint32_t cap = 8u * u + (u + 127u) / 128u + 4u * (clen & 1u);
            beg[0] = get_u32(h + 52);                       // 0 for chunk 0
            beg[1] = get_u32(h + 56);
            bad |= beg[1] < beg[0];
            bad |= beg[1] - beg[0] > cap;
            bad |= (uint64_t)beg[1] > psize;
        } else {
            const uint32_t cap = clen + (clen + 127u) / 128u;   // all-literal coding
            beg[0] = get_u32(h + 32);                           // 0 for chunk 0
            for (int p = 0; p < 4; ++p) {
                beg[p + 1] = get_u32(h + 36 + 4 * p);
                bad |= beg[p + 1] < beg[p];
                bad |= beg[p + 1] - beg[p] > cap;               // longer than any valid stream
            }
            bad |= (uint64_t)beg[4] > psize;
        }
    }
    return bad;
}

// One warp decodes the stream payload[beg, end) into plane[0, len).  Windows
// of 32 stream bytes, one per lane: lane l knows where a token starting at its
// byte would be followed by the next one; composing these jumps by doubling
// (5 levels) gives every lane t the start of the window's t-th token, so lanes
// hold tokens in order.  A warp scan places them; each lane writes the
// unaligned head and tail bytes of its own repeat token and its aligned body
// words when there are at most eight of them, the whole warp a longer body,
// one token per store; literal tokens are copied by the whole warp.  Where a
// window starts with repeat tokens no search is needed (each takes two
// bytes): lane l reads the pair at offset 2l and the leading repeats, up to
// 32, are placed with one scan.  Returns nonzero (the same on every lane) when a token runs
// past its stream or the chunk, or the stream does not yield exactly len bytes.
// plane must be 4-byte aligned.  src(i) returns stream byte i.
struct GlobalBytes {
    const uint8_t* __restrict__ p;
    __device__ __forceinline__ uint32_t operator()(int i) const { return (uint32_t)__ldg(p + i); }
};
struct SharedBytes {     // bytes [off, ...) of the payload staged at p
    const uint8_t* p;
    int off;
    __device__ __forceinline__ uint32_t operator()(int i) const { return (uint32_t)p[i - off]; }
};

// Each lane's repeat token (rep): olen copies of byte tv at plane[o, o+olen).
// The lane writes the unaligned head and tail bytes and a body of at most 8
// words itself; longer bodies are written by the whole warp, one per store.
__device__ __forceinline__ void write_repeats(uint8_t* plane, bool rep, int o, int olen, uint32_t tv, int lane)
{
    uint32_t* p32 = reinterpret_cast<uint32_t*>(plane);
    int head = 0, nw = 0;
    if (rep) {
        head = min(olen, (4 - (o & 3)) & 3);
        nw = (olen - head) >> 2;
        const int tail = olen - head - 4 * nw;
        for (int k = 0; k < head; ++k) plane[o + k] = (uint8_t)tv;
        for (int k = 0; k < tail; ++k) plane[o + head + 4 * nw + k] = (uint8_t)tv;
    }
    const uint32_t pk = (uint32_t)((o + head) >> 2) | ((uint32_t)nw << 16);
    const uint32_t wv = 0x01010101u * (tv & 0xFFu);
    if (nw <= 8)
        for (int k = 0; k < nw; ++k) p32[((o + head) >> 2) + k] = wv;
    for (uint32_t m = __ballot_sync(0xffffffffu, nw > 8); m; m &= m - 1u) {
        const int t = __ffs(m) - 1;
        const uint32_t q = __shfl_sync(0xffffffffu, pk, t);
        const uint32_t x = __shfl_sync(0xffffffffu, wv, t);
        if ((uint32_t)lane < (q >> 16)) p32[(q & 0xFFFFu) + lane] = x;
    }
}

__device__ __forceinline__ int warp_incl_sum(int v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

template <class Src>
__device__ __forceinline__ int decode_plane(const Src& src, int beg, int end, int len, uint8_t* plane, int lane)
{
    int cur = beg, outp = 0;
    while (cur < end) {
        // Fast window: if the bytes at even offsets from cur are repeat
        // controls, each starts a token (a repeat takes exactly two bytes), so
        // lane l holds token l without searching; take the leading run of them.
        {
            const int i2 = cur + 2 * lane;
            const uint32_t c = i2 + 1 < end ? src(i2) : 0u;
            const uint32_t v = i2 + 1 < end ? src(i2 + 1) : 0u;
            const uint32_t lit = __ballot_sync(0xffffffffu, c < 128u);
            const int m = lit ? __ffs(lit) - 1 : 32;
            if (m > 0) {
                const bool valid = lane < m;
                const int olen = valid ? (int)c - 127 : 0;
                const int incl = warp_incl_sum(olen, lane);
                const int total = __shfl_sync(0xffffffffu, incl, 31);
                const int o = outp + incl - olen;
                if (__any_sync(0xffffffffu, valid && o + olen > len)) return 1;
                write_repeats(plane, valid, o, olen, v, lane);
                outp += total;
                cur += 2 * m;
                continue;
            }
        }
        const int i = cur + lane;
        const uint32_t b = i < end ? src(i) : 0u;
        const uint32_t b1 = i + 1 < end ? src(i + 1) : 0u;
        int J = lane + (b >= 128u ? 2 : 2 + (int)b);   // next^(2^k), relative to cur
        int pos = 0;                                   // start of token #lane
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const int y = __shfl_sync(0xffffffffu, J, min(pos, 31));
            if (((lane >> k) & 1) && pos < 32) pos = y;
            if (k < 4) {
                const int z = __shfl_sync(0xffffffffu, J, min(J, 31));
                if (J < 32) J = z;
            }
        }
        // tokens take >= 2 bytes: at most 16 start in the window, and the
        // position after the last one (lane ntok) is exact
        const bool valid = pos < min(32, end - cur);
        const int ntok = __popc(__ballot_sync(0xffffffffu, valid));
        const int sl = __shfl_sync(0xffffffffu, pos, ntok);
        const int ps = min(pos, 31);
        const uint32_t tb = __shfl_sync(0xffffffffu, b, ps);
        const uint32_t tv = __shfl_sync(0xffffffffu, b1, ps);
        const bool trep = tb >= 128u;
        const int olen = valid ? (trep ? (int)tb - 127 : (int)tb + 1) : 0;
        const int tnext = pos + (trep ? 2 : 2 + (int)tb);
        const int incl = warp_incl_sum(olen, lane);
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        const int o = outp + incl - olen;
        if (__any_sync(0xffffffffu, valid && (cur + tnext > end || o + olen > len))) return 1;
        write_repeats(plane, valid && trep, o, olen, tv, lane);
        for (uint32_t m = __ballot_sync(0xffffffffu, valid && !trep); m; m &= m - 1u) {
            const int t = __ffs(m) - 1;
            const int oo = __shfl_sync(0xffffffffu, o, t);
            const int ml = __shfl_sync(0xffffffffu, olen, t);
            const int s0 = cur + __shfl_sync(0xffffffffu, pos, t) + 1;   // after the control
            for (int k = lane; k < ml; k += 32) plane[oo + k] = (uint8_t)src(s0 + k);
        }
        outp += total;
        cur += sl;
    }
    return outp != len;
}

// decode_plane's token walk (and validation), recording runs instead of bytes:
// every repeat token and every literal byte starts a run, in position order.
// Run r starting at position o sets bit o of the plane's bitmap bm (zero on
// entry; 128 words) and stores its byte in val[r].  Returns 0 with *nruns set,
// 1 for a malformed stream (as decode_plane), 2 once there would be more than
// cap runs (nothing about the stream's validity is then known).
template <class Src>
__device__ __forceinline__ int decode_plane_runs(const Src& src, int beg, int end, int len, uint32_t* bm,
                                                 uint8_t* val, int cap, int* nruns, int lane)
{
    int cur = beg, outp = 0, runs = 0;
    while (cur < end) {
        {
            const int i2 = cur + 2 * lane;
            const uint32_t c = i2 + 1 < end ? src(i2) : 0u;
            const uint32_t v = i2 + 1 < end ? src(i2 + 1) : 0u;
            const uint32_t lit = __ballot_sync(0xffffffffu, c < 128u);
            const int m = lit ? __ffs(lit) - 1 : 32;
            if (m > 0) {
                const bool valid = lane < m;
                const int olen = valid ? (int)c - 127 : 0;
                const int incl = warp_incl_sum(olen, lane);
                const int total = __shfl_sync(0xffffffffu, incl, 31);
                const int o = outp + incl - olen;
                if (__any_sync(0xffffffffu, valid && o + olen > len)) return 1;
                if (runs + m > cap) return 2;
                if (valid) {
                    atomicOr(bm + (o >> 5), 1u << (o & 31));
                    val[runs + lane] = (uint8_t)v;
                }
                runs += m;
                outp += total;
                cur += 2 * m;
                continue;
            }
        }
        const int i = cur + lane;
        const uint32_t b = i < end ? src(i) : 0u;
        const uint32_t b1 = i + 1 < end ? src(i + 1) : 0u;
        int J = lane + (b >= 128u ? 2 : 2 + (int)b);   // next^(2^k), relative to cur
        int pos = 0;                                   // start of token #lane
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const int y = __shfl_sync(0xffffffffu, J, min(pos, 31));
            if (((lane >> k) & 1) && pos < 32) pos = y;
            if (k < 4) {
                const int z = __shfl_sync(0xffffffffu, J, min(J, 31));
                if (J < 32) J = z;
            }
        }
        const bool valid = pos < min(32, end - cur);
        const int ntok = __popc(__ballot_sync(0xffffffffu, valid));
        const int sl = __shfl_sync(0xffffffffu, pos, ntok);
        const int ps = min(pos, 31);
        const uint32_t tb = __shfl_sync(0xffffffffu, b, ps);
        const uint32_t tv = __shfl_sync(0xffffffffu, b1, ps);
        const bool trep = tb >= 128u;
        const int olen = valid ? (trep ? (int)tb - 127 : (int)tb + 1) : 0;
        const int tnext = pos + (trep ? 2 : 2 + (int)tb);
        const int incl = warp_incl_sum(olen, lane);
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        const int o = outp + incl - olen;
        if (__any_sync(0xffffffffu, valid && (cur + tnext > end || o + olen > len))) return 1;
        const int nr = valid ? (trep ? 1 : olen) : 0;      // runs this token starts
        const int rinc = warp_incl_sum(nr, lane);
        const int rtot = __shfl_sync(0xffffffffu, rinc, 31);
        if (runs + rtot > cap) return 2;
        const int rb = runs + rinc - nr;
        if (valid && trep) {
            atomicOr(bm + (o >> 5), 1u << (o & 31));
            val[rb] = (uint8_t)tv;
        }
        for (uint32_t m = __ballot_sync(0xffffffffu, valid && !trep); m; m &= m - 1u) {
            const int t = __ffs(m) - 1;
            const int oo = __shfl_sync(0xffffffffu, o, t);
            const int ml = __shfl_sync(0xffffffffu, olen, t);
            const int r0 = __shfl_sync(0xffffffffu, rb, t);
            const int s0 = cur + __shfl_sync(0xffffffffu, pos, t) + 1;   // after the control
            for (int k = lane; k < ml; k += 32) {
                atomicOr(bm + ((oo + k) >> 5), 1u << ((oo + k) & 31));
                val[r0 + k] = (uint8_t)src(s0 + k);
            }
        }
        runs += rtot;
        outp += total;
        cur += sl;
    }
    *nruns = runs;
    return outp != len;
}

}  // namespace rlec
}  // namespace ec
