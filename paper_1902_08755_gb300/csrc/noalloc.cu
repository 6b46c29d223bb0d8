// noalloc.cu -- ec_rle_compress_noalloc: the run-length compressor for callers
// that cannot allocate device memory.
//
// ec_rle_compress needs scratch memory (a record per 4096-element chunk, a pool
// that holds the coded chunks until they are placed, and two counters) that an
// ec_ctx allocates with cudaMalloc.  Some
// callers cannot do that: code that must not allocate once it is running (a
// render loop that reserved all of its memory at start-up, or code whose
// device memory belongs to another framework's pool), and code that cannot
// afford the implicit device synchronisation cudaMalloc/cudaFree may cause.
// This entry point takes its scratch from a fixed array compiled into the
// library instead, so it allocates nothing; the caller passes inputs and
// outputs as usual.
//
// The array is a file-scope __device__ variable: every GPU that loads libec
// holds one copy of it (EC_RLE_NOALLOC_SCRATCH_BYTES) until the process exits.
// Host code cannot use the array's name as a device address, so the first
// call on each device looks the address up with cudaGetSymbolAddress (with
// that device current) and caches it.
#include <string.h>

#include <mutex>

#include "ec_internal.cuh"

namespace {

constexpr size_t kScratchBytes = 16 + (16 + 4 + ec::kRlePoolPerUnit) * EC_RLE_NOALLOC_MAX_CHUNKS;
static_assert(kScratchBytes == EC_RLE_NOALLOC_SCRATCH_BYTES, "documented scratch size");

// Counters, chunk records and pool shared by every call of the entry point.
static __device__ __align__(256) unsigned char g_rle_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of this device's copy of g_rle_scratch (looked up once).
ec_status scratch_for_device(int dev, void** out)
{
    if (dev < 0 || dev >= kMaxDevices) return EC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_lock);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_rle_scratch) != cudaSuccess || !p) return EC_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return EC_OK;
}

}  // namespace

extern "C" ec_status ec_rle_compress_noalloc(const void* src, int32_t w, int32_t h, int32_t pitch,
                                             uint32_t mode, void* dst, size_t dst_capacity,
                                             uint64_t* d_size, uint32_t* d_status, ec_stream_t s)
{
    if (w < 0 || h < 0 || pitch < w || mode > 2) return EC_ERR_INVALID_ARG;
    const uint64_t n = (uint64_t)w * (uint64_t)h;
    if (n > EC_RLE_MAX_ELEMS) return EC_ERR_UNSUPPORTED;
    const uint64_t nchunks = (n + EC_RLE_CHUNK - 1) / EC_RLE_CHUNK;
    if (nchunks > EC_RLE_NOALLOC_MAX_CHUNKS) return EC_ERR_UNSUPPORTED;   // beyond the fixed scratch
    if (!dst || !d_size || !d_status || (n > 0 && !src)) return EC_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(d_size) & 7u) || (reinterpret_cast<uintptr_t>(d_status) & 3u))
        return EC_ERR_INVALID_ARG;
    if (n > 0 && (reinterpret_cast<uintptr_t>(src) & 3u)) return EC_ERR_INVALID_ARG;
    if (dst_capacity < ec_rle_max_size(w, h)) return EC_ERR_CAPACITY;

    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return EC_ERR_CUDA;
    void* scratch = nullptr;
    const ec_status st = scratch_for_device(dev, &scratch);
    if (st != EC_OK) return st;

    ec::RleJobDesc d;
    memset(&d, 0, sizeof(d));
    d.src = reinterpret_cast<const uint32_t*>(src);
    d.dst = dst;
    d.d_size = d_size;
    d.w = w;
    d.h = h;
    d.pitch = pitch;
    d.mode = mode;
    d.n_chunks = (uint32_t)nchunks;
    d.first_unit = 0;
    d.vec = (reinterpret_cast<uintptr_t>(src) & 15u) == 0 &&
            ((w % 4 == 0 && pitch % 4 == 0) || (pitch == w && ((uint64_t)w * (uint64_t)h) % 4 == 0));
    const uint32_t units = nchunks > 0 ? (uint32_t)nchunks : 1u;
    // the launcher clears the counters this call uses (a memset, no
    // allocation) before the kernels run
    return ec::launch_rle_compress(&d, 1, units, scratch, kScratchBytes, d_status, (cudaStream_t)s) == cudaSuccess
               ? EC_OK : EC_ERR_CUDA;
}
