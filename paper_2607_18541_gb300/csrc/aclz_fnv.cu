// Chunked FNV-1a 64 of a device buffer (verification hash; the paper
// checks every GPU result by FNV, abstract and Sec. II).  Each 64 KiB chunk
// is hashed by one thread (FNV-1a is a serial chain); the chunk hashes are
// then hashed in order, 8 little-endian bytes each, followed by the length.
#include <mutex>

#include "aclz_device.cuh"
#include "aclz_internal.h"

using namespace aclz;

namespace {

constexpr uint64_t kBasis = 14695981039346656037ULL;
constexpr uint64_t kPrime = 1099511628211ULL;
constexpr uint64_t kChunk = 65536;

__device__ __forceinline__ uint64_t fnv_word(uint64_t h, uint32_t w) {
#pragma unroll
    for (int k = 0; k < 4; k++) {
        h ^= (w >> (8 * k)) & 0xffu;
        h *= kPrime;
    }
    return h;
}

__global__ void __launch_bounds__(128) k_fnv_chunks(const uint8_t *__restrict__ buf, uint64_t n,
                                                    uint64_t *__restrict__ hashes, uint64_t nchunks) {
    const uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (c >= nchunks) return;
    const uint64_t lo = c * kChunk;
    const uint64_t hi = lo + kChunk < n ? lo + kChunk : n;
    uint64_t h = kBasis;
    uint64_t p = lo;
    // buf is 16-byte aligned and lo is a multiple of 64 KiB
    for (; p + 64 <= hi; p += 64) {
        const uint4 *q = reinterpret_cast<const uint4 *>(buf + p);
        uint4 v[4];
#pragma unroll
        for (int k = 0; k < 4; k++) v[k] = __ldg(q + k);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            h = fnv_word(h, v[k].x);
            h = fnv_word(h, v[k].y);
            h = fnv_word(h, v[k].z);
            h = fnv_word(h, v[k].w);
        }
    }
    for (; p < hi; p++) {
        h ^= buf[p];
        h *= kPrime;
    }
    hashes[c] = h;
}

__global__ void k_fnv_combine(const uint64_t *__restrict__ hashes, uint64_t nchunks, uint64_t n,
                              uint64_t *out) {
    uint64_t h = kBasis;
    for (uint64_t c = 0; c < nchunks; c++) {
        const uint64_t v = hashes[c];
        h = fnv_word(h, (uint32_t)v);
        h = fnv_word(h, (uint32_t)(v >> 32));
    }
    h = fnv_word(h, (uint32_t)n);
    h = fnv_word(h, (uint32_t)(n >> 32));
    *out = h;
}

}  // namespace

namespace aclz {

// Enqueue the two FNV kernels with caller-provided scratch of
// 8 * (nchunks + 1) bytes; the result lands in scratch[nchunks].
int fnv_enqueue(const uint8_t *d_buf, uint64_t n, uint64_t *scratch, cudaStream_t st) {
    const uint64_t nchunks = (n + kChunk - 1) / kChunk;
    if (nchunks) {
        const unsigned grid = (unsigned)((nchunks + 127) / 128);
        k_fnv_chunks<<<grid, 128, 0, st>>>(d_buf, n, scratch, nchunks);
    }
    k_fnv_combine<<<1, 1, 0, st>>>(scratch, nchunks, n, scratch + nchunks);
    return cudaGetLastError() == cudaSuccess ? ACLZ_OK : ACLZ_E_CUDA;
}

}  // namespace aclz

extern "C" int aclz_fnv(const void *d_buf, uint64_t n, uint64_t *out_hash, void *stream) {
    if (!out_hash || (n && !d_buf)) return ACLZ_E_INVAL;
    if (reinterpret_cast<uintptr_t>(d_buf) & 15) return ACLZ_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t nchunks = (n + kChunk - 1) / kChunk;
    uint64_t *scratch = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&scratch, 8 * (nchunks + 1), st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? ACLZ_E_NOMEM : ACLZ_E_CUDA;
    int rc = fnv_enqueue((const uint8_t *)d_buf, n, scratch, st);
    uint64_t hv = 0;
    if (rc == ACLZ_OK &&
        cudaMemcpyAsync(&hv, scratch + nchunks, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = ACLZ_E_CUDA;
    cudaFreeAsync(scratch, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = ACLZ_E_CUDA;
    if (rc == ACLZ_OK) *out_hash = hv;
    return rc;
}

// ---------------------------------------------------------------------
// Allocation-free variant of aclz_fnv.
//
// Some callers cannot allocate device memory at the moment they want a
// verification hash: code that runs while the device is nearly full and a
// failed allocation would abort a long pipeline, code whose device memory
// is owned by an arena or pool manager that forbids out-of-band
// allocations, and latency-critical paths that must not enter the CUDA
// allocator (which may synchronize or block).  For them the chunk hashes
// live in one fixed array in the library's device memory instead of
// stream-ordered scratch.
//
// kNoAllocChunks bounds the input: 65536 chunks of 64 KiB, i.e. 4 GiB.  The
// array (512 KiB + 8 bytes) is held on every device that loads the library
// until the process exits.  All calls share it and it keeps the previous
// call's contents; nothing in it needs to start at zero, because every
// call rewrites every entry it reads.  Calls whose work overlaps on the GPU
// (different streams, or different host threads, without ordering between
// them) race on the array and can return wrong hashes.
constexpr uint64_t kNoAllocChunks = 65536;
static __device__ __align__(256) uint64_t g_fnv_noalloc_scratch[kNoAllocChunks + 1];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
uint64_t *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the fixed array on the current device, looked up once
// per device (the host-side symbol is only a stand-in, never a device
// address).
int noalloc_scratch(uint64_t **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ACLZ_E_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return ACLZ_E_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_fnv_noalloc_scratch);
        if (e != cudaSuccess || !p) return ACLZ_E_CUDA;
        g_noalloc_ptr[dev] = (uint64_t *)p;
    }
    *out = g_noalloc_ptr[dev];
    return ACLZ_OK;
}

}  // namespace

extern "C" int aclz_fnv_noalloc(const void *d_buf, uint64_t n, uint64_t *out_hash, void *stream) {
    if (!out_hash || (n && !d_buf)) return ACLZ_E_INVAL;
    if (reinterpret_cast<uintptr_t>(d_buf) & 15) return ACLZ_E_INVAL;
    const uint64_t nchunks = (n + kChunk - 1) / kChunk;
    if (nchunks > kNoAllocChunks) return ACLZ_E_CAPACITY;
    uint64_t *scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    rc = fnv_enqueue((const uint8_t *)d_buf, n, scratch, st);
    uint64_t hv = 0;
    if (rc == ACLZ_OK &&
        cudaMemcpyAsync(&hv, scratch + nchunks, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = ACLZ_E_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = ACLZ_E_CUDA;
    if (rc == ACLZ_OK) *out_hash = hv;
    return rc;
}
