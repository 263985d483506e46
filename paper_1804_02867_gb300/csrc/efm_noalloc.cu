// efm_noalloc.cu -- sorting supports into the library's output order
// without allocating any memory.
//
// Who needs this: code that may not call cudaMalloc (or any allocator) at
// the point where it orders pathway supports -- for example work recorded
// while a stream is being captured into a CUDA graph (allocation calls are
// not allowed there), code running under a fixed device-memory budget whose
// allocator belongs to another framework, or a loop that must never block on
// the allocator.  Such callers pass device buffers they already own for the
// input and the output; the only other memory the sort needs, its index
// array, lives in a file-scope device array reserved when the library is
// loaded.
//
// Limits and sharing:
//  - at most EFM_NOALLOC_MAX_ROWS rows (the index array holds the row count
//    rounded up to a power of two, 2^20 entries = 4 MiB of device memory,
//    held by every GPU that loads this library until the process exits);
//  - every call uses the same array and leaves its contents behind; each
//    call rewrites every entry it reads before reading it, so nothing needs
//    clearing, but two calls whose work overlaps on the GPU (different
//    streams, no ordering between them) race on the array and may return
//    wrong orders.
//  - the first call on a device looks up the array's device address (no
//    allocation); make that first call before any stream capture begins.
#include <mutex>

#include "efm_internal.cuh"

namespace {

constexpr int64_t kNoallocMaxRows = (int64_t)1 << 20;
constexpr int kMaxDevices = 64;

// index scratch of the bitonic sort (one entry per padded row)
static __device__ __align__(256) uint32_t g_sort_scratch[kNoallocMaxRows];

std::mutex g_mu;
uint32_t *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_sort_scratch on the current device (looked up once
// per device, with that device current).  Host code must not use the
// symbol's name as an address: on the host it names a stand-in object.
cudaError_t scratch_ptr(uint32_t **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (uint32_t *)p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int efm_sort_supports_noalloc(const uint64_t *supports_in, int64_t n_rows, int32_t words_per_set,
                                         uint64_t *supports_out, uintptr_t cuda_stream)
{
    if (n_rows < 0 || words_per_set < 1 || words_per_set > efm::kMaxW) return EFM_EINVAL;
    if (n_rows > kNoallocMaxRows) return EFM_ECAPACITY;
    if (n_rows == 0) return EFM_OK;
    if (!supports_in || !supports_out || supports_in == supports_out) return EFM_EINVAL;
    uint32_t *scratch = nullptr;
    if (scratch_ptr(&scratch) != cudaSuccess) {
        cudaGetLastError();
        return EFM_ECUDA;
    }
    uint64_t n2 = 1;
    while ((int64_t)n2 < n_rows) n2 <<= 1;
    const cudaError_t e = efm::launch_sort_results(supports_in, n_rows, words_per_set, scratch, (int64_t)n2,
                                                   supports_out, n_rows, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return EFM_ECUDA;
    }
    return EFM_OK;
}
