// efm_noalloc.cu -- sorting supports into the library's output order
// without allocating any memory.
//
// Who needs this: code that may not call cudaMalloc (or any allocator) at
// the point where it orders pathway supports -- code running under a fixed
// device-memory budget whose allocator belongs to another framework (which
// would not see, and could not account for, a private cudaMalloc), or a
// loop that must never block on an allocator's synchronisation.  Such
// callers pass device buffers they already own for the input and the
// output; the only other memory the sort needs, its index array, lives in a
// file-scope device array reserved when the library is loaded.
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
//  - the first call on a device (and the first after that device's context
//    changed, e.g. after cudaDeviceReset) looks up the array's device
//    address in the current context (no allocation); make that first call
//    before any stream capture begins.
#include <mutex>

#include "efm_internal.cuh"

namespace {

constexpr int64_t kNoallocMaxRows = (int64_t)1 << 20;
constexpr int kMaxDevices = 64;

// index scratch of the bitonic sort (one entry per padded row)
static __device__ __align__(256) uint32_t g_sort_scratch[kNoallocMaxRows];

std::mutex g_mu;
uint32_t *g_scratch_ptr[kMaxDevices] = {};
void *g_scratch_ctx[kMaxDevices] = {};  // the context each cached address belongs to

// The driver's current context (obtained through the runtime, so the
// library needs no link against the driver library); nullptr if unknown.
void *current_context()
{
    using get_fn = int (*)(void **);
    static get_fn fn = nullptr;
    static bool looked = false;
    if (!looked) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (get_fn)p;
        else
            cudaGetLastError();
        looked = true;
    }
    void *ctx = nullptr;
    if (fn && fn(&ctx) != 0) ctx = nullptr;
    return ctx;
}

// Device address of g_sort_scratch in the current device's current context,
// looked up once per device and again whenever that context changes.  Host
// code must not use the symbol's name as an address: on the host it names a
// stand-in object.
cudaError_t scratch_ptr(uint32_t **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    void *ctx = current_context();
    if (!g_scratch_ptr[dev] || ctx == nullptr || ctx != g_scratch_ctx[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (uint32_t *)p;
        g_scratch_ctx[dev] = current_context();  // the lookup may have created the primary context
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
    if (!supports_in || !supports_out) return EFM_EINVAL;
    // the gather reads rows of the input while it writes the output: the two
    // byte ranges must not overlap at all
    const uintptr_t bytes = (uintptr_t)n_rows * (uintptr_t)words_per_set * 8u;
    const uintptr_t a = (uintptr_t)supports_in, b = (uintptr_t)supports_out;
    if (a < b + bytes && b < a + bytes) return EFM_EINVAL;
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
