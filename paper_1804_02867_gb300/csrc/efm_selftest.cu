// efm_selftest.cu -- the failure path of a bounded device-side wait, on demand.
//
// Every wait of the library's kernels (for a hash slot another warp has
// claimed but not yet published, for a bulk copy's mbarrier) polls a bounded
// number of times; when the bound is reached the kernel sets ERR_TIMEOUT in
// its error word and returns, and the host reports EFM_ETIMEOUT.  This
// kernel runs that path deliberately: one thread waits on a device flag that
// nothing sets, gives up after kWaitSpinLimit polls and flags the timeout.
// The GPU stays usable; nothing faults or hangs.
#include "efm_internal.cuh"

namespace efm {

namespace {

__global__ void stalled_wait_kernel(const uint32_t *flag, int spin_limit, unsigned long long *err,
                                    unsigned long long *polls)
{
    uint32_t v = 0;
    int n = 0;
    while (n < spin_limit) {
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
        ++n;
        if (v) break;
        __nanosleep(256);
    }
    if (!v) atomicOr(err, (unsigned long long)ERR_TIMEOUT);
    *polls = (unsigned long long)n;
}

}  // namespace

cudaError_t launch_stalled_wait(const uint32_t *flag, unsigned long long *err, unsigned long long *polls,
                                cudaStream_t s)
{
    stalled_wait_kernel<<<1, 1, 0, s>>>(flag, kWaitSpinLimit, err, polls);
    return cudaGetLastError();
}

}  // namespace efm
