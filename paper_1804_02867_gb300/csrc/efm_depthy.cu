// efm_depthy.cu -- flux-dependent reactions (Def. 11): the DEPTHy pre-pass
// of the paper's architecture (Alg. 2).
//
// A step from internal metabolite m goes through a column k consuming m to
// an internal metabolite that k produces; the steps out of m are ordered by
// (column, product row), and r is the largest number of steps out of any
// internal metabolite.  As in Alg. 2, one CTA takes one metabolite i and
// each thread j < r^L reads its L base-r digits (lowest first) as the step
// choices of one walk from i.  A walk ends when a digit exceeds the steps
// available (no such walk) or when it comes back to i: then its leaving
// column and its returning column are tagged as flux-dependent for i.
#include "efm_internal.cuh"

namespace efm {

namespace {

// the d-th step out of m: (column, product row), or column -1
__device__ __forceinline__ int2 step_of(const NetView &nv, int m, int d)
{
    const uint32_t *bl = nv.blob;
    int cnt = 0;
    for (int q = (int)bl[nv.o_consptr + m]; q < (int)bl[nv.o_consptr + m + 1]; ++q) {
        const int c = ent_index(bl[nv.o_consent + q]);
        for (int p = (int)bl[nv.o_colptr + c]; p < (int)bl[nv.o_colptr + c + 1]; ++p) {
            const uint32_t e = bl[nv.o_colent + p];
            if (ent_coef(e) > 0) {
                if (cnt == d) return make_int2(c, ent_index(e));
                ++cnt;
            }
        }
    }
    return make_int2(-1, -1);
}

__global__ void step_count_kernel(NetView nv, unsigned *r)
{
    const uint32_t *bl = nv.blob;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < nv.M; m += gridDim.x * blockDim.x) {
        unsigned cnt = 0;
        for (int q = (int)bl[nv.o_consptr + m]; q < (int)bl[nv.o_consptr + m + 1]; ++q) {
            const int c = ent_index(bl[nv.o_consent + q]);
            for (int p = (int)bl[nv.o_colptr + c]; p < (int)bl[nv.o_colptr + c + 1]; ++p)
                cnt += ent_coef(bl[nv.o_colent + p]) > 0 ? 1u : 0u;
        }
        atomicMax(r, cnt);
    }
}

__global__ void depthy_kernel(NetView nv, int L, unsigned r, unsigned long long n_paths, unsigned long long *dep_out,
                              unsigned long long *dep_in)
{
    const int W = nv.W;
    for (int i = blockIdx.x; i < nv.M; i += gridDim.x) {
        for (unsigned long long j = threadIdx.x; j < n_paths; j += blockDim.x) {
            unsigned long long code = j;
            int m = i, first = -1;
            for (int l = 0; l < L; ++l) {
                const int d = (int)(code % r);
                code /= r;
                const int2 st = step_of(nv, m, d);
                if (st.x < 0) break;  // no such walk
                if (first < 0) first = st.x;
                if (st.y == i) {
                    atomicOr(&dep_out[(size_t)i * W + (first >> 6)], 1ull << (first & 63));
                    atomicOr(&dep_in[(size_t)i * W + (st.x >> 6)], 1ull << (st.x & 63));
                    break;
                }
                m = st.y;
            }
        }
    }
}

__global__ void or_words_kernel(uint64_t *a, const uint64_t *b, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] |= b[i];
}

}  // namespace

cudaError_t launch_or_words(uint64_t *a, const uint64_t *b, int64_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    or_words_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, b, n);
    return cudaGetLastError();
}

cudaError_t launch_step_count(const NetView &nv, unsigned *r, cudaStream_t s)
{
    step_count_kernel<<<(nv.M + 255) / 256 > 0 ? (nv.M + 255) / 256 : 1, 256, 0, s>>>(nv, r);
    return cudaGetLastError();
}

cudaError_t launch_depthy(const NetView &nv, int L, unsigned r, unsigned long long n_paths, unsigned long long *dep_out,
                          unsigned long long *dep_in, int sm_count, cudaStream_t s)
{
    if (nv.M <= 0 || n_paths == 0) return cudaSuccess;
    const int grid = std::min(nv.M, sm_count * 8);
    depthy_kernel<<<grid, 256, 0, s>>>(nv, L, r, n_paths, dep_out, dep_in);
    return cudaGetLastError();
}

}  // namespace efm
