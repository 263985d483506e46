// efm_mlp.cu -- the learned proposal of a first-K search: features of
// pathway states, and a two-layer MLP (128 -> 256 ReLU -> 1) with BF16
// weights and FP32 accumulation on the tensor cores (tcgen05, accumulators in
// tensor memory), with its own forward, backward and optimizer kernels.
//
// The proposal only orders the parents of a level; the branch and bound of
// the search is exact, so the results never depend on it.
#include <cuda_bf16.h>

#include "efm_internal.cuh"

namespace efm {

namespace {

constexpr unsigned FULLMASK = 0xFFFFFFFFu;
constexpr int kF = kMlpFeatures;
constexpr int kH = kMlpHidden;
constexpr int kTR = kMlpTileRows;
constexpr uint32_t kXTileBytes = kTR * kF * 2;  // 32 KB
constexpr uint32_t kWBytes = kH * kF * 2;       // 64 KB
constexpr int kMlpThreads = 128;                // 4 warps: one per 32 lanes of tensor memory
constexpr int kWaitLimit = 1 << 22;             // bounded mbarrier waits (x ~0.25 us)

__device__ __forceinline__ uint32_t sm_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t *b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sm_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ bool bar_wait(uint64_t *b, uint32_t parity)
{
    uint32_t done = 0;
    for (int i = 0; i < kWaitLimit && !done; ++i) {
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(done)
                     : "r"(sm_u32(b)), "r"(parity)
                     : "memory");
        if (!done) __nanosleep(64);
    }
    return done != 0;
}

// one thread: expect `bytes` on the barrier, then copy them in 32 KB pieces
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *b)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sm_u32(b)), "r"(bytes) : "memory");
    for (uint32_t off = 0; off < bytes; off += 32768u) {
        const uint32_t n = bytes - off < 32768u ? bytes - off : 32768u;
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         sm_u32((char *)dst + off)),
                     "l"((const char *)src + off), "r"(n), "r"(sm_u32(b))
                     : "memory");
    }
}

__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: start, leading (K-direction) and stride
// (row-group) byte offsets, descriptor version 1, no swizzling.
__device__ __forceinline__ uint64_t sdesc(const void *p, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((sm_u32(p) & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;
    return d;
}

// Instruction descriptor of kind::f16: D F32, A and B BF16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dt, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(dt),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *b)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sm_u32(b))
                 : "memory");
}

// 32 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t tmem_alloc_warp(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sm_u32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    return 0;
}

__device__ __forceinline__ void tmem_free_warp(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Sum over the 32 lanes of v[i] for every i; lane l ends with the sum for
// i = l (recursive halving: each step sends half of the remaining values).
__device__ __forceinline__ float lane_transpose_sum(float (&v)[32], int lane)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < off; ++i) {
            const float send = upper ? v[i] : v[i + off];
            const float keep = upper ? v[i + off] : v[i];
            v[i] = keep + __shfl_xor_sync(FULLMASK, send, off);
        }
    }
    return v[0];
}

__device__ __forceinline__ uint32_t col_hash(uint32_t k)
{
    uint32_t h = k * 0x9E3779B1u;
    h ^= h >> 15;
    h *= 0x85EBCA77u;
    h ^= h >> 13;
    return h;
}

// ---------------------------------------------------------------------------
// Features of a pathway state (one warp per state), written as BF16 into
// row-tiles in the tensor-core operand layout:
//   0 unbalanced internal metabolites / 64      1 static degree of the pivot / 64
//   2 |U| / max_len                             3 secondary steps / max_secondary
//   4-7 the four lowest columns of U / N        8 pivot row / M
//   9 log2(1 + max |b|) / 32                    10 constant 1 (the hidden bias)
//   11 level / (max_len + max_secondary)        12 mean column of U / N
//   13 share of U's columns flux-dependent for the pivot (Def. 11, the DEPTHy tags)
//   14 1 when the pivot has flux-dependent columns at all
//   64-127 hashed embedding of U: column k adds +-1 to bucket h(k) mod 64,
//          scaled by 1 / sqrt(|U|)
// Row r takes the state at position first + r * stride of the arena.
// ---------------------------------------------------------------------------
constexpr int kFeatWarps = 8;

__global__ void __launch_bounds__(kFeatWarps * 32) features_kernel(NetView nv, Arena par, const uint32_t *map,
                                                                   int64_t first, int64_t stride, int64_t n, int level,
                                                                   int max_len, int max_sec, const uint64_t *dep,
                                                                   __nv_bfloat16 *X, int64_t row0)
{
    __shared__ float emb[kFeatWarps][64];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int W = nv.W;
    for (int64_t r = (int64_t)blockIdx.x * kFeatWarps + wid; r < n; r += (int64_t)gridDim.x * kFeatWarps) {
        const int64_t pos = first + r * stride;
        const int64_t p = map ? (int64_t)map[pos] : pos;
        const uint64_t *U = par.U + (size_t)p * W;
        const int32_t *B = par.B + (size_t)p * nv.Mpad;
        const uint32_t meta = par.meta[p];
        int nz = 0;
        uint32_t amax = 0;
        for (int m = lane; m < nv.M; m += 32) {
            const int32_t v = B[m];
            nz += v != 0;
            const uint32_t av = (uint32_t)(v < 0 ? -v : v);
            amax = av > amax ? av : amax;
        }
        emb[wid][lane] = 0.f;
        emb[wid][lane + 32] = 0.f;
        __syncwarp();
        float colsum = 0.f;
        int pcl = 0;
        for (int w = lane; w < W; w += 32) {
            uint64_t x = U[w];
            pcl += __popcll(x);
            while (x) {
                const int b = __ffsll((long long)x) - 1;
                x &= x - 1;
                const uint32_t k = (uint32_t)(w * 64 + b);
                const uint32_t h = col_hash(k);
                atomicAdd(&emb[wid][h & 63u], (h & 64u) ? 1.f : -1.f);
                colsum += (float)k;
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            nz += __shfl_xor_sync(FULLMASK, nz, off);
            pcl += __shfl_xor_sync(FULLMASK, pcl, off);
            colsum += __shfl_xor_sync(FULLMASK, colsum, off);
            const uint32_t o = __shfl_xor_sync(FULLMASK, amax, off);
            amax = o > amax ? o : amax;
        }
        // the four lowest columns: lowest words first, one ballot per word
        float low[4] = {1.f, 1.f, 1.f, 1.f};
        int got = 0;
        for (int w0 = 0; w0 < W && got < 4; w0 += 32) {
            const uint64_t x = (w0 + lane < W) ? U[w0 + lane] : 0ull;
            unsigned nzm = __ballot_sync(FULLMASK, x != 0ull);
            while (nzm && got < 4) {
                const int src = __ffs((int)nzm) - 1;
                nzm &= nzm - 1;
                uint64_t y = __shfl_sync(FULLMASK, x, src);
                while (y && got < 4) {
                    const int b = __ffsll((long long)y) - 1;
                    y &= y - 1;
                    low[got++] = (float)((w0 + src) * 64 + b) / (float)nv.N;
                }
            }
        }
        __syncwarp();
        const int pc = (int)((meta >> 23) & 0x7Fu);
        const int piv = (int)(meta & 0x3FFu);
        // flux-dependent columns of the pivot (tags of dep_out | dep_in) inside U
        int ndep = 0, anydep = 0;
        if (dep && piv < nv.M) {
            const uint64_t *D = dep + (size_t)piv * W;
            for (int w = lane; w < W; w += 32) {
                ndep += __popcll(U[w] & D[w]);
                anydep |= D[w] != 0ull;
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                ndep += __shfl_xor_sync(FULLMASK, ndep, off);
                anydep |= __shfl_xor_sync(FULLMASK, anydep, off);
            }
        }
        const int deg = (int)((meta >> 10) & 0x1FFFu);
        const int sec = level - (pc - 1);
        const float inv_sqrt = pcl > 0 ? rsqrtf((float)pcl) : 0.f;
        float f[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int i = 4 * lane + t;
            float v = 0.f;
            if (i >= 64) {
                v = emb[wid][i - 64] * inv_sqrt;
            } else if (i == 0) {
                v = (float)nz / 64.f;
            } else if (i == 1) {
                v = (float)deg / 64.f;
            } else if (i == 2) {
                v = (float)pc / (float)max_len;
            } else if (i == 3) {
                v = (float)sec / (float)(max_sec > 0 ? max_sec : 1);
            } else if (i < 8) {
                v = low[i - 4];
            } else if (i == 8) {
                v = (float)piv / (float)(nv.M > 0 ? nv.M : 1);
            } else if (i == 9) {
                v = log2f(1.f + (float)amax) / 32.f;
            } else if (i == 10) {
                v = 1.f;
            } else if (i == 11) {
                v = (float)level / (float)(max_len + max_sec);
            } else if (i == 12) {
                v = pcl > 0 ? colsum / (float)pcl / (float)nv.N : 0.f;
            } else if (i == 13) {
                v = pcl > 0 ? (float)ndep / (float)pcl : 0.f;
            } else if (i == 14) {
                v = anydep ? 1.f : 0.f;
            }
            f[t] = v;
        }
        const int64_t row = row0 + r;
        char *tile = reinterpret_cast<char *>(X) + (size_t)(row / kTR) * kXTileBytes;
        __nv_bfloat162 *dst = reinterpret_cast<__nv_bfloat162 *>(tile + mlp_blk_off((int)(row % kTR), 4 * lane));
        dst[0] = __floats2bfloat162_rn(f[0], f[1]);
        dst[1] = __floats2bfloat162_rn(f[2], f[3]);
        __syncwarp();
    }
}

// Training label of a sampled state: 1 when its support lies inside one of
// the answer's supports (the state can still reach that answer).
__global__ void labels_kernel(const uint64_t *Uar, int W, const uint32_t *map, int64_t first, int64_t stride,
                              int64_t n, const uint64_t *ans, int64_t n_ans, float *y, int64_t row0)
{
    const int lane = threadIdx.x & 31;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t pos = first + r * stride;
        const uint64_t *U = Uar + (size_t)(map ? (int64_t)map[pos] : pos) * W;
        bool in = false;
        for (int64_t a = lane; a < n_ans && !in; a += 32) {
            const uint64_t *A = ans + (size_t)a * W;
            bool sub = true;
            for (int w = 0; w < W && sub; ++w) sub = (U[w] & ~A[w]) == 0;
            in = sub;
        }
        const bool any = __any_sync(FULLMASK, in);
        if (lane == 0) y[row0 + r] = any ? 1.f : 0.f;
    }
}

// ---------------------------------------------------------------------------
// Forward pass (scores): persistent CTAs, one 128-row tile at a time.
// Layer 1 is one M=128 N=256 K=128 product on the tensor cores into tensor
// memory; the epilogue (ReLU, layer 2, FP32) reads it back lane by lane.
// ---------------------------------------------------------------------------
struct ScoreSmem {
    static constexpr uint32_t W = 0;
    static constexpr uint32_t X = W + kWBytes;
    static constexpr uint32_t W2 = X + kXTileBytes;
    static constexpr uint32_t BAR = W2 + kH * 4;
    static constexpr uint32_t SLOT = BAR + 16;
    static constexpr uint32_t BYTES = SLOT + 16;
};

__global__ void __launch_bounds__(kMlpThreads, 1) mlp_score_kernel(const __nv_bfloat16 *X, int64_t n_rows,
                                                                   const __nv_bfloat16 *wb, const float *params,
                                                                   float *score, unsigned *err)
{
    extern __shared__ __align__(128) char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint64_t *bar_ld = reinterpret_cast<uint64_t *>(sm + ScoreSmem::BAR);
    uint64_t *bar_mma = bar_ld + 1;
    uint32_t *slot = reinterpret_cast<uint32_t *>(sm + ScoreSmem::SLOT);
    float *w2 = reinterpret_cast<float *>(sm + ScoreSmem::W2);
    const int64_t n_tiles = (n_rows + kTR - 1) / kTR;
    if (tid == 0) {
        bar_init(bar_ld, 1);
        bar_init(bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int j = tid; j < kH; j += kMlpThreads) w2[j] = params[kMlpW2 + j];
    const float b2 = params[kMlpB2];
    if (warp == 0) tmem_alloc_warp(slot, 256);
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tbase = *slot;
    if (tid == 0) bulk_load(sm + ScoreSmem::W, wb, kWBytes, bar_ld);
    uint32_t ph_ld = 0, ph_mma = 0;
    bool ok = bar_wait(bar_ld, ph_ld);
    ph_ld ^= 1;
    constexpr uint32_t idesc = idesc_bf16(128, kH);
    for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        if (tid == 0) bulk_load(sm + ScoreSmem::X, reinterpret_cast<const char *>(X) + (size_t)t * kXTileBytes,
                                kXTileBytes, bar_ld);
        ok = bar_wait(bar_ld, ph_ld);
        ph_ld ^= 1;
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        if (tid == 0) {
            tc_after();
#pragma unroll
            for (int ks = 0; ks < kF / 16; ++ks)
                mma_bf16(tbase, sdesc(sm + ScoreSmem::X + ks * 256, 128, 2048),
                         sdesc(sm + ScoreSmem::W + ks * 256, 128, 2048), idesc, ks > 0 ? 1u : 0u);
            mma_commit(bar_mma);
        }
        ok = bar_wait(bar_mma, ph_mma);
        ph_mma ^= 1;
        tc_after();
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        float s = b2;
#pragma unroll 1
        for (int c = 0; c < kH / 32; ++c) {
            float v[32];
            tmem_ld32(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * c), v);
#pragma unroll
            for (int i = 0; i < 32; ++i) s += fmaxf(v[i], 0.f) * w2[32 * c + i];
        }
        const int64_t row = t * kTR + 32 * warp + lane;
        if (row < n_rows) score[row] = s;
        tc_before();
        __syncthreads();
    }
    if (!ok && tid == 0) atomicOr(err, 1u);
    tc_before();
    __syncthreads();
    tc_after();
    if (warp == 0) tmem_free_warp(tbase, 256);
}

// ---------------------------------------------------------------------------
// Training pass over a list of tiles: forward as above, then per row
//   s = b2 + w2 . relu(h),  h = W1 x
//   loss = wt * (softplus(s) - y s) / n,   ds = wt * (sigmoid(s) - y) / n
//   dh_j = ds * w2_j * [h_j > 0]            (BF16, for the tensor cores)
//   dW1 += dH^T X  (M=128 features, N=256 hidden, K=128 rows, accumulated
//                  in tensor memory over all tiles of the CTA)
//   dw2 += ds * relu(h),  db2 += ds        (FP32, lane-transposed sums)
// wt = pos_weight for y = 1 rows, 1 for y = 0 rows, 0 for padding (y < 0
// or row >= n_rows).  Gradients are added into params-shaped FP32 buffers.
// ---------------------------------------------------------------------------
struct TrainSmem {
    static constexpr uint32_t W = 0;
    static constexpr uint32_t X = W + kWBytes;
    static constexpr uint32_t XT = X + kXTileBytes;
    static constexpr uint32_t DH = XT + kXTileBytes;
    static constexpr uint32_t W2 = DH + kWBytes;
    static constexpr uint32_t BAR = W2 + kH * 4;
    static constexpr uint32_t SLOT = BAR + 16;
    static constexpr uint32_t BYTES = SLOT + 16;
};

__global__ void __launch_bounds__(kMlpThreads, 1)
    mlp_train_kernel(const __nv_bfloat16 *X, const float *y, int64_t n_rows, const int32_t *tiles, int n_tiles,
                     const __nv_bfloat16 *wb, const float *params, float pos_weight, float inv_n, float *grad,
                     float *loss, unsigned *err)
{
    extern __shared__ __align__(128) char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint64_t *bar_ld = reinterpret_cast<uint64_t *>(sm + TrainSmem::BAR);
    uint64_t *bar_mma = bar_ld + 1;
    uint32_t *slot = reinterpret_cast<uint32_t *>(sm + TrainSmem::SLOT);
    float *w2 = reinterpret_cast<float *>(sm + TrainSmem::W2);
    if (tid == 0) {
        bar_init(bar_ld, 1);
        bar_init(bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int j = tid; j < kH; j += kMlpThreads) w2[j] = params[kMlpW2 + j];
    const float b2 = params[kMlpB2];
    if (warp == 0) tmem_alloc_warp(slot, 512);
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tbase = *slot;  // columns 0-255: layer 1; 256-511: dW1^T
    if (tid == 0) bulk_load(sm + TrainSmem::W, wb, kWBytes, bar_ld);
    uint32_t ph_ld = 0, ph_mma = 0;
    bool ok = bar_wait(bar_ld, ph_ld);
    ph_ld ^= 1;
    constexpr uint32_t idesc = idesc_bf16(128, kH);
    float gw2[kH / 32];
#pragma unroll
    for (int c = 0; c < kH / 32; ++c) gw2[c] = 0.f;
    float gb2 = 0.f, lsum = 0.f;
    int done = 0;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    for (int it = blockIdx.x; it < n_tiles && ok; it += gridDim.x) {
        const int64_t t = tiles[it];
        if (tid == 0) bulk_load(sm + TrainSmem::X, reinterpret_cast<const char *>(X) + (size_t)t * kXTileBytes,
                                kXTileBytes, bar_ld);
        ok = bar_wait(bar_ld, ph_ld);
        ph_ld ^= 1;
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        if (tid == 0) {
            tc_after();
#pragma unroll
            for (int ks = 0; ks < kF / 16; ++ks)
                mma_bf16(tbase, sdesc(sm + TrainSmem::X + ks * 256, 128, 2048),
                         sdesc(sm + TrainSmem::W + ks * 256, 128, 2048), idesc, ks > 0 ? 1u : 0u);
            mma_commit(bar_mma);
        }
        ok = bar_wait(bar_mma, ph_mma);
        ph_mma ^= 1;
        tc_after();
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        const int rl = 32 * warp + lane;  // row within the tile
        const int64_t row = t * kTR + rl;
        const float yr = row < n_rows ? y[row] : -1.f;
        const float wt = yr < 0.f ? 0.f : (yr > 0.5f ? pos_weight : 1.f);
        float s = b2;
#pragma unroll 1
        for (int c = 0; c < kH / 32; ++c) {
            float v[32];
            tmem_ld32(tbase + lane_base + (uint32_t)(32 * c), v);
#pragma unroll
            for (int i = 0; i < 32; ++i) s += fmaxf(v[i], 0.f) * w2[32 * c + i];
        }
        const float yy = yr > 0.5f ? 1.f : 0.f;
        const float sig = 1.f / (1.f + __expf(-s));
        const float ds = wt * (sig - yy) * inv_n;
        const float sp = s > 0.f ? s + log1pf(__expf(-s)) : log1pf(__expf(s));
        lsum += wt * (sp - yy * s) * inv_n;
        gb2 += ds;
        // dH (BF16, B operand of the backward product: rows = hidden unit,
        // K = row of the tile) and the layer-2 gradient
        char *dh = sm + TrainSmem::DH;
#pragma unroll 1
        for (int c = 0; c < kH / 32; ++c) {
            float v[32];
            tmem_ld32(tbase + lane_base + (uint32_t)(32 * c), v);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int j = 32 * c + i;
                const float d = v[i] > 0.f ? ds * w2[j] : 0.f;
                *reinterpret_cast<__nv_bfloat16 *>(dh + mlp_blk_off(j, rl)) = __float2bfloat16_rn(d);
                v[i] = ds * fmaxf(v[i], 0.f);
            }
            gw2[c] += lane_transpose_sum(v, lane);
        }
        // X^T (A operand of the backward product: rows = feature, K = row)
        {
            const char *xs = sm + TrainSmem::X;
            char *xt = sm + TrainSmem::XT;
#pragma unroll 1
            for (int q = 0; q < kF / 8; ++q) {
                const uint4 v = *reinterpret_cast<const uint4 *>(xs + mlp_blk_off(rl, 8 * q));
                const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const uint16_t hv = (uint16_t)(wv[e >> 1] >> (16 * (e & 1)));
                    *reinterpret_cast<uint16_t *>(xt + mlp_blk_off(8 * q + e, rl)) = hv;
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_before();
        __syncthreads();
        if (tid == 0) {
            tc_after();
#pragma unroll
            for (int ks = 0; ks < kTR / 16; ++ks)
                mma_bf16(tbase + 256, sdesc(sm + TrainSmem::XT + ks * 256, 128, 2048),
                         sdesc(sm + TrainSmem::DH + ks * 256, 128, 2048), idesc, (done > 0 || ks > 0) ? 1u : 0u);
            mma_commit(bar_mma);
        }
        ok = bar_wait(bar_mma, ph_mma);
        ph_mma ^= 1;
        tc_after();
        ok = __syncthreads_and(ok);
        ++done;
    }
    if (ok && done > 0) {
        // dW1[j][f] for f = this lane's feature, j over the 256 columns
        const int f = 32 * warp + lane;
#pragma unroll 1
        for (int c = 0; c < kH / 32; ++c) {
            float v[32];
            tmem_ld32(tbase + lane_base + 256u + (uint32_t)(32 * c), v);
#pragma unroll
            for (int i = 0; i < 32; ++i) atomicAdd(&grad[kMlpW1 + (32 * c + i) * kF + f], v[i]);
        }
#pragma unroll
        for (int c = 0; c < kH / 32; ++c) atomicAdd(&grad[kMlpW2 + 32 * c + lane], gw2[c]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            gb2 += __shfl_xor_sync(FULLMASK, gb2, off);
            lsum += __shfl_xor_sync(FULLMASK, lsum, off);
        }
        if (lane == 0) {
            atomicAdd(&grad[kMlpB2], gb2);
            atomicAdd(loss, lsum);
        }
    }
    if (!ok && tid == 0) atomicOr(err, 1u);
    tc_before();
    __syncthreads();
    tc_after();
    if (warp == 0) tmem_free_warp(tbase, 512);
}

// Adam step on the FP32 parameters; refreshes the BF16 operand copy of W1
// and clears the gradients.
__global__ void adam_kernel(float *params, float *grad, float *mom, float lr, float c1, float c2, __nv_bfloat16 *wb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    const float g = grad[i];
    float m = mom[i], v = mom[kMlpParams + i];
    m = 0.9f * m + 0.1f * g;
    v = 0.999f * v + 0.001f * g * g;
    mom[i] = m;
    mom[kMlpParams + i] = v;
    const float p = params[i] - lr * (m / c1) / (sqrtf(v / c2) + 1e-8f);
    params[i] = p;
    grad[i] = 0.f;
    if (i < kMlpW2) {
        const int j = i / kF, f = i % kF;
        *reinterpret_cast<__nv_bfloat16 *>(reinterpret_cast<char *>(wb) + mlp_blk_off(j, f)) = __float2bfloat16_rn(p);
    }
}

__global__ void pack_w_kernel(const float *params, __nv_bfloat16 *wb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kH * kF) return;
    const int j = i / kF, f = i % kF;
    *reinterpret_cast<__nv_bfloat16 *>(reinterpret_cast<char *>(wb) + mlp_blk_off(j, f)) =
        __float2bfloat16_rn(params[kMlpW1 + i]);
}

// Order by score, highest first: a counting sort over 4096 buckets of width
// 1/128 on [-16, 16) (the order inside a bucket is unspecified).
constexpr int kScoreBuckets = 4096;

__device__ __forceinline__ int score_bucket(float s)
{
    float x = (16.f - s) * 128.f;
    x = x < 0.f ? 0.f : (x > (float)(kScoreBuckets - 1) ? (float)(kScoreBuckets - 1) : x);
    return (int)x;
}

__global__ void score_hist_kernel(const float *score, int64_t n, unsigned *hist)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&hist[score_bucket(score[i])], 1u);
}

__global__ void score_scan_kernel(unsigned *hist)
{
    // one block of 1024 threads, 4 buckets each: exclusive prefix sum
    __shared__ unsigned part[1024];
    const int t = threadIdx.x;
    unsigned v[4], s = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        v[i] = hist[4 * t + i];
        s += v[i];
    }
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const unsigned x = t >= off ? part[t - off] : 0u;
        __syncthreads();
        part[t] += x;
        __syncthreads();
    }
    unsigned base = part[t] - s;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        hist[4 * t + i] = base;
        base += v[i];
    }
}

__global__ void score_scatter_kernel(const float *score, int64_t n, const uint32_t *map, unsigned *offs,
                                     uint32_t *perm)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned pos = atomicAdd(&offs[score_bucket(score[i])], 1u);
        perm[pos] = map ? map[i] : (uint32_t)i;
    }
}

// host FP32 rows (row-major, 128 features) -> BF16 operand tiles at row0
__global__ void pack_rows_kernel(const float *x, int64_t n, __nv_bfloat16 *X, int64_t row0)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * kF) return;
    const int64_t r = row0 + i / kF;
    const int f = (int)(i % kF);
    char *tile = reinterpret_cast<char *>(X) + (size_t)(r / kTR) * kXTileBytes;
    *reinterpret_cast<__nv_bfloat16 *>(tile + mlp_blk_off((int)(r % kTR), f)) = __float2bfloat16_rn(x[i]);
}

int sm_count_cached()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

}  // namespace

cudaError_t launch_features(const NetView &nv, const Arena &par, const uint32_t *map, int64_t first, int64_t stride,
                            int64_t n, int level, int max_len, int max_sec, const uint64_t *dep, void *X, int64_t row0,
                            cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + kFeatWarps - 1) / kFeatWarps, (int64_t)sm_count_cached() * 16);
    features_kernel<<<(unsigned)blocks, kFeatWarps * 32, 0, s>>>(nv, par, map, first, stride, n, level, max_len,
                                                                 max_sec, dep, reinterpret_cast<__nv_bfloat16 *>(X),
                                                                 row0);
    return cudaGetLastError();
}

cudaError_t launch_labels(const uint64_t *U, int W, const uint32_t *map, int64_t first, int64_t stride, int64_t n,
                          const uint64_t *ans, int64_t n_ans, float *y, int64_t row0, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 7) / 8, (int64_t)sm_count_cached() * 16);
    labels_kernel<<<(unsigned)blocks, 256, 0, s>>>(U, W, map, first, stride, n, ans, n_ans, y, row0);
    return cudaGetLastError();
}

cudaError_t launch_mlp_score(const void *X, int64_t n_rows, const void *wb, const float *params, float *score,
                             unsigned *err, cudaStream_t s)
{
    if (n_rows <= 0) return cudaSuccess;
    const int64_t tiles = (n_rows + kTR - 1) / kTR;
    const int grid = (int)std::min<int64_t>(tiles, sm_count_cached());
    cudaFuncSetAttribute(mlp_score_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ScoreSmem::BYTES);
    mlp_score_kernel<<<grid, kMlpThreads, ScoreSmem::BYTES, s>>>(reinterpret_cast<const __nv_bfloat16 *>(X), n_rows,
                                                                 reinterpret_cast<const __nv_bfloat16 *>(wb), params,
                                                                 score, err);
    return cudaGetLastError();
}

cudaError_t launch_mlp_train(const void *X, const float *y, int64_t n_rows, const int32_t *tiles, int n_tiles,
                             const void *wb, const float *params, float pos_weight, float inv_n, float *grad,
                             float *loss, unsigned *err, cudaStream_t s)
{
    if (n_tiles <= 0) return cudaSuccess;
    const int grid = std::min(n_tiles, sm_count_cached());
    cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TrainSmem::BYTES);
    mlp_train_kernel<<<grid, kMlpThreads, TrainSmem::BYTES, s>>>(
        reinterpret_cast<const __nv_bfloat16 *>(X), y, n_rows, tiles, n_tiles,
        reinterpret_cast<const __nv_bfloat16 *>(wb), params, pos_weight, inv_n, grad, loss, err);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *params, float *grad, float *mom, float lr, int step, void *wb, cudaStream_t s)
{
    const float c1 = 1.f - powf(0.9f, (float)step), c2 = 1.f - powf(0.999f, (float)step);
    adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(params, grad, mom, lr, c1, c2,
                                                        reinterpret_cast<__nv_bfloat16 *>(wb));
    return cudaGetLastError();
}

cudaError_t launch_pack_w(const float *params, void *wb, cudaStream_t s)
{
    pack_w_kernel<<<(kH * kF + 255) / 256, 256, 0, s>>>(params, reinterpret_cast<__nv_bfloat16 *>(wb));
    return cudaGetLastError();
}

cudaError_t launch_score_order(const float *score, int64_t n, const uint32_t *map, unsigned *hist, uint32_t *perm,
                               cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(hist, 0, kScoreBuckets * 4, s);
    if (e != cudaSuccess) return e;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count_cached() * 8);
    score_hist_kernel<<<blocks, 256, 0, s>>>(score, n, hist);
    score_scan_kernel<<<1, 1024, 0, s>>>(hist);
    score_scatter_kernel<<<blocks, 256, 0, s>>>(score, n, map, hist, perm);
    return cudaGetLastError();
}

cudaError_t launch_pack_rows(const float *x, int64_t n, void *X, int64_t row0, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    pack_rows_kernel<<<(unsigned)((n * kF + 255) / 256), 256, 0, s>>>(x, n, reinterpret_cast<__nv_bfloat16 *>(X), row0);
    return cudaGetLastError();
}

size_t mlp_score_smem() { return ScoreSmem::BYTES; }
size_t mlp_train_smem() { return TrainSmem::BYTES; }

}  // namespace efm
