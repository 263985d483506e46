// efm_kernels.cu -- sm_103a kernels of the pathway traversal.
//
// One traversal level (expansion of the frontier F_{l-1} into F_l) is the
// METAx step of Alg. 3 restated exhaustively and in exact integers:
//   * the acting metabolite of a pathway is its unbalanced internal
//     metabolite with the fewest reactions able to fix it (ties by index);
//     extra flux EF_i > 0 is a forward flow and all outputs of i are tried,
//     EF_i < 0 a backward flow and all inputs are tried (Def. 9, Eq. 3);
//   * the AND update gives the new reaction the flux that zeroes EF_i,
//     EF' = a*EF + c*S_int[:,k] with a = |S_ik|/g, c = |EF_i|/g,
//     g = gcd(|EF_i|, |S_ik|), then divides EF' by the gcd of its entries;
//     adding flux to a reaction already in the pathway is a secondary step
//     (Def. 10, Eq. 4) bounded by max_secondary (MAX_LOOP, Sec. 3.2);
//   * a balanced child (all metabolites Stable) goes to the arbiter
//     (Sec. 3.2.2) through a support hash set; an unbalanced child whose
//     support contains an accepted result is pruned (Def. 3 minimality);
//     the rest is deduplicated on (support, EF) in a hash table and the
//     new states are compacted into the next frontier.
// The arbiter decides minimality exactly: nullity(S_int[:,U]) == 1 is
// tested by Gaussian elimination modulo primes p = 2^31 - c, with enough
// primes that their product exceeds the Hadamard bound of the columns.
//
// Layout: one warp owns one parent pathway; lane l holds balance entries
// l, l + 32, ... (EPL per lane) and support words l, l + 32.  The static
// network (CSR by column and by metabolite, twins, pivot keys) is staged
// into shared memory with one bulk async copy (no multicast) when it fits.
#include "efm_internal.cuh"

namespace efm {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int kSpinLimit = 1 << 20;  // x ~1 us sleep: about one second

// primes p = 2^31 - c (c < 2^10), the 24 largest below 2^31
__constant__ uint32_t c_prime_c[kNumPrimes] = {1,   19,  61,  69,  85,  99,  105, 151, 159, 171, 225, 249,
                                              295, 325, 379, 399, 411, 469, 477, 511, 525, 571, 579, 589};

__device__ __forceinline__ uint64_t mix64(uint64_t x)
{
    // splitmix64 finaliser (Steele, Lea, Flood 2014)
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return x;
}

__device__ __forceinline__ uint64_t gcd64(uint64_t a, uint64_t b)
{
    // binary gcd (Stein)
    if (a == 0) return b;
    if (b == 0) return a;
    const int sh = __ffsll((long long)(a | b)) - 1;
    a >>= __ffsll((long long)a) - 1;
    while (b != 0) {
        b >>= __ffsll((long long)b) - 1;
        if (a > b) {
            const uint64_t t = a;
            a = b;
            b = t;
        }
        b -= a;
    }
    return a << sh;
}

__device__ __forceinline__ uint32_t gcd32(uint32_t a, uint32_t b)
{
    if (a == 0) return b;
    if (b == 0) return a;
    const int sh = __ffs((int)(a | b)) - 1;
    a >>= __ffs((int)a) - 1;
    while (b != 0) {
        b >>= __ffs((int)b) - 1;
        if (a > b) {
            const uint32_t t = a;
            a = b;
            b = t;
        }
        b -= a;
    }
    return a << sh;
}

__device__ __forceinline__ uint64_t abs64(int64_t x) { return x < 0 ? (uint64_t)(-x) : (uint64_t)x; }

template <int EPL>
__device__ __forceinline__ int32_t pick(const int32_t (&v)[EPL], int i)
{
    int32_t r = v[0];
#pragma unroll
    for (int e = 1; e < EPL; ++e)
        if (i == e) r = v[e];
    return r;
}

__device__ __forceinline__ bool bit_of(const uint64_t *U, int k) { return (U[k >> 6] >> (k & 63)) & 1ull; }

__device__ __forceinline__ unsigned long long load_volatile(unsigned long long *p)
{
    return *(volatile unsigned long long *)p;
}

// ---------------------------------------------------------------------------
// static network staging (a4): bulk async copy global -> shared, mbarrier
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Returns the blob pointer to use (shared if staged, else global).  On a
// wait that does not finish, flags ERR_TIMEOUT and returns nullptr.
__device__ const uint32_t *stage_blob(const NetView &nv, uint32_t *sblob, uint64_t *mbar, bool staged,
                                      unsigned long long *ctr)
{
    if (!staged) return nv.blob;
    const uint32_t bytes = (uint32_t)nv.blob_words * 4u;
    const uint32_t bar = smem_addr(mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        const uint32_t chunk = 32768u;
        for (uint32_t off = 0; off < bytes; off += chunk) {
            const uint32_t n = bytes - off < chunk ? bytes - off : chunk;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_addr(sblob) + off),
                "l"((const char *)nv.blob + off), "r"(n), "r"(bar)
                : "memory");
        }
    }
    uint32_t done = 0;
    for (int spin = 0; spin < kSpinLimit && !done; ++spin) {
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(bar), "r"(0)
            : "memory");
        if (!done) __nanosleep(256);
    }
    const int all_done = __syncthreads_and((int)done);
    if (!all_done) {
        if (threadIdx.x == 0) atomicOr(&ctr[C_ERR], (unsigned long long)ERR_TIMEOUT);
        return nullptr;
    }
    return sblob;
}

// ---------------------------------------------------------------------------
// warp-cooperative hash sets
// ---------------------------------------------------------------------------

enum { INS_NEW = 1, INS_DUP = 0, INS_ARENA_FULL = -1, INS_TIMEOUT = -2, INS_TABLE_FULL = -3 };

// Spin until the slot's index is published.  Returns the slot value or
// kEmpty on timeout.
__device__ __forceinline__ unsigned long long wait_published(unsigned long long *slot, unsigned long long v, int lane)
{
    int spins = 0;
    while ((uint32_t)v == kPending) {
        if (++spins > kSpinLimit) return kEmpty;
        __nanosleep(64);
        if (lane == 0) v = load_volatile(slot);
        v = __shfl_sync(FULL, v, 0);
    }
    return v;
}

__device__ __forceinline__ void slot_tag_pos(uint64_t h, uint64_t mask, uint64_t &pos, uint32_t &tag)
{
    const uint64_t f = mix64(h);
    pos = f & mask;
    tag = (uint32_t)(f >> 32);
    if (tag == 0xFFFFFFFFu) tag = 0xFFFFFFFEu;
}

// Insert a support set (balanced pathway) into the candidate set.
// Lane l holds words l and l + 32 of U in u0 / u1.
__device__ int insert_support(const LevelArgs &a, int W, uint64_t u0, uint64_t u1, int lane)
{
    uint64_t h = 0;
    if (lane < W) h += mix64(u0 ^ (0x51ed27f3a5b1c3d9ull * (uint64_t)(lane + 1)));
    if (lane + 32 < W) h += mix64(u1 ^ (0x51ed27f3a5b1c3d9ull * (uint64_t)(lane + 33)));
    const uint32_t lo = __reduce_add_sync(FULL, (uint32_t)h);
    const uint32_t hi = __reduce_add_sync(FULL, (uint32_t)(h >> 32));
    uint64_t pos;
    uint32_t tag;
    slot_tag_pos(((uint64_t)hi << 32) | lo, a.cslot_mask, pos, tag);
    for (uint64_t probe = 0; probe <= a.cslot_mask; ++probe) {
        unsigned long long v = 0;
        if (lane == 0) v = atomicCAS(&a.cslots[pos], kEmpty, ((unsigned long long)tag << 32) | kPending);
        v = __shfl_sync(FULL, v, 0);
        if (v == kEmpty) {
            unsigned long long idx = 0;
            if (lane == 0) idx = atomicAdd(&a.ctr[C_CAND_N], 1ull);
            idx = __shfl_sync(FULL, idx, 0);
            if ((int64_t)idx >= a.cand_cap) {
                if (lane == 0) {
                    atomicOr(&a.ctr[C_ERR], (unsigned long long)ERR_CAND_CAP);
                    atomicExch(&a.cslots[pos], ((unsigned long long)tag << 32) | kOverflowIdx);
                }
                return INS_ARENA_FULL;
            }
            uint64_t *dst = a.cand + (size_t)idx * W;
            if (lane < W) dst[lane] = u0;
            if (lane + 32 < W) dst[lane + 32] = u1;
            __threadfence();
            __syncwarp();
            if (lane == 0) atomicExch(&a.cslots[pos], ((unsigned long long)tag << 32) | idx);
            return INS_NEW;
        }
        if ((uint32_t)(v >> 32) == tag) {
            v = wait_published(&a.cslots[pos], v, lane);
            if (v == kEmpty) {
                if (lane == 0) atomicOr(&a.ctr[C_ERR], (unsigned long long)ERR_TIMEOUT);
                return INS_TIMEOUT;
            }
            const uint32_t idx = (uint32_t)v;
            if (idx == kOverflowIdx) return INS_ARENA_FULL;
            __threadfence();
            const uint64_t *src = a.cand + (size_t)idx * W;
            bool eq = true;
            if (lane < W) eq = __ldcg(src + lane) == u0;
            if (lane + 32 < W) eq = eq && (__ldcg(src + lane + 32) == u1);
            if (__all_sync(FULL, eq)) return INS_DUP;
        }
        pos = (pos + 1) & a.cslot_mask;
    }
    if (lane == 0) atomicOr(&a.ctr[C_ERR], (unsigned long long)ERR_TABLE_FULL);
    return INS_TABLE_FULL;
}

// Insert a pathway state (support + normalised extra flux) into the level's
// hash table; a new state is written into the child arena before its slot
// is published.
template <int EPL>
__device__ int insert_state(const LevelArgs &a, int W, int Mpad, uint64_t u0, uint64_t u1, const int32_t (&t)[EPL],
                            uint32_t meta, int lane)
{
    uint64_t h = 0;
    if (lane < W) h += mix64(u0 ^ (0x2545f4914f6cdd1dull * (uint64_t)(lane + 1)));
    if (lane + 32 < W) h += mix64(u1 ^ (0x2545f4914f6cdd1dull * (uint64_t)(lane + 33)));
#pragma unroll
    for (int e = 0; e < EPL; ++e)
        if (t[e] != 0) h += mix64(((uint64_t)(uint32_t)(lane + 32 * e) << 32) | (uint32_t)t[e]);
    const uint32_t lo = __reduce_add_sync(FULL, (uint32_t)h);
    const uint32_t hi = __reduce_add_sync(FULL, (uint32_t)(h >> 32));
    uint64_t pos;
    uint32_t tag;
    slot_tag_pos(((uint64_t)hi << 32) | lo, a.slot_mask, pos, tag);
    for (uint64_t probe = 0; probe <= a.slot_mask; ++probe) {
        unsigned long long v = 0;
        if (lane == 0) v = atomicCAS(&a.slots[pos], kEmpty, ((unsigned long long)tag << 32) | kPending);
        v = __shfl_sync(FULL, v, 0);
        if (v == kEmpty) {
            unsigned long long idx = 0;
            if (lane == 0) idx = atomicAdd(&a.ctr[C_NEXT], 1ull);
            idx = __shfl_sync(FULL, idx, 0);
            if ((int64_t)idx >= a.child.cap) {
                if (lane == 0) atomicExch(&a.slots[pos], ((unsigned long long)tag << 32) | kOverflowIdx);
                return INS_ARENA_FULL;
            }
            uint64_t *du = a.child.U + (size_t)idx * W;
            if (lane < W) du[lane] = u0;
            if (lane + 32 < W) du[lane + 32] = u1;
            int32_t *db = a.child.B + (size_t)idx * Mpad;
#pragma unroll
            for (int e = 0; e < EPL; ++e) db[lane + 32 * e] = t[e];
            if (lane == 0) a.child.meta[idx] = meta;
            __threadfence();
            __syncwarp();
            if (lane == 0) atomicExch(&a.slots[pos], ((unsigned long long)tag << 32) | idx);
            return INS_NEW;
        }
        if ((uint32_t)(v >> 32) == tag) {
            v = wait_published(&a.slots[pos], v, lane);
            if (v == kEmpty) {
                if (lane == 0) atomicOr(&a.ctr[C_ERR], (unsigned long long)ERR_TIMEOUT);
                return INS_TIMEOUT;
            }
            const uint32_t idx = (uint32_t)v;
            if (idx == kOverflowIdx) return INS_ARENA_FULL;
            __threadfence();
            const uint64_t *su = a.child.U + (size_t)idx * W;
            const int32_t *sb = a.child.B + (size_t)idx * Mpad;
            bool eq = true;
            if (lane < W) eq = __ldcg(su + lane) == u0;
            if (lane + 32 < W) eq = eq && (__ldcg(su + lane + 32) == u1);
#pragma unroll
            for (int e = 0; e < EPL; ++e) eq = eq && (__ldcg(sb + lane + 32 * e) == t[e]);
            if (__all_sync(FULL, eq)) return INS_DUP;
        }
        pos = (pos + 1) & a.slot_mask;
    }
    if (lane == 0) atomicOr(&a.ctr[C_ERR], (unsigned long long)ERR_TABLE_FULL);
    return INS_TABLE_FULL;
}

// ---------------------------------------------------------------------------
// shared pieces of the AND update
// ---------------------------------------------------------------------------

// Divide the raw child balance by the gcd of its entries (warp-wide) and
// report zero (balanced) and int32 overflow.  t64 in, t32 out.
template <int EPL>
__device__ __forceinline__ void normalise(int64_t (&t64)[EPL], int32_t (&t32)[EPL], bool &zero, bool &ovf)
{
    bool one = false, nz = false;
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
        one = one || (t64[e] == 1 || t64[e] == -1);
        nz = nz || (t64[e] != 0);
    }
    zero = !__any_sync(FULL, nz);
    if (zero) {
#pragma unroll
        for (int e = 0; e < EPL; ++e) t32[e] = 0;
        ovf = false;
        return;
    }
    if (!__any_sync(FULL, one)) {
        uint64_t g = 0;
#pragma unroll
        for (int e = 0; e < EPL; ++e) g = gcd64(g, abs64(t64[e]));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) g = gcd64(g, __shfl_xor_sync(FULL, g, off));
        if (g > 1) {
#pragma unroll
            for (int e = 0; e < EPL; ++e) t64[e] /= (int64_t)g;
        }
    }
    bool big = false;
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
        big = big || (t64[e] > 2147483647ll || t64[e] < -2147483647ll);
        t32[e] = (int32_t)t64[e];
    }
    ovf = __any_sync(FULL, big);
}

// Pivot key of a state: min over unbalanced rows of (degree << 16 | row).
template <int EPL>
__device__ __forceinline__ uint32_t pivot_key(const uint32_t *bl, const NetView &nv, const int32_t (&t)[EPL], int lane)
{
    uint32_t kmin = 0xFFFFFFFFu;
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
        if (t[e] != 0) {
            const int m = lane + 32 * e;
            const uint32_t k = t[e] > 0 ? bl[nv.o_keypos + m] : bl[nv.o_keyneg + m];
            kmin = k < kmin ? k : kmin;
        }
    }
    return __reduce_min_sync(FULL, kmin);
}

// Does any result E in [beg, end) (through the index list if ids != null)
// satisfy E subset of U' = U + column k?
__device__ bool any_result_subset(const uint64_t *res, int W, const int32_t *ids, int64_t beg, int64_t end,
                                  const uint64_t *Us, int kword, uint64_t kbit, int lane)
{
    for (int64_t base = beg; base < end; base += 32) {
        const int64_t i = base + lane;
        bool hit = false;
        if (i < end) {
            const int64_t r = ids ? (int64_t)ids[i] : i;
            const uint64_t *E = res + (size_t)r * W;
            hit = true;
            for (int w = 0; w < W; ++w) {
                const uint64_t uw = Us[w] | (w == kword ? kbit : 0ull);
                if (E[w] & ~uw) {
                    hit = false;
                    break;
                }
            }
        }
        if (__any_sync(FULL, hit)) return true;
    }
    return false;
}

// ---------------------------------------------------------------------------
// a0: seeds (INIT kernel analogue): flux 1 on every column producing the
// target (every column for target -1).
// ---------------------------------------------------------------------------

template <int EPL>
__global__ void __launch_bounds__(kExpandWarps * 32) seed_kernel(NetView nv, LevelArgs a, int target)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t *bl = nv.blob;
    const int W = nv.W;
    unsigned long long n_seed = 0, n_bal = 0, deg_sum = 0;
    const int n_items = target >= 0 ? nv.metptr[target + 1] - nv.metptr[target] : nv.N;
    for (int it = gw; it < n_items; it += nw) {
        int k = it;
        if (target >= 0) {
            const uint32_t e = nv.metent[nv.metptr[target] + it];
            if (ent_coef(e) <= 0) continue;
            k = ent_index(e);
        }
        ++n_seed;
        int64_t t64[EPL];
#pragma unroll
        for (int e = 0; e < EPL; ++e) t64[e] = 0;
        for (int q = (int)bl[nv.o_colptr + k]; q < (int)bl[nv.o_colptr + k + 1]; ++q) {
            const uint32_t ent = bl[nv.o_colent + q];
            const int row = ent_index(ent);
#pragma unroll
            for (int e = 0; e < EPL; ++e)
                if (row == lane + 32 * e) t64[e] = ent_coef(ent);
        }
        int32_t t[EPL];
        bool zero, ovf;
        normalise<EPL>(t64, t, zero, ovf);
        const uint64_t u0 = (lane == (k >> 6)) ? (1ull << (k & 63)) : 0ull;
        const uint64_t u1 = (lane + 32 == (k >> 6)) ? (1ull << (k & 63)) : 0ull;
        if (zero) {
            ++n_bal;
            insert_support(a, W, u0, u1, lane);
            continue;
        }
        const uint32_t key = pivot_key<EPL>(bl, nv, t, lane);
        // seeds are distinct columns: no deduplication needed
        unsigned long long idx = 0;
        if (lane == 0) idx = atomicAdd(&a.ctr[C_NEXT], 1ull);
        idx = __shfl_sync(FULL, idx, 0);
        if ((int64_t)idx < a.child.cap) {
            uint64_t *du = a.child.U + (size_t)idx * W;
            if (lane < W) du[lane] = u0;
            if (lane + 32 < W) du[lane + 32] = u1;
            int32_t *db = a.child.B + (size_t)idx * nv.Mpad;
#pragma unroll
            for (int e = 0; e < EPL; ++e) db[lane + 32 * e] = t[e];
            if (lane == 0) a.child.meta[idx] = key;
            deg_sum += key >> 16;
        }
    }
    if (lane == 0) {
        if (n_seed) atomicAdd(&a.ctr[C_SEEDS], n_seed);
        if (n_bal) atomicAdd(&a.ctr[C_BAL], n_bal);
        if (deg_sum) atomicAdd(&a.ctr[C_DEGSUM], deg_sum);
    }
}

// ---------------------------------------------------------------------------
// a1-a6: one level of expansion
// ---------------------------------------------------------------------------

template <int EPL>
__global__ void __launch_bounds__(kExpandWarps * 32) expand_kernel(NetView nv, LevelArgs a, int staged)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int W = nv.W;
    const int Mpad = nv.Mpad;
    uint32_t *sblob = smem;
    const int blob_words = staged ? nv.blob_words : 0;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + blob_words);
    uint64_t *Us = reinterpret_cast<uint64_t *>(smem + blob_words + 4) + wid * kMaxW;
    const uint32_t *bl = stage_blob(nv, sblob, mbar, staged != 0, a.ctr);
    if (bl == nullptr) return;

    unsigned long long n_exp = 0, n_ovf = 0, n_bal = 0, n_pruned = 0, deg_sum = 0;
    const int64_t gw = (int64_t)blockIdx.x * kExpandWarps + wid;
    const int64_t nw = (int64_t)gridDim.x * kExpandWarps;
    bool stop = false;
    for (int64_t p = gw; p < a.n_par && !stop; p += nw) {
        // load the parent pathway
        const uint64_t *pu = a.par.U + (size_t)p * W;
        const uint64_t pu0 = lane < W ? pu[lane] : 0ull;
        const uint64_t pu1 = lane + 32 < W ? pu[lane + 32] : 0ull;
        Us[lane] = pu0;
        Us[lane + 32] = pu1;
        int32_t b[EPL];
        const int32_t *pb = a.par.B + (size_t)p * Mpad;
#pragma unroll
        for (int e = 0; e < EPL; ++e) b[e] = pb[lane + 32 * e];
        const uint32_t meta = a.par.meta[p];
        __syncwarp();
        const int pc = __reduce_add_sync(FULL, (unsigned)(__popcll(pu0) + __popcll(pu1)));
        const int sec = a.level - pc;  // secondary steps taken by the parent
        const int piv = (int)(meta & 0xFFFFu);
        const int32_t bi = __shfl_sync(FULL, pick<EPL>(b, piv >> 5), piv & 31);
        const bool fwd = bi > 0;  // forward flow: consume the surplus
        const uint32_t abi = (uint32_t)(bi < 0 ? -bi : bi);
        const int lbeg = (int)bl[(fwd ? nv.o_consptr : nv.o_prodptr) + piv];
        const int lend = (int)bl[(fwd ? nv.o_consptr : nv.o_prodptr) + piv + 1];
        const int lent = fwd ? nv.o_consent : nv.o_prodent;
        for (int q = lbeg; q < lend; ++q) {
            const uint32_t br = bl[lent + q];
            const int k = ent_index(br);
            const uint32_t sik = (uint32_t)ent_coef(br);  // |S_ik|
            const int tw = (int)bl[nv.o_twin + k];
            if (tw >= 0 && bit_of(Us, tw)) continue;
            const bool in_u = bit_of(Us, k);
            if (!in_u && pc + 1 > a.max_len) continue;
            if (in_u && sec + 1 > a.max_sec) continue;
            ++n_exp;
            // AND update (Eq. 3 / Eq. 4 in integers)
            const uint32_t g = gcd32(abi, sik);
            const int64_t A = (int64_t)(sik / g), C = (int64_t)(abi / g);
            int64_t t64[EPL];
#pragma unroll
            for (int e = 0; e < EPL; ++e) t64[e] = A * (int64_t)b[e];
            for (int r = (int)bl[nv.o_colptr + k]; r < (int)bl[nv.o_colptr + k + 1]; ++r) {
                const uint32_t ent = bl[nv.o_colent + r];
                const int row = ent_index(ent);
                const int64_t add = C * (int64_t)ent_coef(ent);
#pragma unroll
                for (int e = 0; e < EPL; ++e)
                    if (row == lane + 32 * e) t64[e] += add;
            }
            int32_t t[EPL];
            bool zero, ovf;
            normalise<EPL>(t64, t, zero, ovf);
            if (ovf) {
                ++n_ovf;
                continue;
            }
            const int kword = k >> 6;
            const uint64_t kbit = 1ull << (k & 63);
            const uint64_t cu0 = pu0 | (lane == kword ? kbit : 0ull);
            const uint64_t cu1 = pu1 | (lane + 32 == kword ? kbit : 0ull);
            if (zero) {
                ++n_bal;
                const int rc = insert_support(a, W, cu0, cu1, lane);
                if (rc < INS_DUP) stop = true;
                continue;
            }
            // superset pruning against accepted results: results containing
            // column k (if new) and every result of the previous level
            bool pr = false;
            if (!in_u) pr = any_result_subset(a.res, W, a.bidx, a.bptr[k], a.bptr[k + 1], Us, kword, kbit, lane);
            if (!pr && a.recent_end > a.recent_begin)
                pr = any_result_subset(a.res, W, nullptr, a.recent_begin, a.recent_end, Us, kword, kbit, lane);
            if (pr) {
                ++n_pruned;
                continue;
            }
            const uint32_t key = pivot_key<EPL>(bl, nv, t, lane);
            const int rc = insert_state<EPL>(a, W, Mpad, cu0, cu1, t, key, lane);
            if (rc == INS_NEW) deg_sum += key >> 16;
            if (rc == INS_TIMEOUT || rc == INS_TABLE_FULL) stop = true;
        }
    }
    if (lane == 0) {
        if (n_exp) atomicAdd(&a.ctr[C_EXP], n_exp);
        if (n_ovf) atomicAdd(&a.ctr[C_OVF], n_ovf);
        if (n_bal) atomicAdd(&a.ctr[C_BAL], n_bal);
        if (n_pruned) atomicAdd(&a.ctr[C_PRUNED], n_pruned);
        if (deg_sum) atomicAdd(&a.ctr[C_DEGSUM], deg_sum);
    }
}

// ---------------------------------------------------------------------------
// a7/a8: exact minimality test by elimination modulo primes, then append.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t mulmod(uint32_t x, uint32_t y, uint32_t p, uint32_t c)
{
    // p = 2^31 - c: 2^31 == c (mod p)
    const uint64_t z = (uint64_t)x * y;
    const uint64_t r1 = (z & 0x7FFFFFFFull) + (z >> 31) * c;
    uint32_t r2 = (uint32_t)((r1 & 0x7FFFFFFFull) + (r1 >> 31) * c);
    if (r2 >= p) r2 -= p;
    return r2;
}

__device__ __forceinline__ uint32_t submod(uint32_t x, uint32_t y, uint32_t p) { return x >= y ? x - y : x + p - y; }

__device__ __forceinline__ uint32_t powmod(uint32_t x, uint32_t e, uint32_t p, uint32_t c)
{
    uint32_t r = 1;
    while (e) {
        if (e & 1u) r = mulmod(r, x, p, c);
        x = mulmod(x, x, p, c);
        e >>= 1;
    }
    return r;
}

__device__ __forceinline__ uint32_t to_mod(int32_t s, uint32_t p)
{
    return s >= 0 ? (uint32_t)s : p - (uint32_t)(-s);
}

// coefficient S_int[row, col] from the column CSR (0 if absent)
__device__ __forceinline__ int32_t coef_at(const uint32_t *bl, const NetView &nv, int col, int row)
{
    for (int q = (int)bl[nv.o_colptr + col]; q < (int)bl[nv.o_colptr + col + 1]; ++q) {
        const uint32_t e = bl[nv.o_colent + q];
        if (ent_index(e) == row) return ent_coef(e);
    }
    return 0;
}

// Do the columns cols[0..nn) of S_int have full column rank modulo p?
// Rows touched by the columns are streamed; each is reduced against the
// echelon basis held in shared memory (lane l owns columns l and l + 32).
__device__ bool full_rank_mod_p(const uint32_t *bl, const NetView &nv, const int *cols, int nn, uint32_t p, uint32_t c,
                                uint32_t *basis /* [64][64] */, int *pivcol /* [64] */, uint32_t *rowmap /* M bits */,
                                int lane)
{
    const int mwords = (nv.M + 31) >> 5;
    for (int w = lane; w < mwords; w += 32) rowmap[w] = 0;
    __syncwarp();
    const int c0 = lane < nn ? cols[lane] : -1;
    const int c1 = lane + 32 < nn ? cols[lane + 32] : -1;
    int rank = 0;
    for (int j = 0; j < nn; ++j) {
        const int col = cols[j];
        for (int q = (int)bl[nv.o_colptr + col]; q < (int)bl[nv.o_colptr + col + 1]; ++q) {
            const int row = ent_index(bl[nv.o_colent + q]);
            const uint32_t word = rowmap[row >> 5];
            if ((word >> (row & 31)) & 1u) continue;
            __syncwarp();
            if (lane == 0) rowmap[row >> 5] = word | (1u << (row & 31));
            __syncwarp();
            uint32_t y0 = c0 >= 0 ? to_mod(coef_at(bl, nv, c0, row), p) : 0u;
            uint32_t y1 = c1 >= 0 ? to_mod(coef_at(bl, nv, c1, row), p) : 0u;
            for (int i = 0; i < rank; ++i) {
                const int pc = pivcol[i];
                const uint32_t f = __shfl_sync(FULL, pc < 32 ? y0 : y1, pc & 31);
                if (f != 0) {
                    y0 = submod(y0, mulmod(f, basis[i * 64 + lane], p, c), p);
                    y1 = submod(y1, mulmod(f, basis[i * 64 + lane + 32], p, c), p);
                }
            }
            const unsigned m0 = __ballot_sync(FULL, y0 != 0);
            const unsigned m1 = __ballot_sync(FULL, y1 != 0);
            if (m0 == 0 && m1 == 0) continue;
            const int pv = m0 ? __ffs((int)m0) - 1 : 32 + __ffs((int)m1) - 1;
            const uint32_t v = __shfl_sync(FULL, pv < 32 ? y0 : y1, pv & 31);
            const uint32_t inv = powmod(v, p - 2u, p, c);
            basis[rank * 64 + lane] = mulmod(y0, inv, p, c);
            basis[rank * 64 + lane + 32] = mulmod(y1, inv, p, c);
            if (lane == 0) pivcol[rank] = pv;
            __syncwarp();
            ++rank;
            if (rank == nn) return true;
        }
    }
    return false;
}

__global__ void __launch_bounds__(kAcceptWarps * 32) accept_kernel(NetView nv, AcceptArgs a)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int W = nv.W;
    uint32_t *basis = smem + wid * (64 * 64);
    int *cols = reinterpret_cast<int *>(smem + kAcceptWarps * 64 * 64) + wid * 64;
    int *pivcol = reinterpret_cast<int *>(smem + kAcceptWarps * 64 * 64 + kAcceptWarps * 64) + wid * 64;
    uint32_t *rowmap = smem + kAcceptWarps * 64 * 64 + 2 * kAcceptWarps * 64 + wid * 32;
    const uint32_t *bl = nv.blob;
    unsigned long long n_acc = 0;
    const int64_t gw = (int64_t)blockIdx.x * kAcceptWarps + wid;
    const int64_t nw = (int64_t)gridDim.x * kAcceptWarps;
    for (int64_t ci = a.cand_begin + gw; ci < a.cand_end; ci += nw) {
        const uint64_t *U = a.cand + (size_t)ci * W;
        const uint64_t u0 = lane < W ? U[lane] : 0ull;
        const uint64_t u1 = lane + 32 < W ? U[lane + 32] : 0ull;
        // ascending column list: words 0..31 (lanes, slot 0), then 32..63
        const int n0 = __popcll(u0), n1 = __popcll(u1);
        int s0 = n0, s1 = n1;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int x0 = __shfl_up_sync(FULL, s0, off), x1 = __shfl_up_sync(FULL, s1, off);
            if (lane >= off) {
                s0 += x0;
                s1 += x1;
            }
        }
        const int tot0 = __shfl_sync(FULL, s0, 31);
        const int n = tot0 + __shfl_sync(FULL, s1, 31);
        if (n > 64) {
            if (lane == 0) atomicOr(&a.ctr[C_ERR], (unsigned long long)ERR_LEN);
            continue;
        }
        int pos0 = s0 - n0, pos1 = tot0 + s1 - n1;
        for (uint64_t x = u0; x; x &= x - 1) cols[pos0++] = lane * 64 + __ffsll((long long)x) - 1;
        for (uint64_t x = u1; x; x &= x - 1) cols[pos1++] = (lane + 32) * 64 + __ffsll((long long)x) - 1;
        __syncwarp();
        // Drop one column: the kept nn = n - 1 columns must be independent.
        // (The balanced flux ray is positive on every column of U, so the
        // dropped column is a combination of the others.)
        const int nn = n - 1;
        uint32_t hb = 0;
        if (lane < nn) hb += bl[nv.o_hbits + cols[lane]];
        if (lane + 32 < nn) hb += bl[nv.o_hbits + cols[lane + 32]];
        hb = __reduce_add_sync(FULL, hb);  // log2 of the squared Hadamard bound
        const int kp = (int)(hb / 61u) + 1;  // each prime gives > 2^30.5 = 2^(61/2)
        if (kp > kNumPrimes) {
            if (lane == 0) atomicOr(&a.ctr[C_ERR], (unsigned long long)ERR_PRIMES);
            continue;
        }
        bool ok = nn == 0;
        for (int pi = 0; pi < kp && !ok; ++pi) {
            const uint32_t cc = c_prime_c[pi];
            ok = full_rank_mod_p(bl, nv, cols, nn, 0x80000000u - cc, cc, basis, pivcol, rowmap, lane);
        }
        if (ok) {
            unsigned long long idx = 0;
            if (lane == 0) idx = atomicAdd(&a.ctr[C_RES_N], 1ull);
            idx = __shfl_sync(FULL, idx, 0);
            if ((int64_t)idx < a.res_cap) {
                uint64_t *dst = a.res + (size_t)idx * W;
                if (lane < W) dst[lane] = u0;
                if (lane + 32 < W) dst[lane + 32] = u1;
            } else if (lane == 0) {
                atomicOr(&a.ctr[C_ERR], (unsigned long long)ERR_RES_CAP);
            }
            ++n_acc;
        }
        __syncwarp();
    }
    if (lane == 0 && n_acc) atomicAdd(&a.ctr[C_RES], n_acc);
}

// ---------------------------------------------------------------------------
// result buckets by column (for the superset test)
// ---------------------------------------------------------------------------

__global__ void bucket_count_kernel(const uint64_t *res, int64_t n, int W, int32_t *bcnt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * W) return;
    const int w = (int)(i % W);
    for (uint64_t x = res[i]; x; x &= x - 1) atomicAdd(&bcnt[w * 64 + __ffsll((long long)x) - 1], 1);
}

__global__ void bucket_scan_kernel(const int32_t *bcnt, int N, int32_t *bptr)
{
    // single CTA of 1024 threads, N <= 4096: exclusive scan
    __shared__ int32_t part[1024];
    const int per = (N + 1023) / 1024;
    const int beg = threadIdx.x * per;
    int32_t s = 0;
    for (int i = beg; i < beg + per && i < N; ++i) s += bcnt[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int32_t run = part[threadIdx.x] - s;
    for (int i = beg; i < beg + per && i < N; ++i) {
        bptr[i] = run;
        run += bcnt[i];
    }
    if (threadIdx.x == 1023) bptr[N] = part[1023];
}

__global__ void bucket_fill_kernel(const uint64_t *res, int64_t n, int W, const int32_t *bptr, int32_t *bfill,
                                   int32_t *bidx)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * W) return;
    const int w = (int)(i % W);
    const int32_t r = (int32_t)(i / W);
    for (uint64_t x = res[i]; x; x &= x - 1) {
        const int k = w * 64 + __ffsll((long long)x) - 1;
        bidx[bptr[k] + atomicAdd(&bfill[k], 1)] = r;
    }
}

// ---------------------------------------------------------------------------
// output order: (|U|, ascending column list), bitonic sort of indices
// ---------------------------------------------------------------------------

__device__ bool support_greater(const uint64_t *res, int W, uint32_t x, uint32_t y)
{
    if (x == 0xFFFFFFFFu) return y != 0xFFFFFFFFu;
    if (y == 0xFFFFFFFFu) return false;
    const uint64_t *a = res + (size_t)x * W, *b = res + (size_t)y * W;
    int ca = 0, cb = 0;
    for (int w = 0; w < W; ++w) {
        ca += __popcll(a[w]);
        cb += __popcll(b[w]);
    }
    if (ca != cb) return ca > cb;
    for (int w = 0; w < W; ++w) {
        const uint64_t d = a[w] ^ b[w];
        if (d) {
            const uint64_t low = d & (~d + 1);
            return (a[w] & low) == 0;  // the set holding the smaller column is smaller
        }
    }
    return false;
}

__global__ void sort_init_kernel(uint32_t *idx, int64_t n, int64_t n2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n2) idx[i] = i < n ? (uint32_t)i : 0xFFFFFFFFu;
}

__global__ void bitonic_step_kernel(const uint64_t *res, int W, uint32_t *idx, int64_t n2, int64_t k, int64_t j)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n2) return;
    const int64_t l = i ^ j;
    if (l <= i) return;
    const uint32_t x = idx[i], y = idx[l];
    const bool up = (i & k) == 0;
    if (support_greater(res, W, x, y) == up) {
        idx[i] = y;
        idx[l] = x;
    }
}

__global__ void gather_kernel(const uint64_t *res, int W, const uint32_t *idx, int64_t n_keep, uint64_t *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_keep * W) return;
    const int64_t r = i / W;
    const int w = (int)(i % W);
    out[i] = res[(size_t)idx[r] * W + w];
}

template <int EPL>
cudaError_t launch_seed_t(const NetView &nv, const LevelArgs &a, int target, cudaStream_t s)
{
    const int items = target >= 0 ? 1024 : nv.N;
    int blocks = (items + kExpandWarps - 1) / kExpandWarps;
    if (blocks > 1024) blocks = 1024;
    seed_kernel<EPL><<<blocks, kExpandWarps * 32, 0, s>>>(nv, a, target);
    return cudaGetLastError();
}

template <int EPL>
cudaError_t launch_expand_t(const NetView &nv, const LevelArgs &a, int grid, cudaStream_t s)
{
    const bool staged = nv.blob_words * 4 <= kStageLimitBytes;
    const size_t sm = (size_t)(staged ? nv.blob_words : 0) * 4 + 16 + (size_t)kExpandWarps * kMaxW * 8;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(expand_kernel<EPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kStageLimitBytes + 16 + kExpandWarps * kMaxW * 8);
        attr_set = true;
    }
    expand_kernel<EPL><<<grid, kExpandWarps * 32, sm, s>>>(nv, a, staged ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace

#define EFM_EPL_DISPATCH(EPLV, CALL) \
    switch (EPLV) {                  \
    case 1: return CALL(1);          \
    case 2: return CALL(2);          \
    case 4: return CALL(4);          \
    case 8: return CALL(8);          \
    case 16: return CALL(16);        \
    case 28: return CALL(28);        \
    case 32: return CALL(32);        \
    default: return cudaErrorInvalidValue; \
    }

cudaError_t launch_seed(const NetView &nv, const LevelArgs &a, int target, cudaStream_t s)
{
#define CALL_SEED(E) launch_seed_t<E>(nv, a, target, s)
    EFM_EPL_DISPATCH(nv.EPL, CALL_SEED)
#undef CALL_SEED
}

cudaError_t launch_expand(const NetView &nv, const LevelArgs &a, int grid, cudaStream_t s)
{
#define CALL_EXP(E) launch_expand_t<E>(nv, a, grid, s)
    EFM_EPL_DISPATCH(nv.EPL, CALL_EXP)
#undef CALL_EXP
}

int expand_grid(const NetView &nv, int sm_count)
{
    // resident CTAs per SM are bounded by registers at 256 threads; take a
    // fixed multiple of the SM count (persistent grid-stride loop inside)
    (void)nv;
    return sm_count * 4;
}

cudaError_t launch_accept(const NetView &nv, const AcceptArgs &a, cudaStream_t s)
{
    const int64_t n = a.cand_end - a.cand_begin;
    if (n <= 0) return cudaSuccess;
    const size_t sm = (size_t)kAcceptWarps * (64 * 64 + 64 + 64 + 32) * 4;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(accept_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        attr_set = true;
    }
    int64_t blocks = (n + kAcceptWarps - 1) / kAcceptWarps;
    if (blocks > 4096) blocks = 4096;
    accept_kernel<<<(int)blocks, kAcceptWarps * 32, sm, s>>>(nv, a);
    return cudaGetLastError();
}

cudaError_t launch_buckets(const NetView &nv, const uint64_t *res, int64_t n_res, int32_t *bcnt, int32_t *bptr,
                           int32_t *bfill, int32_t *bidx, cudaStream_t s)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(bcnt, 0, sizeof(int32_t) * (size_t)nv.N, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(bfill, 0, sizeof(int32_t) * (size_t)nv.N, s)) != cudaSuccess) return e;
    const int64_t items = n_res * nv.W;
    const int tb = 256;
    if (items > 0) bucket_count_kernel<<<(int)((items + tb - 1) / tb), tb, 0, s>>>(res, n_res, nv.W, bcnt);
    bucket_scan_kernel<<<1, 1024, 0, s>>>(bcnt, nv.N, bptr);
    if (items > 0) bucket_fill_kernel<<<(int)((items + tb - 1) / tb), tb, 0, s>>>(res, n_res, nv.W, bptr, bfill, bidx);
    return cudaGetLastError();
}

cudaError_t launch_sort_results(const uint64_t *res, int64_t n, int W, uint32_t *idx, int64_t n2, uint64_t *out,
                                int64_t n_keep, cudaStream_t s)
{
    if (n <= 0 || n_keep <= 0) return cudaSuccess;
    const int tb = 256;
    const int blocks = (int)((n2 + tb - 1) / tb);
    sort_init_kernel<<<blocks, tb, 0, s>>>(idx, n, n2);
    for (int64_t k = 2; k <= n2; k <<= 1)
        for (int64_t j = k >> 1; j > 0; j >>= 1) bitonic_step_kernel<<<blocks, tb, 0, s>>>(res, W, idx, n2, k, j);
    const int64_t items = n_keep * W;
    gather_kernel<<<(int)((items + tb - 1) / tb), tb, 0, s>>>(res, W, idx, n_keep, out);
    return cudaGetLastError();
}

}  // namespace efm
