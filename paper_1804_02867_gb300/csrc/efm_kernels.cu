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
// Layout: a frontier is an arena of states, each a row of W support words,
// a row of Mpad int32 extra-flux entries (16-byte aligned) and a meta word
// (acting metabolite, its degree, |U|).  The expansion gives every lane its
// own child; the seed and minimality kernels give a warp one item.  The
// static network (CSR by column and by metabolite, twins, pivot keys) is
// staged into shared memory with one bulk async copy (no multicast) when it
// fits.
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

__device__ __forceinline__ bool bit_of(const uint64_t *U, int k) { return (U[k >> 6] >> (k & 63)) & 1ull; }

__device__ __forceinline__ unsigned long long load_volatile(unsigned long long *p)
{
    return *(volatile unsigned long long *)p;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

constexpr uint64_t kWatchdogNs = 20ull * 1000000000ull;  // a level that runs longer gives up
constexpr int kMaxRounds = 1 << 22;

// Record the first failed self-check (code, offending value, its limit) and
// raise the error bit; the caller skips the access.
__device__ void record_diag(unsigned long long *ctr, unsigned bit, unsigned long long code, long long value,
                            long long limit, int level)
{
    atomicOr(&ctr[C_ERR], (unsigned long long)bit);
    if (atomicCAS(&ctr[C_DIAG], 0ull, code) == 0ull) {
        ctr[C_DIAG + 1] = (unsigned long long)value;
        ctr[C_DIAG + 2] = (unsigned long long)limit;
        ctr[C_DIAG + 3] = (unsigned long long)level;
    }
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
__device__ const uint32_t *stage_words(const NetView &nv, uint32_t *sblob, uint64_t *mbar, int w0, int nwords,
                                       unsigned long long *ctr);

__device__ const uint32_t *stage_blob(const NetView &nv, uint32_t *sblob, uint64_t *mbar, bool staged,
                                      unsigned long long *ctr)
{
    if (!staged) return nv.blob;
    return stage_words(nv, sblob, mbar, 0, nv.blob_words, ctr);
}

// words [w0, w0 + nwords) of the blob into shared memory (w0 and nwords
// multiples of 4: 16-byte aligned bulk copies), one mbarrier, bounded wait
__device__ const uint32_t *stage_words(const NetView &nv, uint32_t *sblob, uint64_t *mbar, int w0, int nwords,
                                       unsigned long long *ctr)
{
    const uint32_t bytes = (uint32_t)nwords * 4u;
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
                "l"((const char *)(nv.blob + w0) + off), "r"(n), "r"(bar)
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
// hash sets (publish-after-write slots)
//
// A slot is one 64-bit word: (tag << 32) | index.  An inserter claims an
// empty slot with CAS as (tag, PENDING), writes the record, fences, then
// publishes the index.  A prober whose tag matches waits (bounded) for the
// index and compares the full record; records are never compared by tag
// alone, so the set is exact.
// ---------------------------------------------------------------------------

enum { INS_NEW = 1, INS_DUP = 0, INS_ARENA_FULL = -1, INS_TIMEOUT = -2, INS_TABLE_FULL = -3 };

__device__ __forceinline__ void slot_tag_pos(uint64_t h, uint64_t mask, uint64_t &pos, uint32_t &tag)
{
    const uint64_t f = mix64(h);
    pos = f & mask;
    tag = (uint32_t)(f >> 32);
    if (tag == 0xFFFFFFFFu) tag = 0xFFFFFFFEu;
}

// word w of the support U' = U (pu, or empty if null) plus column k
__device__ __forceinline__ uint64_t child_word(const uint64_t *pu, int w, int k)
{
    uint64_t x = pu ? pu[w] : 0ull;
    if (w == (k >> 6)) x |= 1ull << (k & 63);
    return x;
}

// Insert the support U' = U + {k} of a balanced pathway into the set of
// supports judged in this traversal (one thread).
__device__ __noinline__ int insert_support(const LevelArgs &a, int W, const uint64_t *pu, int k)
{
    uint64_t h = 0;
    for (int w = 0; w < W; ++w) h += mix64(child_word(pu, w, k) ^ (0x51ed27f3a5b1c3d9ull * (uint64_t)(w + 1)));
    uint64_t pos;
    uint32_t tag;
    slot_tag_pos(h, a.cslot_mask, pos, tag);
    for (uint64_t probe = 0; probe <= a.cslot_mask; ++probe) {
        unsigned long long v = atomicCAS(&a.cslots[pos], kEmpty, ((unsigned long long)tag << 32) | kPending);
        if (v == kEmpty) {
            const unsigned long long idx = atomicAdd(&a.ctr[C_CAND_N], 1ull);
            if ((int64_t)idx >= a.cand_cap) {
                atomicOr(&a.ctr[C_ERR], (unsigned long long)ERR_CAND_CAP);
                atomicExch(&a.cslots[pos], ((unsigned long long)tag << 32) | kOverflowIdx);
                return INS_ARENA_FULL;
            }
            uint64_t *dst = a.cand + (size_t)idx * W;
            for (int w = 0; w < W; ++w) dst[w] = child_word(pu, w, k);
            __threadfence();
            atomicExch(&a.cslots[pos], ((unsigned long long)tag << 32) | idx);
            return INS_NEW;
        }
        if ((uint32_t)(v >> 32) == tag) {
            int spins = 0;
            while ((uint32_t)v == kPending) {
                if (++spins > kSpinLimit) {
                    atomicOr(&a.ctr[C_ERR], (unsigned long long)ERR_TIMEOUT);
                    return INS_TIMEOUT;
                }
                __nanosleep(64);
                v = load_volatile(&a.cslots[pos]);
            }
            const uint32_t idx = (uint32_t)v;
            if (idx == kOverflowIdx) return INS_ARENA_FULL;
            const uint64_t *src = a.cand + (size_t)idx * W;
            bool eq = true;
            for (int w = 0; w < W && eq; ++w) eq = __ldcg(src + w) == child_word(pu, w, k);
            if (eq) return INS_DUP;
        }
        pos = (pos + 1) & a.cslot_mask;
    }
    atomicOr(&a.ctr[C_ERR], (unsigned long long)ERR_TABLE_FULL);
    return INS_TABLE_FULL;
}

// 64-bit recomputation of a child's raw entries (rare: some entry left the
// int32 range): gcd and largest magnitude over the lane's entries.
struct GcdMax {
    uint64_t g, m;
};
__device__ __noinline__ GcdMax raw_gcd_max(const int4 *prow4, const int4 *col4, int gl, int G, int CPL, int32_t A,
                                           int32_t C)
{
    GcdMax r{0, 0};
    for (int i = 0; i < CPL; ++i) {
        const int4 v = prow4[gl + G * i];
        const int4 w = col4[gl + G * i];
        const int32_t pv[4] = {v.x, v.y, v.z, v.w}, cv[4] = {w.x, w.y, w.z, w.w};
        for (int jj = 0; jj < 4; ++jj) {
            const uint64_t at = abs64((int64_t)A * pv[jj] + (int64_t)C * cv[jj]);
            if (at != 0) {
                r.g = r.g == 0 ? at : gcd64(r.g, at);
                r.m = at > r.m ? at : r.m;
            }
        }
    }
    return r;
}

// Supports of more than two words: does the result with bucket position i
// (id list, column lists) lie inside U + {k}?  Its columns are probed
// independently (no early exit), so the loads overlap.
__device__ __forceinline__ bool result_inside_wide(const LevelArgs &a, const uint64_t *pu, int k, int64_t i)
{
    const uint16_t *lst = a.rcols + (size_t)a.bids[i] * kRcolStride;
    const int n = lst[0];
    bool sub = true;
    for (int j = 1; j <= n; ++j) {
        const int c = lst[j];
        sub = sub && (c == k || bit_of(pu, c));
    }
    return sub;
}

// pivot key (degree << 16 | row) -> state meta: row | degree << 10 | |U| << 23
__device__ __forceinline__ uint32_t pack_meta(uint32_t key, int pc)
{
    return (key & 0x3FFu) | ((key >> 16) << 10) | ((uint32_t)pc << 23);
}

// Pivot key of a state: min over unbalanced rows of (degree << 16 | row)
// (warp-cooperative; lane l holds rows l + 32 e).
template <int EPL>
__device__ __forceinline__ uint32_t pivot_key(const uint32_t *bl, const NetView &nv, const int32_t (&t)[EPL], int lane)
{
    uint32_t kmin = 0xFFFFFFFFu;
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
        const int m = lane + 32 * e;
        if (t[e] != 0 && m < nv.M) {  // rows past M hold flux (subtractive variant) or padding
            const uint32_t k = t[e] > 0 ? bl[nv.o_keypos + m] : bl[nv.o_keyneg + m];
            kmin = k < kmin ? k : kmin;
        }
    }
    return __reduce_min_sync(FULL, kmin);
}

// The meta word's degree field counts the branches a state has: the list of
// the pivot's side, plus (subtractive variant) the opposite list.
__device__ __forceinline__ uint32_t branch_key(const uint32_t *bl, const NetView &nv, uint32_t key, int sub)
{
    if (!sub) return key;
    const int m = (int)(key & 0xFFFFu);
    const uint32_t deg = (bl[nv.o_consptr + m + 1] - bl[nv.o_consptr + m]) + (bl[nv.o_prodptr + m + 1] - bl[nv.o_prodptr + m]);
    return (deg << 16) | (key & 0xFFFFu);
}

// warp-wide test: all balance rows (m < M) of a row held across the warp are 0
template <int EPL>
__device__ __forceinline__ bool balance_zero(const int32_t (&t)[EPL], int M, int lane)
{
    bool nz = false;
#pragma unroll
    for (int e = 0; e < EPL; ++e) nz = nz || (t[e] != 0 && lane + 32 * e < M);
    return !__any_sync(FULL, nz);
}

// warp-cooperative normalisation of a seed column (t64 in, t32 out)
template <int EPL>
__device__ __forceinline__ void normalise(int64_t (&t64)[EPL], int32_t (&t32)[EPL], bool &zero)
{
    bool nz = false;
    uint64_t g = 0;
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
        nz = nz || (t64[e] != 0);
        g = gcd64(g, abs64(t64[e]));
    }
    zero = !__any_sync(FULL, nz);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) g = gcd64(g, __shfl_xor_sync(FULL, g, off));
#pragma unroll
    for (int e = 0; e < EPL; ++e) t32[e] = (int32_t)(g > 1 ? t64[e] / (int64_t)g : t64[e]);
}

// ---------------------------------------------------------------------------
// narrow networks (at most 64 internal rows): per-state summaries of the
// extra-flux row, see generate_narrow below
// ---------------------------------------------------------------------------

struct NarrowSum {
    uint64_t rh, pm, nm, um, om;
    uint32_t pmax;
};

__device__ __forceinline__ uint64_t blob_u64(const uint32_t *bl, int o)
{
    return (uint64_t)bl[o] | ((uint64_t)bl[o + 1] << 32);
}

// Summaries of a full row held across a warp (entry m = lane + 32 e).
template <int EPL>
__device__ NarrowSum warp_summary(const uint32_t *bl, const NetView &nv, const int32_t (&t)[EPL], int lane)
{
    NarrowSum r{0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
        const int m = lane + 32 * e;
        const int32_t v = t[e];
        if (m < nv.M && v != 0) {
            const uint32_t rk = bl[nv.o_rank + m];
            if (v > 0) r.pm |= 1ull << (rk & 0xFFu);
            else r.nm |= 1ull << ((rk >> 8) & 0xFFu);
            if (v == 1 || v == -1) r.um |= 1ull << m;
            if (v & 1) r.om |= 1ull << m;
            const uint32_t a = (uint32_t)(v < 0 ? -v : v);
            r.pmax = a > r.pmax ? a : r.pmax;
            r.rh += (uint64_t)(int64_t)v * blob_u64(bl, nv.o_hrow + 2 * m);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        r.pm |= __shfl_xor_sync(FULL, r.pm, off);
        r.nm |= __shfl_xor_sync(FULL, r.nm, off);
        r.um |= __shfl_xor_sync(FULL, r.um, off);
        r.om |= __shfl_xor_sync(FULL, r.om, off);
        r.rh += __shfl_xor_sync(FULL, r.rh, off);
        const uint32_t o = __shfl_xor_sync(FULL, r.pmax, off);
        r.pmax = o > r.pmax ? o : r.pmax;
    }
    return r;
}

// the summary record of a state: 6 words, written as three 16-byte stores
__device__ __forceinline__ void put_summary(uint64_t *d, const NarrowSum &s)
{
    *reinterpret_cast<ulonglong2 *>(d) = make_ulonglong2(s.rh, s.pm);
    *reinterpret_cast<ulonglong2 *>(d + 2) = make_ulonglong2(s.nm, s.um);
    *reinterpret_cast<ulonglong2 *>(d + 4) = make_ulonglong2(s.om, (uint64_t)s.pmax);
}

__device__ __forceinline__ NarrowSum get_summary(const uint64_t *d)
{
    const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(d);
    const ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(d + 2);
    const ulonglong2 c = *reinterpret_cast<const ulonglong2 *>(d + 4);
    return NarrowSum{a.x, a.y, b.x, b.y, c.x, (uint32_t)c.y};
}

__device__ __forceinline__ void store_summary(const Arena &ar, uint64_t idx, const NarrowSum &s, int lane)
{
    if (lane == 0) put_summary(ar.sum + (size_t)idx * kSumWords, s);
}

// pivot key from the two masks (0xFFFFFFFF when balanced)
__device__ __forceinline__ uint32_t mask_key(const uint32_t *bl, const NetView &nv, uint64_t pm, uint64_t nm)
{
    const uint32_t kp = pm ? bl[nv.o_keyr + __ffsll((long long)pm) - 1] : 0xFFFFFFFFu;
    const uint32_t kn = nm ? bl[nv.o_keyr + kNarrowKeyRanks + __ffsll((long long)nm) - 1] : 0xFFFFFFFFu;
    return kp < kn ? kp : kn;
}

// 64-bit hash of the support words (W words of U plus column k)
__device__ __forceinline__ uint64_t support_hash(const uint64_t *pu, int W, int k)
{
    uint64_t h = 0;
    for (int w = 0; w < W; ++w) h += mix64(child_word(pu, w, k) ^ (0x2545f4914f6cdd1dull * (uint64_t)(w + 1)));
    return h;
}

// ---------------------------------------------------------------------------
// a0: seeds (INIT kernel analogue): flux 1 on every column producing the
// target (every column for target -1).  One warp per seed.
// ---------------------------------------------------------------------------

template <int EPL>
__device__ void seed_range(const NetView &nv, const LevelArgs &a, int target, int gw, int nw)
{
    const int lane = threadIdx.x & 31;
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
        // the seed's row: column k of the dense copy (S_int[:, k], then, in
        // the subtractive variant's view, flux 1 on k)
        const int32_t *dk = reinterpret_cast<const int32_t *>(bl + nv.o_dcols) + (size_t)k * nv.Mpad;
        int64_t t64[EPL];
#pragma unroll
        for (int e = 0; e < EPL; ++e) t64[e] = dk[lane + 32 * e];
        int32_t t[EPL];
        bool zero;
        normalise<EPL>(t64, t, zero);
        zero = balance_zero<EPL>(t, nv.M, lane);
        if (zero) {
            ++n_bal;
            if (lane == 0) insert_support(a, W, nullptr, k);
            __syncwarp();
            continue;
        }
        const uint32_t key = pivot_key<EPL>(bl, nv, t, lane);
        // seeds are distinct columns: no deduplication needed
        unsigned long long idx = 0;
        if (lane == 0) idx = atomicAdd(&a.ctr[C_NEXT], 1ull);
        idx = __shfl_sync(FULL, idx, 0);
        if ((int64_t)idx < a.child.cap) {
            uint64_t *du = a.child.U + (size_t)idx * W;
            for (int w = lane; w < W; w += 32) du[w] = child_word(nullptr, w, k);
            int32_t *db = a.child.B + (size_t)idx * nv.Mpad;
#pragma unroll
            for (int e = 0; e < EPL; ++e) db[lane + 32 * e] = t[e];
            const uint32_t bkey = branch_key(bl, nv, key, a.sub);
            if (lane == 0) a.child.meta[idx] = pack_meta(bkey, 1);
            deg_sum += bkey >> 16;
            if (a.child.fx) {  // the lane masks of {k}: column k's own
                const int G = EPL >= 8 ? 32 : 4 * EPL;
                for (int x = lane; x < 2 * G; x += 32)
                    a.child.fx[(size_t)idx * (2 * G) + x] = bl[(x < G ? nv.o_fixc : nv.o_fixp) + k * G + x % G];
            }
        }
        if (EPL <= 2 && nv.narrow && a.child.sum) {
            const NarrowSum sm = warp_summary<EPL>(bl, nv, t, lane);
            if ((int64_t)idx < a.child.cap) store_summary(a.child, idx, sm, lane);
        }
    }
    if (lane == 0) {
        if (n_seed) atomicAdd(&a.ctr[C_SEEDS], n_seed);
        if (n_bal) atomicAdd(&a.ctr[C_BAL], n_bal);
        if (deg_sum) atomicAdd(&a.ctr[C_DEGSUM], deg_sum);
    }
}

template <int EPL>
__global__ void __launch_bounds__(kExpandWarps * 32) seed_kernel(NetView nv, LevelArgs a, int target)
{
    seed_range<EPL>(nv, a, target, (blockIdx.x * blockDim.x + threadIdx.x) >> 5, (gridDim.x * blockDim.x) >> 5);
}

// ---------------------------------------------------------------------------
// Monte-Carlo mode: the paper's own random walks (Alg. 3 with one random OR
// branch per step), in the exact integer form of the traversal.  One warp
// per walk; entry m of the extra-flux row sits in lane m % 32.  Walk w draws
// its numbers from counters 128 w + s (s = 0 picks the seed column, s >= 1
// the branch of step s): the first output of SplitMix64 (Steele, Lea and
// Flood, 2014) started from state seed + counter * 0x9E3779B97F4A7C15.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint64_t splitmix_at(uint64_t seed, uint64_t c)
{
    uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// gcd normalisation of a row held across the warp, with the int32 range test
template <int EPL>
__device__ __forceinline__ void walk_normalise(const int64_t (&t64)[EPL], int32_t (&t)[EPL], bool &zero, bool &ovf)
{
    uint64_t g = 0;
#pragma unroll
    for (int e = 0; e < EPL; ++e) g = gcd64(g, abs64(t64[e]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) g = gcd64(g, __shfl_xor_sync(FULL, g, off));
    zero = g == 0;
    bool bad = false;
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
        const int64_t v = g > 1 ? t64[e] / (int64_t)g : t64[e];
        bad = bad || v > 2147483647ll || v < -2147483647ll;
        t[e] = (int32_t)v;
    }
    ovf = __any_sync(FULL, bad);
}

template <int EPL>
__global__ void __launch_bounds__(kExpandWarps * 32) walk_kernel(NetView nv, LevelArgs a, int target, uint64_t seed,
                                                                 int64_t n_walks)
{
    __shared__ uint64_t sU[kExpandWarps][kMaxW];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t *U = sU[wid];
    const uint32_t *bl = nv.blob;
    const int W = nv.W, Mpad = nv.Mpad;
    const int32_t *dcol = reinterpret_cast<const int32_t *>(bl + nv.o_dcols);
    unsigned long long n_walk = 0, n_exp = 0, n_ovf = 0, n_bal = 0, n_dead = 0, max_steps = 0;
    bool fatal = false;
    // the target's seed columns: its row's positive entries, ascending columns
    const int tb = target >= 0 ? nv.metptr[target] : 0;
    const int te = target >= 0 ? nv.metptr[target + 1] : 0;
    int n_seeds = target >= 0 ? 0 : nv.N;
    for (int q0 = tb; q0 < te; q0 += 32) {
        const int q = q0 + lane;
        n_seeds += __popc(__ballot_sync(FULL, q < te && ent_coef(nv.metent[q]) > 0));
    }
    const int64_t gw = (int64_t)blockIdx.x * kExpandWarps + wid, nw = (int64_t)gridDim.x * kExpandWarps;
    for (int64_t w = gw; w < n_walks && n_seeds > 0 && !fatal; w += nw) {
        const uint64_t c0 = (uint64_t)w * 128u;
        int pick = (int)(splitmix_at(seed, c0) % (uint64_t)n_seeds);
        int j = pick;
        if (target >= 0) {
            for (int q0 = tb; q0 < te; q0 += 32) {
                const int q = q0 + lane;
                const unsigned m = __ballot_sync(FULL, q < te && ent_coef(nv.metent[q]) > 0);
                const int c = __popc(m);
                if (pick < c) {
                    j = ent_index(nv.metent[q0 + (int)__fns(m, 0, pick + 1)]);
                    break;
                }
                pick -= c;
            }
        }
        ++n_walk;
        for (int x = lane; x < W; x += 32) U[x] = x == (j >> 6) ? 1ull << (j & 63) : 0ull;
        __syncwarp();
        int64_t t64[EPL];
#pragma unroll
        for (int e = 0; e < EPL; ++e) t64[e] = dcol[(size_t)j * Mpad + lane + 32 * e];
        int32_t t[EPL];
        bool zero, ovf;
        walk_normalise<EPL>(t64, t, zero, ovf);
        if (ovf) {
            ++n_ovf;
            continue;
        }
        int pc = 1, sec = 0;
        unsigned long long steps = 0;
        for (int s = 1;; ++s) {
            if (zero) {
                ++n_bal;
                if (lane == 0 && insert_support(a, W, U, j) < INS_DUP) fatal = true;
                fatal = __any_sync(FULL, fatal);
                break;
            }
            if (s > 127) {  // every step adds a column or a secondary step: unreachable
                if (lane == 0) record_diag(a.ctr, ERR_BOUNDS, 5, s, 127, 0);
                fatal = true;
                break;
            }
            const uint32_t key = pivot_key<EPL>(bl, nv, t, lane);
            const int piv = (int)(key & 0xFFFFu);
            int32_t mine = 0;
#pragma unroll
            for (int e = 0; e < EPL; ++e)
                if (e == (piv >> 5)) mine = t[e];
            const int32_t bi = __shfl_sync(FULL, mine, piv & 31);
            const bool fwd = bi > 0;
            const int lptr = (fwd ? nv.o_consptr : nv.o_prodptr) + piv;
            const int lb = (int)bl[lptr], le = (int)bl[lptr + 1];
            const int lent = fwd ? nv.o_consent : nv.o_prodent;
            auto valid_at = [&](int q) -> bool {
                if (q >= le) return false;
                const int k = ent_index(bl[lent + q]);
                const int tw = (int)bl[nv.o_twin + k];
                if (tw >= 0 && bit_of(U, tw)) return false;
                return bit_of(U, k) ? sec + 1 <= a.max_sec : pc + 1 <= a.max_len;
            };
            int cnt = 0;
            for (int q0 = lb; q0 < le; q0 += 32) cnt += __popc(__ballot_sync(FULL, valid_at(q0 + lane)));
            if (cnt == 0) {
                ++n_dead;
                break;
            }
            int r = (int)(splitmix_at(seed, c0 + (uint64_t)s) % (uint64_t)cnt);
            int qs = lb;
            for (int q0 = lb; q0 < le; q0 += 32) {
                const unsigned m = __ballot_sync(FULL, valid_at(q0 + lane));
                const int c = __popc(m);
                if (r < c) {
                    qs = q0 + (int)__fns(m, 0, r + 1);
                    break;
                }
                r -= c;
            }
            const uint32_t br = bl[lent + qs];
            const int k = ent_index(br);
            const uint32_t sik = (uint32_t)ent_coef(br);  // |S_ik|
            const uint32_t abi = (uint32_t)(bi < 0 ? -bi : bi);
            const uint32_t g0 = gcd32(abi, sik);
            const int64_t A = (int64_t)(sik / g0), C = (int64_t)(abi / g0);
#pragma unroll
            for (int e = 0; e < EPL; ++e) t64[e] = A * t[e] + C * dcol[(size_t)k * Mpad + lane + 32 * e];
            ++n_exp;
            ++steps;
            const bool in_u = bit_of(U, k);
            __syncwarp();
            if (in_u) {
                ++sec;
            } else {
                if (lane == 0) U[k >> 6] |= 1ull << (k & 63);
                ++pc;
            }
            __syncwarp();
            j = k;
            walk_normalise<EPL>(t64, t, zero, ovf);
            if (ovf) {
                ++n_ovf;
                break;
            }
        }
        max_steps = steps > max_steps ? steps : max_steps;
    }
    if (lane == 0) {
        if (n_walk) atomicAdd(&a.ctr[C_SEEDS], n_walk);
        if (n_exp) atomicAdd(&a.ctr[C_EXP], n_exp);
        if (n_ovf) atomicAdd(&a.ctr[C_OVF], n_ovf);
        if (n_bal) atomicAdd(&a.ctr[C_BAL], n_bal);
        if (n_dead) atomicAdd(&a.ctr[C_PRUNED], n_dead);
        if (max_steps) atomicMax(&a.ctr[C_LEVELS], max_steps);
    }
}

// Seed set R_in (Prop. 1): one state with flux 1 on each column of R_in,
// EF = the sum of their S_int columns, normalised.  One warp.
template <int EPL>
__global__ void __launch_bounds__(32) seedset_kernel(NetView nv, LevelArgs a, const int32_t *cols, int n_cols)
{
    __shared__ uint64_t U[kMaxW];
    const int lane = threadIdx.x & 31;
    const int W = nv.W, Mpad = nv.Mpad;
    const int32_t *dcol = reinterpret_cast<const int32_t *>(nv.blob + nv.o_dcols);
    for (int x = lane; x < W; x += 32) U[x] = 0ull;
    __syncwarp();
    int64_t t64[EPL];
#pragma unroll
    for (int e = 0; e < EPL; ++e) t64[e] = 0;
    for (int i = 0; i < n_cols; ++i) {
        const int k = cols[i];
#pragma unroll
        for (int e = 0; e < EPL; ++e) t64[e] += dcol[(size_t)k * Mpad + lane + 32 * e];
        if (lane == 0) U[k >> 6] |= 1ull << (k & 63);
        __syncwarp();
    }
    int32_t t[EPL];
    bool zero, ovf;
    walk_normalise<EPL>(t64, t, zero, ovf);
    zero = balance_zero<EPL>(t, nv.M, lane);
    if (lane == 0) atomicAdd(&a.ctr[C_SEEDS], 1ull);
    if (ovf) {
        if (lane == 0) atomicAdd(&a.ctr[C_OVF], 1ull);
        return;
    }
    if (zero) {
        if (lane == 0) {
            atomicAdd(&a.ctr[C_BAL], 1ull);
            insert_support(a, W, U, cols[0]);
        }
        return;
    }
    const uint32_t key = pivot_key<EPL>(nv.blob, nv, t, lane);
    if (a.child.cap < 1) return;
    if (EPL <= 2 && nv.narrow && a.child.sum) {
        const NarrowSum sm = warp_summary<EPL>(nv.blob, nv, t, lane);
        store_summary(a.child, 0, sm, lane);
    }
    for (int x = lane; x < W; x += 32) a.child.U[x] = U[x];
#pragma unroll
    for (int e = 0; e < EPL; ++e) a.child.B[lane + 32 * e] = t[e];
    if (a.child.fx) {  // the lane masks of R_in: the union of its columns'
        const int G = EPL >= 8 ? 32 : 4 * EPL;
        for (int x = lane; x < 2 * G; x += 32) {
            uint32_t f = 0;
            for (int i = 0; i < n_cols; ++i) f |= nv.blob[(x < G ? nv.o_fixc : nv.o_fixp) + cols[i] * G + x % G];
            a.child.fx[x] = f;
        }
    }
    const uint32_t bkey = branch_key(nv.blob, nv, key, a.sub);
    if (lane == 0) {
        a.child.meta[0] = pack_meta(bkey, n_cols);
        atomicAdd(&a.ctr[C_NEXT], 1ull);
        atomicAdd(&a.ctr[C_DEGSUM], (unsigned long long)(bkey >> 16));
    }
}

// ---------------------------------------------------------------------------
// a1-a6: one level of expansion.
//
// Phase 1: a warp takes up to 32 consecutive parents; their branch counts
// (the static degree of each parent's acting metabolite, kept in the state's
// meta word) are prefix-summed across the lanes.  The warp then examines the
// flattened (parent, branch) items 32 at a time, one per lane (branch
// selection and the twin, length and first-K rules), and its groups of G
// lanes take the valid items in order, one child per group.  In a group,
// lane l holds the 16-byte chunks l, l + G, ... of the extra-flux row (CPL
// chunks, 4 * CPL entries), so row loads are coalesced and every reduction
// is log2(G) shuffles.  The AND update reads column k of S_int from a dense
// column-major copy of S_int (staged in shared memory with the rest of the
// static network when it fits) and stays in 32 bits unless a group needs the
// gcd or has an entry outside int32.  The group then applies the superset
// rule (its lanes split the results containing the new column) and appends
// surviving unbalanced children to a per-warp batch in shared memory.
//
// Phase 2 (one lane per batched child, NB children at once; the whole warp
// per child for wide rows): claim / write / publish / compare in the state
// hash table, so the latency of the atomics is paid once per batch, not per
// child.
// ---------------------------------------------------------------------------

template <int G>
__device__ __forceinline__ uint32_t group_or(uint32_t x)
{
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) x |= __shfl_xor_sync(FULL, x, off);
    return x;
}
template <int G>
__device__ __forceinline__ uint32_t group_min(uint32_t x)
{
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        const uint32_t y = __shfl_xor_sync(FULL, x, off);
        x = y < x ? y : x;
    }
    return x;
}
template <int G>
__device__ __forceinline__ uint32_t group_add(uint32_t x)
{
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) x += __shfl_xor_sync(FULL, x, off);
    return x;
}
template <int G>
__device__ __forceinline__ uint32_t group_xor(uint32_t x)
{
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) x ^= __shfl_xor_sync(FULL, x, off);
    return x;
}

__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void store_release(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long cas_acquire(unsigned long long *p, unsigned long long cmp,
                                                          unsigned long long v)
{
    unsigned long long old;
    asm volatile("atom.acquire.gpu.global.cas.b64 %0, [%1], %2, %3;" : "=l"(old) : "l"(p), "l"(cmp), "l"(v) : "memory");
    return old;
}

// 32-bit mixing of one balance entry (row m, value v) into two sums
__device__ __forceinline__ void hash_entry(uint32_t m, uint32_t v, uint32_t &lo, uint32_t &hi)
{
    const uint32_t x = (v ^ (m * 0x9E3779B9u)) * 0x85EBCA6Bu;
    lo += x ^ (x >> 16);
    hi ^= x + m;
}

// children per warp batch for a row of 16-byte chunks nch (shared memory
// per warp: NB padded rows plus 32 bytes of bookkeeping per child)
// First-K bound (output order: |U|, then the ascending column list): true
// when the child support (U with column k) comes after R, both of size |R|.
// Of two sets of equal size, the one holding the lowest column of their
// symmetric difference comes first.
__device__ __forceinline__ bool child_after(const uint64_t *pu, int k, const uint64_t *R, int W)
{
    for (int w = 0; w < W; ++w) {
        const uint64_t c = child_word(pu, w, k);
        const uint64_t d = c ^ __ldg(R + w);
        if (d) return (c & (d & (~d + 1))) == 0;
    }
    return false;
}

// Superset rule through the sentinel index (W <= 2): does a result E with
// k in E lie inside U + {k}?  Only the cells (k, s) with s in U are scanned:
// E's sentinel is one of its columns other than k, so E inside U + {k}
// requires the sentinel in U.
__device__ __forceinline__ bool pruned_indexed(const LevelArgs &a, const uint64_t *pu, int k, int W, int N)
{
    if (a.csingle[k]) return true;
    const uint64_t u0 = child_word(pu, 0, k), u1 = W == 2 ? child_word(pu, 1, k) : 0ull;
    for (int w = 0; w < W; ++w) {
        uint64_t m = __ldg(a.cne + (size_t)k * W + w) & (w == 0 ? u0 : u1);
        while (m) {
            const int sent = w * 64 + __ffsll((long long)m) - 1;
            m &= m - 1;
            const int32_t lo = __ldg(a.cptr + (size_t)k * N + sent), hi = __ldg(a.cptr + (size_t)k * N + sent + 1);
            for (int32_t e = lo; e < hi; ++e) {
                const uint64_t *E = a.cent + (size_t)e * W;
                const uint64_t e0 = __ldg(E), e1 = W == 2 ? __ldg(E + 1) : 0ull;
                if (((e0 & ~u0) | (e1 & ~u1)) == 0) return true;
            }
        }
    }
    return false;
}

template <int G, int CPL>
struct BatchShape {
    static constexpr int NCH = G * CPL;          // 16-byte chunks per row
    static constexpr int NB = NCH <= 16 ? 16 : (NCH <= 32 ? 8 : 2);
    static constexpr int ROW = NCH + 1;          // padded row (int4 units): conflict-free per-lane access
    static constexpr int BYTES = NB * ROW * 16 + NB * 32;
};

// One level of expansion by the warps worker = 0 .. nworkers-1 (the whole
// grid, or the warps of one CTA in the batched kernel).  bl: the static
// network (shared or global); wbase: this warp's batch region.
template <int G, int CPL>
__device__ void expand_range(const NetView &nv, const LevelArgs &a, const uint32_t *bl, char *wbase, int64_t worker,
                             int64_t nworkers)
{
    constexpr int NG = 32 / G;    // children per warp round
    constexpr int EPL = 4 * CPL;  // balance entries per lane
    using BS = BatchShape<G, CPL>;
    constexpr int NB = BS::NB;
    const int lane = threadIdx.x & 31;
    const int gi = lane / G;  // group in the warp
    const int gl = lane % G;  // lane in the group
    const int lead = gi * G;  // group leader lane
    const int W = nv.W;
    const int Mpad = nv.Mpad;
    // per-warp batch: rows, then (pos, tag, key, info, parent) per child
    int4 *brow = reinterpret_cast<int4 *>(wbase);
    uint64_t *bpos = reinterpret_cast<uint64_t *>(wbase + NB * BS::ROW * 16);
    uint32_t *btag = reinterpret_cast<uint32_t *>(bpos + NB);
    uint32_t *bkey = btag + NB;
    uint32_t *binfo = bkey + NB;  // k | in_u << 12 | pc1 << 13
    uint32_t *bpar = binfo + NB;  // parent index
    const int4 *dcol = reinterpret_cast<const int4 *>(bl + nv.o_dcols);

    unsigned long long n_exp = 0, n_ovf = 0, n_bal = 0, n_pruned = 0, deg_sum = 0;
    bool fatal = false;
    bool full = false;  // the child arena reached its capacity
    int nb = 0;         // children in the batch (warp-uniform)
    const uint64_t t_start = global_ns();

    // Phase 2 for wide rows (more than 32 chunks): the whole warp claims and
    // copies or compares one batched child at a time.
    auto flush_wide = [&]() {
        __syncwarp();
        for (int b = 0; b < nb; ++b) {
            const uint32_t info = binfo[b];
            const int k = (int)(info & 0xFFFu);
            const uint64_t *pu = a.par.U + (size_t)bpar[b] * W;
            if (full) continue;
            uint64_t pos = bpos[b];
            const uint32_t tag = btag[b];
            const int4 *row = brow + (size_t)b * BS::ROW;
            for (uint64_t probe = 0;; ++probe) {
                if (probe > a.slot_mask) {
                    if (lane == 0) atomicOr(&a.ctr[C_ERR], (unsigned long long)ERR_TABLE_FULL);
                    fatal = true;
                    break;
                }
                unsigned long long v = kEmpty;
                if (lane == 0) v = cas_acquire(&a.slots[pos], kEmpty, ((unsigned long long)tag << 32) | kPending);
                v = __shfl_sync(FULL, v, 0);
                if (v == kEmpty) {
                    unsigned long long idx = 0;
                    if (lane == 0) idx = atomicAdd(&a.ctr[C_NEXT], 1ull);
                    idx = __shfl_sync(FULL, idx, 0);
                    if ((int64_t)idx >= a.child.cap) {
                        full = true;
                        if (lane == 0) store_release(&a.slots[pos], ((unsigned long long)tag << 32) | kOverflowIdx);
                        break;
                    }
                    int4 *db = reinterpret_cast<int4 *>(a.child.B + (size_t)idx * Mpad);
                    for (int c = lane; c < BS::NCH; c += 32) db[c] = row[c];
                    uint64_t *du = a.child.U + (size_t)idx * W;
                    for (int w = lane; w < W; w += 32) du[w] = child_word(pu, w, k);
                    if (lane == 0) a.child.meta[idx] = pack_meta(bkey[b], (int)(info >> 13));
                    __threadfence();
                    __syncwarp();
                    if (lane == 0) {
                        store_release(&a.slots[pos], ((unsigned long long)tag << 32) | idx);
                        deg_sum += bkey[b] >> 16;
                    }
                    break;
                }
                if ((uint32_t)(v >> 32) != tag) {
                    pos = (pos + 1) & a.slot_mask;
                    continue;
                }
                int spins = 0;
                while ((uint32_t)v == kPending && spins < kSpinLimit) {
                    __nanosleep(64);
                    ++spins;
                    if (lane == 0) v = cas_acquire(&a.slots[pos], kEmpty, kEmpty);
                    v = __shfl_sync(FULL, v, 0);
                }
                if ((uint32_t)v == kPending) {
                    if (lane == 0) atomicOr(&a.ctr[C_ERR], (unsigned long long)ERR_TIMEOUT);
                    fatal = true;
                    break;
                }
                if ((uint32_t)v == kOverflowIdx) break;
                const uint32_t ci = (uint32_t)v;
                const int4 *sb = reinterpret_cast<const int4 *>(a.child.B + (size_t)ci * Mpad);
                bool eq = true;
                for (int c = lane; c < BS::NCH && eq; c += 32) {
                    const int4 x = __ldcg(sb + c), o = row[c];
                    eq = x.x == o.x && x.y == o.y && x.z == o.z && x.w == o.w;
                }
                const uint64_t *su = a.child.U + (size_t)ci * W;
                for (int w = lane; w < W && eq; w += 32) eq = __ldcg(su + w) == child_word(pu, w, k);
                if (__all_sync(FULL, eq)) break;  // duplicate of a state already in the frontier
                pos = (pos + 1) & a.slot_mask;
            }
            if (__any_sync(FULL, fatal)) break;
        }
        fatal = __any_sync(FULL, fatal);
        full = __any_sync(FULL, full);
        nb = 0;
        __syncwarp();
    };

    // Phase 2: insert the batched children, one lane each.
    auto flush = [&]() {
        if (BS::NCH > 32) {
            flush_wide();
            return;
        }
        __syncwarp();
        const bool mine = lane < nb;
        const uint32_t info = mine ? binfo[lane] : 0u;
        const int k = (int)(info & 0xFFFu);
        const uint64_t *pu = a.par.U + (size_t)(mine ? bpar[lane] : 0u) * W;
        bool todo = mine;
        if (full) todo = false;
        const uint64_t row_i = (uint64_t)lane * BS::ROW;
        uint64_t pos = mine ? bpos[lane] : 0ull;
        const uint32_t tag = mine ? btag[lane] : 0u;
        uint64_t probes = 0;
        int spins = 0, rounds = 0;
        while (__any_sync(FULL, todo)) {
            const bool expired = ++rounds > kMaxRounds || ((rounds & 63) == 0 && global_ns() - t_start > kWatchdogNs);
            if (__any_sync(FULL, expired)) {  // warp-uniform decision
                if (lane == 0) record_diag(a.ctr, ERR_WATCHDOG, 2, rounds, kMaxRounds, a.level);
                fatal = true;
                break;
            }
            unsigned long long v = kEmpty;
            if (todo) v = cas_acquire(&a.slots[pos], kEmpty, ((unsigned long long)tag << 32) | kPending);
            const bool won = todo && v == kEmpty;
            const bool other = todo && !won && (uint32_t)(v >> 32) != tag;
            const bool waiting = todo && !won && !other && (uint32_t)v == kPending;
            const bool over = todo && !won && !other && (uint32_t)v == kOverflowIdx;
            const bool cmp = todo && !won && !other && !waiting && !over;
            if (other) {
                pos = (pos + 1) & a.slot_mask;
                if (++probes > a.slot_mask) {
                    atomicOr(&a.ctr[C_ERR], (unsigned long long)ERR_TABLE_FULL);
                    todo = false;
                    fatal = true;
                }
            }
            if (over) todo = false;
            const unsigned wmask = __ballot_sync(FULL, won);
            if (wmask) {
                const int leader = __ffs((int)wmask) - 1;
                unsigned long long base_idx = 0;
                if (lane == leader) base_idx = atomicAdd(&a.ctr[C_NEXT], (unsigned long long)__popc(wmask));
                base_idx = __shfl_sync(FULL, base_idx, leader);
                const uint64_t idx = base_idx + (uint64_t)__popc(wmask & ((1u << lane) - 1u));
                bool wrote = false;
                if (won) {
                    if ((int64_t)idx >= a.child.cap) {
                        full = true;  // level truncated: stop claiming
                        store_release(&a.slots[pos], ((unsigned long long)tag << 32) | kOverflowIdx);
                    } else {
                        int4 *db = reinterpret_cast<int4 *>(a.child.B + (size_t)idx * Mpad);
                        for (int c = 0; c < BS::NCH; ++c) db[c] = brow[row_i + c];
                        uint64_t *du = a.child.U + (size_t)idx * W;
                        for (int w = 0; w < W; ++w) du[w] = child_word(pu, w, k);
                        a.child.meta[idx] = pack_meta(bkey[lane], (int)(info >> 13));
                        wrote = true;
                    }
                    todo = false;
                }
                __threadfence_block();  // order each lane's row writes before its release store
                if (wrote) {
                    store_release(&a.slots[pos], ((unsigned long long)tag << 32) | idx);
                    deg_sum += bkey[lane] >> 16;
                }
            }
            if (cmp) {
                const uint32_t ci = (uint32_t)v;
                const int4 *sb = reinterpret_cast<const int4 *>(a.child.B + (size_t)ci * Mpad);
                bool eq = true;
                for (int c = 0; c < BS::NCH && eq; ++c) {
                    const int4 s = __ldcg(sb + c);
                    const int4 o = brow[row_i + c];
                    eq = s.x == o.x && s.y == o.y && s.z == o.z && s.w == o.w;
                }
                const uint64_t *su = a.child.U + (size_t)ci * W;
                for (int w = 0; w < W && eq; ++w) eq = __ldcg(su + w) == child_word(pu, w, k);
                if (eq) {
                    todo = false;  // duplicate of a state already in the frontier
                } else {
                    pos = (pos + 1) & a.slot_mask;
                    ++probes;
                }
            }
            if (__any_sync(FULL, waiting)) {
                if (waiting && ++spins > kSpinLimit) {
                    atomicOr(&a.ctr[C_ERR], (unsigned long long)ERR_TIMEOUT);
                    todo = false;
                    fatal = true;
                }
                __nanosleep(32);
            }
            full = __any_sync(FULL, full);
            if (full) todo = false;
        }
        nb = 0;
        __syncwarp();
    };

    // chunks of cpw parents per warp (fewer for small levels, so that the
    // items of a small level spread over all warps)
    const int cpw = a.cpw;
    const int64_t wstride = nworkers * cpw;
    for (int64_t p0 = worker * cpw; p0 < a.n_par; p0 += wstride) {
        const int64_t pl = p0 + lane;
        const bool pin = lane < cpw && pl < a.n_par;
        const int64_t pid = pin ? (a.perm ? (int64_t)a.perm[pl] : pl) : 0;  // this lane's parent
        // pull this chunk's and the next chunk's parents toward L2
        if (pin) {
            const char *rp = reinterpret_cast<const char *>(a.par.B + (size_t)pid * Mpad);
            for (int off = 0; off < Mpad * 4; off += 128) prefetch_l2(rp + off);
            prefetch_l2(a.par.U + (size_t)pid * W);
        }
        const int64_t pn = pl + wstride;
        if (lane < cpw && pn < a.n_par) {
            const int64_t nid = a.perm ? (int64_t)a.perm[pn] : pn;
            const char *rp = reinterpret_cast<const char *>(a.par.B + (size_t)nid * Mpad);
            for (int off = 0; off < Mpad * 4; off += 128) prefetch_l2(rp + off);
            prefetch_l2(a.par.U + (size_t)nid * W);
            prefetch_l2(a.par.meta + nid);
        }
        const uint32_t mj = pin ? a.par.meta[pid] : 0u;
        int dj = pin ? (int)((mj >> 10) & 0x1FFFu) : 0;
        // first-K: a parent larger than the bound has no descendant among the K smallest
        if (a.fk_pc > 0 && (int)((mj >> 23) & 0x7Fu) > a.fk_pc) dj = 0;
        int incl = dj;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int x = __shfl_up_sync(FULL, incl, off);
            if (lane >= off) incl += x;
        }
        const int prej = incl - dj;
        const int T = __shfl_sync(FULL, incl, 31);
        if (T > 32 * nv.N) {
            if (lane == 0) record_diag(a.ctr, ERR_BOUNDS, 3, T, 32 * nv.N, a.level);
            fatal = true;
        }
        for (int base = 0; base < T; base += 32) {
            if (__any_sync(FULL, fatal)) break;
            // --- branch selection: one (parent, branch) item per lane ---
            const int c = base + lane;
            int j = 0;  // largest j with pre_j <= c
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int v = __shfl_sync(FULL, prej, j + step);
                if (v <= c) j += step;
            }
            const uint32_t pm = __shfl_sync(FULL, mj, j);
            const int q = c - __shfl_sync(FULL, prej, j);
            const int64_t pl_ = __shfl_sync(FULL, pid, j);
            bool okl = c < T;
            int kl = 0, pcl = 0;
            bool inl = false;
            int32_t Al = 0, Cl = 0;
            if (okl) {
                const int32_t *prow_l = a.par.B + (size_t)pl_ * Mpad;
                const uint64_t *pu_l = a.par.U + (size_t)pl_ * W;
                const int piv = (int)(pm & 0x3FFu);
                pcl = (int)((pm >> 23) & 0x7Fu);
                const int32_t bi = piv < nv.M ? prow_l[piv] : 0;
                const bool fwd = bi > 0;  // forward flow: consume the surplus
                const uint32_t abi = (uint32_t)(bi < 0 ? -bi : bi);
                const int lptr = (fwd ? nv.o_consptr : nv.o_prodptr) + (piv < nv.M ? piv : 0);
                const int lb = (int)bl[lptr];
                const int le = (int)bl[lptr + 1];
                if (piv >= nv.M || bi == 0 || lb + q >= le) {
                    record_diag(a.ctr, ERR_BOUNDS, 1 + (piv >= nv.M ? 10 : 0) + (bi == 0 ? 100 : 0), (long long)q,
                                (long long)(le - lb), a.level);
                    fatal = true;
                    okl = false;
                } else {
                    const uint32_t br = bl[(fwd ? nv.o_consent : nv.o_prodent) + lb + q];
                    kl = ent_index(br);
                    const uint32_t sik = (uint32_t)ent_coef(br);  // |S_ik|
                    const int tw = (int)bl[nv.o_twin + kl];
                    inl = bit_of(pu_l, kl);
                    const int sec = a.level - pcl;
                    okl = !(tw >= 0 && bit_of(pu_l, tw)) && (inl ? sec + 1 <= a.max_sec : pcl + 1 <= a.max_len);
                    if (okl && a.fk_pc > 0) {
                        // first-K branch and bound: the child's descendants keep
                        // its support or grow it, so a child past the K-th
                        // result found so far cannot yield one of the K smallest
                        const int pc2 = pcl + (inl ? 0 : 1);
                        okl = pc2 < a.fk_pc || (pc2 == a.fk_pc && !child_after(pu_l, kl, a.fk_sup, W));
                    }
                    const uint32_t g0 = (abi == 1u || sik == 1u) ? 1u : gcd32(abi, sik);
                    Al = (int32_t)(sik / g0);
                    Cl = (int32_t)(abi / g0);
                }
            }
            if (okl) ++n_exp;
            // packed item: column | |U| << 12 | secondary << 19; parent as 32 bits
            const uint32_t infol = (uint32_t)kl | ((uint32_t)pcl << 12) | (inl ? 1u << 19 : 0u);
            const uint32_t pl32 = (uint32_t)pl_;
            // the groups take the valid items of this pass NG at a time, in order
            unsigned vmask = __ballot_sync(FULL, okl);
            while (vmask) {
                if (__any_sync(FULL, fatal)) break;
                const int src = gi < __popc(vmask) ? (int)__fns(vmask, 0, gi + 1) : -1;
#pragma unroll
                for (int t = 0; t < NG; ++t) vmask &= vmask - 1;
                const int sl = src < 0 ? 0 : src;
                const bool ok = src >= 0;
                const uint32_t info_i = __shfl_sync(FULL, infol, sl);
                const int k = (int)(info_i & 0xFFFu);
                const int pc = (int)((info_i >> 12) & 0x7Fu);
                const bool in_u = (info_i >> 19) & 1u;
                const int32_t A = __shfl_sync(FULL, Al, sl);
                const int32_t C = __shfl_sync(FULL, Cl, sl);
                const int64_t p = (int64_t)__shfl_sync(FULL, pl32, sl);
                const int32_t *prow = a.par.B + (size_t)p * Mpad;
                const uint64_t *pu = a.par.U + (size_t)p * W;

                // --- AND update (Eq. 3 / Eq. 4 in integers), group-parallel ---
                int32_t t32[EPL];
                uint32_t fl = 0;  // bit0 nonzero, bit1 some |t| == 1, bit2 some t outside int32
                const int4 *prow4 = reinterpret_cast<const int4 *>(prow);
                const int4 *col4 = dcol + (size_t)k * (Mpad >> 2);
                if (ok) {
    #pragma unroll
                    for (int i = 0; i < CPL; ++i) {
                        const int4 v = prow4[gl + G * i];
                        const int4 w = col4[gl + G * i];
                        const int32_t pv[4] = {v.x, v.y, v.z, v.w}, cv[4] = {w.x, w.y, w.z, w.w};
    #pragma unroll
                        for (int jj = 0; jj < 4; ++jj) {
                            const int64_t tt = (int64_t)A * pv[jj] + (int64_t)C * cv[jj];
                            const int32_t lo = (int32_t)tt;
                            const bool fits = tt == (int64_t)lo && lo != INT32_MIN;
                            t32[4 * i + jj] = lo;
                            fl |= (tt != 0 ? 1u : 0u) | ((lo == 1 || lo == -1) ? 2u : 0u) | (fits ? 0u : 4u);
                        }
                    }
                } else {
    #pragma unroll
                    for (int e = 0; e < EPL; ++e) t32[e] = 0;
                }
                fl = group_or<G>(fl);
                const bool nz = fl & 1u;
                // slow path: the gcd is needed (no unit entry), or an entry is
                // outside int32 (then the raw entries are recomputed in 64 bits)
                const bool slow = ok && nz && ((fl & 6u) != 2u);
                const bool big = (fl & 4u) != 0u;
                bool ovf = false;
                if (__any_sync(FULL, slow)) {
                    uint64_t gg = 0, amax = 0;
                    if (slow && !big) {
    #pragma unroll
                        for (int e = 0; e < EPL; ++e) {
                            const uint32_t at = (uint32_t)(t32[e] < 0 ? -t32[e] : t32[e]);
                            if (at != 0) gg = gg == 0 ? at : gcd32((uint32_t)gg, at);
                        }
                    } else if (slow) {
                        const GcdMax gm = raw_gcd_max(prow4, col4, gl, G, CPL, A, C);
                        gg = gm.g;
                        amax = gm.m;
                    }
    #pragma unroll
                    for (int off = G / 2; off > 0; off >>= 1) {
                        const uint64_t og = __shfl_xor_sync(FULL, gg, off);
                        gg = og == 0 ? gg : (gg == 0 ? og : gcd64(gg, og));
                        const uint64_t y = __shfl_xor_sync(FULL, amax, off);
                        amax = y > amax ? y : amax;
                    }
                    if (slow) {
                        ovf = big && amax / gg > 2147483647ull;
                        if (!ovf && gg > 1) {
                            const bool pow2 = (gg & (gg - 1)) == 0;
                            const int sh = __ffsll((long long)gg) - 1;
                            if (!big) {
    #pragma unroll
                                for (int e = 0; e < EPL; ++e)
                                    t32[e] = t32[e] == 0 ? 0 : (pow2 ? (t32[e] >> sh) : t32[e] / (int32_t)gg);
                            } else {
    #pragma unroll
                                for (int i = 0; i < CPL; ++i) {
                                    const int4 v = prow4[gl + G * i];
                                    const int4 w = col4[gl + G * i];
                                    const int32_t pv[4] = {v.x, v.y, v.z, v.w}, cv[4] = {w.x, w.y, w.z, w.w};
    #pragma unroll
                                    for (int jj = 0; jj < 4; ++jj) {
                                        const int64_t tt = (int64_t)A * pv[jj] + (int64_t)C * cv[jj];
                                        t32[4 * i + jj] = (int32_t)(tt / (int64_t)gg);
                                    }
                                }
                            }
                        }
                    }
                }
                const bool bal = ok && !nz;
                const bool grown = ok && nz && !ovf;
                if (ovf && gl == 0) ++n_ovf;
                if (bal && gl == 0) {
                    ++n_bal;  // all metabolites stable: to the arbiter
                    if (insert_support(a, W, pu, k) < INS_DUP) fatal = true;
                }
                fatal = group_or<G>(fatal ? 1u : 0u) != 0;
                // superset pruning (counted on a truncated level too): the new
                // column k completes a result accepted at an earlier level.  The
                // G lanes of the group split the results containing k.
                bool pr = false;
                if (grown && !in_u) {
                    const int64_t b1 = a.bptr[k];
                    const int64_t n = a.bptr[k + 1] - b1;
                    if (W <= 2) {
                        const uint64_t u0 = child_word(pu, 0, k), u1 = W == 2 ? child_word(pu, 1, k) : 0ull;
                        // every result containing k holds their intersection: if the
                        // child lacks part of it, none of them lies inside the child
                        bool maybe = true;
                        if (a.band) {
                            const uint64_t i0 = __ldg(a.band + (size_t)k * W), i1 = W == 2 ? __ldg(a.band + (size_t)k * W + 1) : 0ull;
                            maybe = ((i0 & ~u0) | (i1 & ~u1)) == 0;
                        }
                        for (int64_t i = gl; i < n && !pr && maybe; i += G) {
                            const uint64_t *E = a.bres + (size_t)(b1 + i) * W;
                            const uint64_t e0 = __ldg(E), e1 = W == 2 ? __ldg(E + 1) : 0ull;
                            pr = ((e0 & ~u0) | (e1 & ~u1)) == 0;
                        }
                    } else {
                        for (int64_t i = gl; i < n && !pr; i += G) pr = result_inside_wide(a, pu, k, b1 + i);
                    }
                }
                pr = group_or<G>(pr ? 1u : 0u) != 0;
                if (pr && gl == 0) ++n_pruned;
                const bool norm = grown && !pr;

                // --- pivot key and fingerprint, then append to the batch ---
                uint32_t key = 0xFFFFFFFFu, hlo = 0, hhi = 0;
                if (norm) {
    #pragma unroll
                    for (int i = 0; i < CPL; ++i)
    #pragma unroll
                        for (int jj = 0; jj < 4; ++jj) {
                            const int m = 4 * (gl + G * i) + jj;
                            const int32_t v = t32[4 * i + jj];
                            if (v != 0) {
                                const uint32_t kk = bl[(v > 0 ? nv.o_keypos : nv.o_keyneg) + m];
                                key = kk < key ? kk : key;
                            }
                            hash_entry((uint32_t)m, (uint32_t)v, hlo, hhi);
                        }
                    for (int w = gl; w < W; w += G) {
                        const uint64_t x = mix64(child_word(pu, w, k) ^ (0x2545f4914f6cdd1dull * (uint64_t)(w + 1)));
                        hlo += (uint32_t)x;
                        hhi ^= (uint32_t)(x >> 32);
                    }
                }
                key = group_min<G>(key);
                hlo = group_add<G>(hlo);
                hhi = group_xor<G>(hhi);
                const unsigned nm = __ballot_sync(FULL, norm && gl == 0);
                if (norm) {
                    const int slot = nb + __popc(nm & ((1u << lead) - 1u));
                    int4 *r = brow + (size_t)slot * BS::ROW;
    #pragma unroll
                    for (int i = 0; i < CPL; ++i)
                        r[gl + G * i] = make_int4(t32[4 * i + 0], t32[4 * i + 1], t32[4 * i + 2], t32[4 * i + 3]);
                    if (gl == 0) {
                        uint64_t pos;
                        uint32_t tag;
                        slot_tag_pos(((uint64_t)hhi << 32) | hlo, a.slot_mask, pos, tag);
                        prefetch_l2(&a.slots[pos]);
                        bpos[slot] = pos;
                        btag[slot] = tag;
                        bkey[slot] = key;
                        binfo[slot] = (uint32_t)k | (in_u ? 1u << 12 : 0u) | ((uint32_t)(pc + (in_u ? 0 : 1)) << 13);
                        bpar[slot] = (uint32_t)p;
                    }
                }
                nb += __popc(nm);
                if (nb > NB - NG) flush();

            }
        }
        if (__any_sync(FULL, fatal)) break;
    }
    if (nb > 0 && !__any_sync(FULL, fatal)) flush();
    if (n_exp) atomicAdd(&a.ctr[C_EXP], n_exp);
    if (n_ovf) atomicAdd(&a.ctr[C_OVF], n_ovf);
    if (n_bal) atomicAdd(&a.ctr[C_BAL], n_bal);
    if (n_pruned) atomicAdd(&a.ctr[C_PRUNED], n_pruned);
    if (deg_sum) atomicAdd(&a.ctr[C_DEGSUM], deg_sum);
}


// ---------------------------------------------------------------------------
// a1-a5 as two passes (single-job traversal): generate, then deduplicate.
//
// Generate: the same per-item work as phase 1 above (branch selection, AND
// update, balance test, superset rule, pivot key, fingerprint), but every
// surviving unbalanced child is written straight from registers to a row of
// the child arena that its warp reserved in advance (rows are reserved blk
// at a time with one atomic), together with its 64-bit fingerprint.  Nothing
// waits on another child: no hash-table probe, no publish/compare protocol.
// Children whose reserved row lies past the arena's capacity keep only their
// fingerprint (the level is then decided from fingerprints, or run again
// with a larger arena).
//
// Dedup: one thread per reserved row inserts (tag, row) into the level's
// hash table with a plain CAS.  Every row was written by the previous
// launch, so a tag match is settled at once by comparing the two rows; the
// first row of every distinct (U, EF) survives and is appended to the live
// list, which the next level reads its parents through.
// ---------------------------------------------------------------------------

template <int G, int CPL>
__device__ void generate_range(const NetView &nv, const LevelArgs &a, const uint32_t *bl, const uint32_t *blg,
                               int64_t worker,
                               int64_t nworkers)
{
    constexpr int NG = 32 / G;    // children per warp round
    constexpr int EPL = 4 * CPL;  // balance entries per lane
    const int lane = threadIdx.x & 31;
    const int gi = lane / G;  // group in the warp
    const int gl = lane % G;  // lane in the group
    const int lead = gi * G;  // group leader lane
    const int W = nv.W;
    const int Mpad = nv.Mpad;
    // bl: the static network (its sparse tables possibly in shared memory);
    // blg: the same words, for the dense columns and the first-K tables
    const int4 *dcol = reinterpret_cast<const int4 *>(blg + nv.o_dcols);
    const int64_t row_cap = a.child.cap;

    unsigned long long n_exp = 0, n_ovf = 0, n_bal = 0, n_pruned = 0, n_unwritten = 0, n_zero = 0, n_capdead = 0;
    bool fatal = false;
    // this warp's reserved rows: [pool_next, pool_next + pool_left)
    uint64_t pool_next = 0;
    int pool_left = 0;

    const int cpw = a.cpw;
    const int64_t wstride = nworkers * cpw;
    for (int64_t p0 = worker * cpw; p0 < a.n_par; p0 += wstride) {
        const int64_t pl = p0 + lane;
        const bool pin = lane < cpw && pl < a.n_par;
        const int64_t pid = pin ? (a.perm ? (int64_t)a.perm[pl] : a.par_base + pl) : 0;  // this lane's parent
        const int64_t pn = pl + wstride;
        if (lane < cpw && pn < a.n_par) {
            const int64_t nid = a.perm ? (int64_t)a.perm[pn] : a.par_base + pn;
            const char *rp = reinterpret_cast<const char *>(a.par.B + (size_t)nid * Mpad);
            for (int off = 0; off < Mpad * 4; off += 128) prefetch_l2(rp + off);
            prefetch_l2(a.par.U + (size_t)nid * W);
            prefetch_l2(a.par.meta + nid);
        }
        const uint32_t mj = pin ? a.par.meta[pid] : 0u;
        int dj = pin ? (int)((mj >> 10) & 0x1FFFu) : 0;
        // first-K: a parent larger than the bound has no descendant among the K smallest
        if (a.fk_pc > 0 && (int)((mj >> 23) & 0x7Fu) > a.fk_pc) dj = 0;
        int incl = dj;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int x = __shfl_up_sync(FULL, incl, off);
            if (lane >= off) incl += x;
        }
        const int prej = incl - dj;
        const int T = __shfl_sync(FULL, incl, 31);
        if (T > 32 * nv.N) {
            if (lane == 0) record_diag(a.ctr, ERR_BOUNDS, 3, T, 32 * nv.N, a.level);
            fatal = true;
        }
        for (int base = 0; base < T; base += 32) {
            if (__any_sync(FULL, fatal)) break;
            // --- branch selection: one (parent, branch) item per lane ---
            const int c = base + lane;
            int j = 0;  // largest j with pre_j <= c
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int v = __shfl_sync(FULL, prej, j + step);
                if (v <= c) j += step;
            }
            const uint32_t pm = __shfl_sync(FULL, mj, j);
            const int q = c - __shfl_sync(FULL, prej, j);
            const int64_t pl_ = __shfl_sync(FULL, pid, j);
            bool okl = c < T;
            int kl = 0, pcl = 0;
            bool inl = false, subl = false;
            int32_t Al = 0, Cl = 0;
            if (okl) {
                const int32_t *prow_l = a.par.B + (size_t)pl_ * Mpad;
                const uint64_t *pu_l = a.par.U + (size_t)pl_ * W;
                const int piv = (int)(pm & 0x3FFu);
                pcl = (int)((pm >> 23) & 0x7Fu);
                const int32_t bi = piv < nv.M ? prow_l[piv] : 0;
                const bool fwd = bi > 0;  // forward flow: consume the surplus
                const uint32_t abi = (uint32_t)(bi < 0 ? -bi : bi);
                const int pv_ = piv < nv.M ? piv : 0;
                const int lptr = (fwd ? nv.o_consptr : nv.o_prodptr) + pv_;
                const int lb = (int)bl[lptr];
                const int le = (int)bl[lptr + 1];
                // subtractive variant: after the side list, the opposite list
                // (Eq. 5: less flux on a column of U that moves i the same way)
                const int optr = (fwd ? nv.o_prodptr : nv.o_consptr) + pv_;
                const int on = a.sub ? (int)bl[optr + 1] - (int)bl[optr] : 0;
                if (piv >= nv.M || bi == 0 || q >= (le - lb) + on) {
                    record_diag(a.ctr, ERR_BOUNDS, 1 + (piv >= nv.M ? 10 : 0) + (bi == 0 ? 100 : 0), (long long)q,
                                (long long)(le - lb + on), a.level);
                    fatal = true;
                    okl = false;
                } else if (q >= le - lb) {
                    const uint32_t br = bl[(fwd ? nv.o_prodent : nv.o_consent) + (int)bl[optr] + (q - (le - lb))];
                    kl = ent_index(br);
                    const uint32_t sik = (uint32_t)ent_coef(br);  // |S_ik|
                    inl = bit_of(pu_l, kl);
                    okl = inl && (a.level - pcl) + 1 <= a.max_sec;
                    subl = true;
                    const uint32_t g0 = (abi == 1u || sik == 1u) ? 1u : gcd32(abi, sik);
                    Al = (int32_t)(sik / g0);
                    Cl = (int32_t)(abi / g0);
                } else {
                    const uint32_t br = bl[(fwd ? nv.o_consent : nv.o_prodent) + lb + q];
                    kl = ent_index(br);
                    const uint32_t sik = (uint32_t)ent_coef(br);  // |S_ik|
                    const int tw = (int)bl[nv.o_twin + kl];
                    inl = bit_of(pu_l, kl);
                    const int sec = a.level - pcl;
                    okl = !(tw >= 0 && bit_of(pu_l, tw)) && (inl ? sec + 1 <= a.max_sec : pcl + 1 <= a.max_len);
                    if (okl && a.fk_pc > 0) {
                        const int pc2 = pcl + (inl ? 0 : 1);
                        okl = pc2 < a.fk_pc || (pc2 == a.fk_pc && !child_after(pu_l, kl, a.fk_sup, W));
                    }
                    const uint32_t g0 = (abi == 1u || sik == 1u) ? 1u : gcd32(abi, sik);
                    Al = (int32_t)(sik / g0);
                    Cl = (int32_t)(abi / g0);
                }
            }
            if (okl) ++n_exp;
            const uint32_t infol = (uint32_t)kl | ((uint32_t)pcl << 12) | (inl ? 1u << 19 : 0u) | (subl ? 1u << 20 : 0u);
            const uint32_t pl32 = (uint32_t)pl_;
            // the groups take the valid items of this pass NG at a time, in order
            unsigned vmask = __ballot_sync(FULL, okl);
            while (vmask) {
                if (__any_sync(FULL, fatal)) break;
                const int src = gi < __popc(vmask) ? (int)__fns(vmask, 0, gi + 1) : -1;
#pragma unroll
                for (int t = 0; t < NG; ++t) vmask &= vmask - 1;
                const int sl = src < 0 ? 0 : src;
                const bool ok = src >= 0;
                const uint32_t info_i = __shfl_sync(FULL, infol, sl);
                const int k = (int)(info_i & 0xFFFu);
                const int pc = (int)((info_i >> 12) & 0x7Fu);
                const bool in_u = (info_i >> 19) & 1u;
                const bool subi = (info_i >> 20) & 1u;  // Eq. 5: flux taken away from k
                const int32_t A = __shfl_sync(FULL, Al, sl);
                const int32_t C0 = __shfl_sync(FULL, Cl, sl);
                const int32_t C = subi ? -C0 : C0;
                const int64_t p = (int64_t)__shfl_sync(FULL, pl32, sl);
                const int32_t *prow = a.par.B + (size_t)p * Mpad;
                const uint64_t *pu = a.par.U + (size_t)p * W;
                // Prop. 3: a subtractive step must leave k with positive flux
                // (the flux of column k sits at row M + k)
                bool zflux = false;
                if (ok && subi) zflux = (int64_t)A * prow[nv.M + k] - (int64_t)C0 <= 0;

                // --- AND update (Eq. 3 / Eq. 4 in integers), group-parallel ---
                int32_t t32[EPL];
                uint32_t fl = 0;  // bit0 nonzero, bit1 some |t| == 1, bit2 some t outside int32
                const int4 *prow4 = reinterpret_cast<const int4 *>(prow);
                const int4 *col4 = dcol + (size_t)k * (Mpad >> 2);
                if (ok) {
#pragma unroll
                    for (int i = 0; i < CPL; ++i) {
                        const int4 v = prow4[gl + G * i];
                        const int4 w = col4[gl + G * i];
                        const int32_t pv[4] = {v.x, v.y, v.z, v.w}, cv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) {
                            const int64_t tt = (int64_t)A * pv[jj] + (int64_t)C * cv[jj];
                            const int32_t lo = (int32_t)tt;
                            const bool fits = tt == (int64_t)lo && lo != INT32_MIN;
                            t32[4 * i + jj] = lo;
                            // bit0: a balance row (m < M; the rest is flux or padding) is nonzero
                            const bool brow = 4 * (gl + G * i) + jj < nv.M;
                            fl |= ((tt != 0 && brow) ? 1u : 0u) | ((lo == 1 || lo == -1) ? 2u : 0u) | (fits ? 0u : 4u);
                        }
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < EPL; ++e) t32[e] = 0;
                }
                fl = group_or<G>(fl);
                const bool nz = fl & 1u;
                // slow path: the gcd is needed (no unit entry), or an entry is
                // outside int32 (then the raw entries are recomputed in 64 bits)
                const bool slow = ok && !zflux && nz && ((fl & 6u) != 2u);
                const bool big = (fl & 4u) != 0u;
                bool ovf = false;
                if (__any_sync(FULL, slow)) {
                    uint64_t gg = 0, amax = 0;
                    if (slow && !big) {
#pragma unroll
                        for (int e = 0; e < EPL; ++e) {
                            const uint32_t at = (uint32_t)(t32[e] < 0 ? -t32[e] : t32[e]);
                            if (at != 0) gg = gg == 0 ? at : gcd32((uint32_t)gg, at);
                        }
                    } else if (slow) {
                        const GcdMax gm = raw_gcd_max(prow4, col4, gl, G, CPL, A, C);
                        gg = gm.g;
                        amax = gm.m;
                    }
#pragma unroll
                    for (int off = G / 2; off > 0; off >>= 1) {
                        const uint64_t og = __shfl_xor_sync(FULL, gg, off);
                        gg = og == 0 ? gg : (gg == 0 ? og : gcd64(gg, og));
                        const uint64_t y = __shfl_xor_sync(FULL, amax, off);
                        amax = y > amax ? y : amax;
                    }
                    if (slow) {
                        ovf = big && amax / gg > 2147483647ull;
                        if (!ovf && gg > 1) {
                            const bool pow2 = (gg & (gg - 1)) == 0;
                            const int sh = __ffsll((long long)gg) - 1;
                            if (!big) {
#pragma unroll
                                for (int e = 0; e < EPL; ++e)
                                    t32[e] = t32[e] == 0 ? 0 : (pow2 ? (t32[e] >> sh) : t32[e] / (int32_t)gg);
                            } else {
#pragma unroll
                                for (int i = 0; i < CPL; ++i) {
                                    const int4 v = prow4[gl + G * i];
                                    const int4 w = col4[gl + G * i];
                                    const int32_t pv[4] = {v.x, v.y, v.z, v.w}, cv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                                    for (int jj = 0; jj < 4; ++jj) {
                                        const int64_t tt = (int64_t)A * pv[jj] + (int64_t)C * cv[jj];
                                        t32[4 * i + jj] = (int32_t)(tt / (int64_t)gg);
                                    }
                                }
                            }
                        }
                    }
                }
                if (zflux && gl == 0) ++n_zero;
                const bool bal = ok && !zflux && !nz;
                const bool grown = ok && !zflux && nz && !ovf;
                if (ovf && !zflux && gl == 0) ++n_ovf;
                if (bal && gl == 0) {
                    ++n_bal;  // all metabolites stable: to the arbiter
                    if (insert_support(a, W, pu, k) < INS_DUP) fatal = true;
                }
                fatal = group_or<G>(fatal ? 1u : 0u) != 0;
                // superset rule: the new column k completes a result accepted
                // at an earlier level (the group's lanes split its bucket)
                bool pr = false;
                if (grown && !in_u) {
                    const int64_t b1 = a.bptr[k];
                    const int64_t n = a.bptr[k + 1] - b1;
                    if (W <= 2 && a.cptr) {
                        if (gl == 0) pr = pruned_indexed(a, pu, k, W, nv.N);
                    } else if (W <= 2) {
                        const uint64_t u0 = child_word(pu, 0, k), u1 = W == 2 ? child_word(pu, 1, k) : 0ull;
                        bool maybe = n > 0;
                        if (maybe && a.band) {
                            const uint64_t i0 = __ldg(a.band + (size_t)k * W), i1 = W == 2 ? __ldg(a.band + (size_t)k * W + 1) : 0ull;
                            maybe = ((i0 & ~u0) | (i1 & ~u1)) == 0;
                        }
                        for (int64_t i = gl; i < n && !pr && maybe; i += G) {
                            const uint64_t *E = a.bres + (size_t)(b1 + i) * W;
                            const uint64_t e0 = __ldg(E), e1 = W == 2 ? __ldg(E + 1) : 0ull;
                            pr = ((e0 & ~u0) | (e1 & ~u1)) == 0;
                        }
                    } else {
                        for (int64_t i = gl; i < n && !pr; i += G) pr = result_inside_wide(a, pu, k, b1 + i);
                    }
                }
                pr = group_or<G>(pr ? 1u : 0u) != 0;
                if (pr && gl == 0) ++n_pruned;
                bool norm = grown && !pr;
                // first-K: the lane masks of the rows the child's support
                // consumes and produces (the parent's, plus column k's)
                uint32_t fxc = 0, fxp = 0;
                if (a.child.fx && norm) {
                    const size_t fo = (size_t)p * (2 * G);
                    fxc = a.par.fx[fo + gl] | blg[nv.o_fixc + k * G + gl];
                    fxp = a.par.fx[fo + G + gl] | blg[nv.o_fixp + k * G + gl];
                }
                // first-K at the length cap: the child can only take secondary
                // steps, which add flux to columns of its support.  A row with a
                // surplus (deficit) that no column of the support consumes
                // (produces) keeps its sign under every such step, so the child
                // never balances; with no secondary step left it cannot move.
                if (a.cap_dead && __any_sync(FULL, norm && pc + (in_u ? 0 : 1) >= a.max_len)) {
                    bool dead = false;
                    const int pcc = pc + (in_u ? 0 : 1);
                    if (norm && pcc >= a.max_len) {
                        if (a.level - pcc + 1 >= a.max_sec) {
                            dead = true;
                        } else if (a.child.fx) {
#pragma unroll
                            for (int i = 0; i < CPL; ++i)
#pragma unroll
                                for (int jj = 0; jj < 4; ++jj) {
                                    const int32_t v = t32[4 * i + jj];
                                    const uint32_t fix = v > 0 ? fxc : fxp;
                                    if (v != 0 && 4 * (gl + G * i) + jj < nv.M && !((fix >> (4 * i + jj)) & 1u))
                                        dead = true;
                                }
                        }
                    }
                    dead = group_or<G>(dead ? 1u : 0u) != 0;
                    if (dead && gl == 0) ++n_capdead;
                    norm = norm && !dead;
                }

                // first-K one below the cap: the child's results have support U
                // or U + {c} for one more column c.  Balance needs both signs in
                // every row a support touches, and a row that U touches with one
                // sign only (a surplus with no consumer, a deficit with no
                // producer in U) is a row EF keeps nonzero under secondary
                // steps.  With such rows, some column c must give each of them
                // the missing sign and find the opposite sign in U for every
                // row of its own (twin rule kept); the group tries the columns
                // able to fix the one-sided row with the shortest fixer list.
                if (a.cap_dead && a.child.fx && __any_sync(FULL, norm && pc + (in_u ? 0 : 1) == a.max_len - 1)) {
                    const bool mine = norm && pc + (in_u ? 0 : 1) == a.max_len - 1;
                    uint32_t dl = 0;            // this lane's one-sided rows, bits as in fxc / fxp
                    uint32_t pick = 0xFFFFFFFFu;  // list length << 20 | surplus << 19 | row
                    if (mine) {
#pragma unroll
                        for (int i = 0; i < CPL; ++i)
#pragma unroll
                            for (int jj = 0; jj < 4; ++jj) {
                                const int r = 4 * (gl + G * i) + jj;
                                const int32_t v = t32[4 * i + jj];
                                const uint32_t fix = v > 0 ? fxc : fxp;
                                if (v != 0 && r < nv.M && !((fix >> (4 * i + jj)) & 1u)) {
                                    dl |= 1u << (4 * i + jj);
                                    const int lp = (v > 0 ? nv.o_consptr : nv.o_prodptr) + r;
                                    const uint32_t len = min(bl[lp + 1] - bl[lp], 4095u);
                                    const uint32_t cand = (len << 20) | (v > 0 ? 1u << 19 : 0u) | (uint32_t)r;
                                    pick = cand < pick ? cand : pick;
                                }
                            }
                    }
                    const uint32_t nd = group_add<G>((uint32_t)__popc(dl));
                    pick = group_min<G>(pick);
                    bool open = mine && nd > 0;  // still looking for a completing column
                    const int r0 = (int)(pick & 0x7FFFFu);
                    const bool sur0 = (pick >> 19) & 1u;
                    const int lp0 = open ? (sur0 ? nv.o_consptr : nv.o_prodptr) + r0 : 0;
                    const int b0 = open ? (int)bl[lp0] : 0;
                    const int n0 = open ? (int)bl[lp0 + 1] - b0 : 0;
                    const int eo0 = sur0 ? nv.o_consent : nv.o_prodent;
                    bool found = false;
                    for (int c0 = 0; __any_sync(FULL, open && c0 < n0); c0 += G) {
                        const bool act = open && c0 < n0;
                        const int ci = c0 + gl;
                        int kc = -1;
                        if (act && ci < n0) kc = ent_index(bl[eo0 + b0 + ci]);
                        bool ok2 = kc >= 0;
                        if (ok2) {
                            const int tw = (int)bl[nv.o_twin + kc];
                            ok2 = !(tw >= 0 && (tw == k || ((pu[tw >> 6] >> (tw & 63)) & 1ull)));
                        }
                        const int cb = ok2 ? (int)blg[nv.o_colptr + kc] : 0;
                        const int cn = ok2 ? (int)blg[nv.o_colptr + kc + 1] - cb : 0;
                        const int cmax = (int)__reduce_max_sync(FULL, (unsigned)cn);
                        uint32_t hit = 0;  // one-sided rows of U the column fixes
                        for (int q = 0; q < cmax; ++q) {
                            int r = 0, sg = 0;
                            if (q < cn) {
                                const uint32_t ent = blg[nv.o_colent + cb + q];
                                r = ent_index(ent);
                                sg = ent_coef(ent) > 0 ? 1 : -1;
                            }
                            const int src = lead + ((r >> 2) % G);
                            const int bit = 4 * ((r >> 2) / G) + (r & 3);
                            const uint32_t wc = __shfl_sync(FULL, fxc, src);
                            const uint32_t wp = __shfl_sync(FULL, fxp, src);
                            const uint32_t wd = __shfl_sync(FULL, dl, src);
                            if (q < cn) {
                                // the column produces r: U must consume it, and the reverse
                                if (!(((sg > 0 ? wc : wp) >> bit) & 1u)) ok2 = false;
                                hit += (wd >> bit) & 1u;
                            }
                        }
                        ok2 = ok2 && hit == nd;
                        const bool any2 = group_or<G>(ok2 ? 1u : 0u) != 0;
                        if (act && any2) {
                            found = true;
                            open = false;
                        }
                    }
                    const bool dead = mine && nd > 0 && !found;
                    if (dead && gl == 0) ++n_capdead;
                    norm = norm && !dead;
                }

                // --- pivot key and fingerprint ---
                uint32_t key = 0xFFFFFFFFu, hlo = 0, hhi = 0;
                if (norm) {
#pragma unroll
                    for (int i = 0; i < CPL; ++i)
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) {
                            const int m = 4 * (gl + G * i) + jj;
                            const int32_t v = t32[4 * i + jj];
                            if (v != 0 && m < nv.M) {
                                const uint32_t kk = bl[(v > 0 ? nv.o_keypos : nv.o_keyneg) + m];
                                key = kk < key ? kk : key;
                            }
                            hash_entry((uint32_t)m, (uint32_t)v, hlo, hhi);
                        }
                    for (int w = gl; w < W; w += G) {
                        const uint64_t x = mix64(child_word(pu, w, k) ^ (0x2545f4914f6cdd1dull * (uint64_t)(w + 1)));
                        hlo += (uint32_t)x;
                        hhi ^= (uint32_t)(x >> 32);
                    }
                }
                key = group_min<G>(key);
                hlo = group_add<G>(hlo);
                hhi = group_xor<G>(hhi);

                // --- a reserved row for every surviving child of the round ---
                const unsigned nm = __ballot_sync(FULL, norm && gl == 0);
                const int cnt = __popc(nm);
                if (cnt > 0) {
                    const int rank = __popc(nm & ((1u << lead) - 1u));
                    uint64_t fresh = 0;
                    if (pool_left < cnt) {
                        if (lane == 0) fresh = atomicAdd(&a.ctr[C_WRITTEN], (unsigned long long)a.blk);
                        fresh = __shfl_sync(FULL, fresh, 0);
                    }
                    const uint64_t idx = rank < pool_left ? pool_next + (uint64_t)rank
                                                          : fresh + (uint64_t)(rank - pool_left);
                    if (pool_left < cnt) {
                        pool_next = fresh + (uint64_t)(cnt - pool_left);
                        pool_left = a.blk - (cnt - pool_left);
                    } else {
                        pool_next += (uint64_t)cnt;
                        pool_left -= cnt;
                    }
                    if (norm) {
                        if ((int64_t)idx < row_cap) {
                            int4 *db = reinterpret_cast<int4 *>(a.child.B + (size_t)idx * Mpad);
#pragma unroll
                            for (int i = 0; i < CPL; ++i)
                                db[gl + G * i] = make_int4(t32[4 * i + 0], t32[4 * i + 1], t32[4 * i + 2], t32[4 * i + 3]);
                            uint64_t *du = a.child.U + (size_t)idx * W;
                            for (int w = gl; w < W; w += G) du[w] = child_word(pu, w, k);
                            if (a.child.fx) {
                                a.child.fx[(size_t)idx * (2 * G) + gl] = fxc;
                                a.child.fx[(size_t)idx * (2 * G) + G + gl] = fxp;
                            }
                            if (gl == 0) a.child.meta[idx] = pack_meta(branch_key(bl, nv, key, a.sub), pc + (in_u ? 0 : 1));
                        } else if (gl == 0) {
                            ++n_unwritten;
                        }
                        if (gl == 0) {
                            if ((int64_t)idx < a.fp_cap) {
                                uint64_t f = ((uint64_t)hhi << 32) | hlo;
                                if (f == kDeadFp) f = kDeadFp - 1;
                                a.fp[idx] = f;
                            } else {
                                record_diag(a.ctr, ERR_BOUNDS, 7, (long long)idx, a.fp_cap, a.level);
                                fatal = true;
                            }
                        }
                    }
                }
            }
        }
        if (__any_sync(FULL, fatal)) break;
    }
    // rows reserved but not used: no fingerprint (the dedup pass skips them) and
    // no branches (the next level reads every row of the arena)
    for (int x = lane; x < pool_left; x += 32) {
        if ((int64_t)(pool_next + x) < a.fp_cap) a.fp[pool_next + x] = kDeadFp;
        if ((int64_t)(pool_next + x) < row_cap) a.child.meta[pool_next + x] = 0u;
    }
    if (n_exp) atomicAdd(&a.ctr[C_EXP], n_exp);
    if (n_ovf) atomicAdd(&a.ctr[C_OVF], n_ovf);
    if (n_bal) atomicAdd(&a.ctr[C_BAL], n_bal);
    if (n_pruned) atomicAdd(&a.ctr[C_PRUNED], n_pruned);
    if (n_unwritten) atomicAdd(&a.ctr[C_UNWRITTEN], n_unwritten);
    if (n_zero) atomicAdd(&a.ctr[C_ZERO], n_zero);
    if (n_capdead) atomicAdd(&a.ctr[C_CAPDEAD], n_capdead);
}

template <int G, int CPL>
__global__ void __launch_bounds__(kExpandWarps * 32, (CPL <= 2 ? 3 : 2)) generate_kernel(NetView nv, LevelArgs a,
                                                                                      int staged)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int wid = threadIdx.x >> 5;
    // staged: 0 nothing, 1 the whole blob, 2 its sparse tables [o_consptr, o_hbits)
    const int w0 = staged == 2 ? nv.o_consptr : 0;
    const int nw = staged == 1 ? nv.blob_words : (staged == 2 ? nv.o_hbits - nv.o_consptr : 0);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + nw);
    const uint32_t *bl = nv.blob;
    if (staged) {
        const uint32_t *sb = stage_words(nv, smem, mbar, w0, nw, a.ctr);
        if (sb == nullptr) return;
        // offsets index the blob: the staged range answers for [w0, w0 + nw)
        bl = reinterpret_cast<const uint32_t *>(reinterpret_cast<uintptr_t>(sb) - (uintptr_t)w0 * 4u);
    }
    generate_range<G, CPL>(nv, a, bl, staged == 2 ? nv.blob : bl, (int64_t)blockIdx.x * kExpandWarps + wid,
                           (int64_t)gridDim.x * kExpandWarps);
}

// ---------------------------------------------------------------------------
// Generate, narrow networks (at most 64 internal rows): incremental state
// summaries.
//
// The AND update t = A p + C s changes the sign pattern of the extra-flux
// row only on the rows of column k (A > 0), so a state carries summaries
// that a child updates from those few rows instead of scanning the whole
// row:
//   * two 64-bit masks of its positive and negative entries, with each row
//     at its rank in the positive / negative pivot-key order: the child's
//     pivot is the lowest set bit of either mask (Alg. 3's acting metabolite
//     under the fewest-reactions rule), and both masks empty means balanced;
//   * a linear row hash sum_m t_m R[m] (mod 2^64): the child's is
//     A h(p) + C h(S_int[:, k]);
//   * the rows holding +-1: with gcd(A, C) = 1, if the parent has a +-1 on a
//     row outside column k and either A = 1 or the entries of column k are
//     coprime, then every prime dividing all of t would divide A and
//     therefore, through the rows of column k, every entry of the column --
//     or divide the +-1 entry times A -- so gcd(t) = 1 with no gcd at all;
//   * a bound on max |t|: A pmax + C max|s| < 2^31 lets the update run in
//     plain 32-bit multiply-adds with no overflow test.
// A child without such a certificate, or with a possible overflow, takes the
// full-row path (exact gcd, 64-bit entries) and recomputes what it must.
//
// Work is split by its shape: everything per child (branch rules, the
// summaries from the rows of column k, balance test, superset rule, key,
// fingerprint, support and summary stores) runs one item per lane, 32
// children at once; only the dense extra-flux row (and a slow child's gcd)
// runs on groups of G lanes, each lane holding two 16-byte chunks, so the
// row's loads and stores are coalesced.
// ---------------------------------------------------------------------------

template <int G>
__device__ void generate_narrow(const NetView &nv, const LevelArgs &a, const uint32_t *bl, int64_t worker,
                                int64_t nworkers)
{
    constexpr int CPL = 2;
    constexpr int NG = 32 / G;
    const int lane = threadIdx.x & 31;
    const int gi = lane / G;
    const int gl = lane % G;
    const int W = nv.W;
    const int Mpad = nv.Mpad;
    const int4 *dcol = reinterpret_cast<const int4 *>(bl + nv.o_dcols);
    const int64_t row_cap = a.child.cap;

    unsigned long long n_exp = 0, n_ovf = 0, n_bal = 0, n_pruned = 0, n_unwritten = 0;
    bool fatal = false;
    uint64_t pool_next = 0;
    int pool_left = 0;
    uint64_t spool_next = 0;  // this warp's settle-record slots
    int spool_left = 0;
    // rows for cnt children of the warp (warp-uniform call); returns the
    // first row of the calling lane's share given its rank among them
    auto reserve = [&](int cnt, int rank) -> uint64_t {
        uint64_t fresh = 0;
        if (pool_left < cnt) {
            const int want = cnt > a.blk ? cnt : a.blk;
            if (lane == 0) fresh = atomicAdd(&a.ctr[C_WRITTEN], (unsigned long long)want);
            fresh = __shfl_sync(FULL, fresh, 0);
            const uint64_t idx = rank < pool_left ? pool_next + (uint64_t)rank : fresh + (uint64_t)(rank - pool_left);
            pool_next = fresh + (uint64_t)(cnt - pool_left);
            pool_left = want - (cnt - pool_left);
            return idx;
        }
        const uint64_t idx = pool_next + (uint64_t)rank;
        pool_next += (uint64_t)cnt;
        pool_left -= cnt;
        return idx;
    };

    const int cpw = a.cpw;
    const int64_t wstride = nworkers * cpw;
    for (int64_t p0 = worker * cpw; p0 < a.n_par; p0 += wstride) {
        const int64_t pl = p0 + lane;
        const bool pin = lane < cpw && pl < a.n_par;
        const int64_t pid = pin ? (a.perm ? (int64_t)a.perm[pl] : a.par_base + pl) : 0;
        // (no L2 prefetch of the next chunk's parents: measured slower here)
        const uint32_t mj = pin ? a.par.meta[pid] : 0u;
        int dj = pin ? (int)((mj >> 10) & 0x1FFFu) : 0;
        if (a.fk_pc > 0 && (int)((mj >> 23) & 0x7Fu) > a.fk_pc) dj = 0;
        int incl = dj;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int x = __shfl_up_sync(FULL, incl, off);
            if (lane >= off) incl += x;
        }
        const int prej = incl - dj;
        const int T = __shfl_sync(FULL, incl, 31);
        if (T > 32 * nv.N) {
            if (lane == 0) record_diag(a.ctr, ERR_BOUNDS, 3, T, 32 * nv.N, a.level);
            fatal = true;
        }
        for (int base = 0; base < T; base += 32) {
            if (__any_sync(FULL, fatal)) break;
            // === phase A: one (parent, branch) item per lane.  Branch rules,
            // then the child's summaries from the rows of column k only ===
            const int c = base + lane;
            int j = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int v = __shfl_sync(FULL, prej, j + step);
                if (v <= c) j += step;
            }
            const uint32_t pm = __shfl_sync(FULL, mj, j);
            const int q = c - __shfl_sync(FULL, prej, j);
            const int64_t pl_ = __shfl_sync(FULL, pid, j);
            bool okl = c < T;
            int kl = 0, pcl = 0;
            bool inl = false;
            int32_t Al = 0, Cl = 0;
            const uint64_t *pu_l = a.par.U + (size_t)pl_ * W;
            const int32_t *prow_l = a.par.B + (size_t)pl_ * Mpad;
            if (okl) {
                const int piv = (int)(pm & 0x3FFu);
                pcl = (int)((pm >> 23) & 0x7Fu);
                const int32_t bi = piv < nv.M ? prow_l[piv] : 0;
                const bool fwd = bi > 0;
                const uint32_t abi = (uint32_t)(bi < 0 ? -bi : bi);
                const int lptr = (fwd ? nv.o_consptr : nv.o_prodptr) + (piv < nv.M ? piv : 0);
                const int lb = (int)bl[lptr];
                const int le = (int)bl[lptr + 1];
                if (piv >= nv.M || bi == 0 || lb + q >= le) {
                    record_diag(a.ctr, ERR_BOUNDS, 1 + (piv >= nv.M ? 10 : 0) + (bi == 0 ? 100 : 0), (long long)q,
                                (long long)(le - lb), a.level);
                    fatal = true;
                    okl = false;
                } else {
                    const uint32_t br = bl[(fwd ? nv.o_consent : nv.o_prodent) + lb + q];
                    kl = ent_index(br);
                    const uint32_t sik = (uint32_t)ent_coef(br);
                    const int tw = (int)bl[nv.o_twin + kl];
                    inl = bit_of(pu_l, kl);
                    const int sec = a.level - pcl;
                    okl = !(tw >= 0 && bit_of(pu_l, tw)) && (inl ? sec + 1 <= a.max_sec : pcl + 1 <= a.max_len);
                    if (okl && a.fk_pc > 0) {
                        const int pc2 = pcl + (inl ? 0 : 1);
                        okl = pc2 < a.fk_pc || (pc2 == a.fk_pc && !child_after(pu_l, kl, a.fk_sup, W));
                    }
                    const uint32_t g0 = (abi == 1u || sik == 1u) ? 1u : gcd32(abi, sik);
                    Al = (int32_t)(sik / g0);
                    Cl = (int32_t)(abi / g0);
                }
            }
            if (okl) ++n_exp;
            // summaries of the child (exact signs from 64-bit entries)
            NarrowSum sm{0, 0, 0, 0, 0, 0};
            bool fast = false, cert = false;
            uint32_t gtl = 1;  // gcd of the changed entries (when fast)
            if (okl) {
                const NarrowSum ps = get_summary(a.par.sum + (size_t)pl_ * kSumWords);
                const uint32_t pmaxp = ps.pmax;
                const int ox = nv.o_colx + kColxWordsDev * kl;
                const uint64_t suppP = blob_u64(bl, ox), suppN = blob_u64(bl, ox + 2), suppR = blob_u64(bl, ox + 4);
                const uint32_t smax = bl[ox + 8], gcd1 = bl[ox + 9];
                fast = (uint64_t)Al * pmaxp + (uint64_t)Cl * smax <= 2147483647ull;
                uint64_t newp = 0, newn = 0, newu = 0, newo = 0, tmax = 0;
                uint32_t gt = 0;  // gcd of the changed entries (exact when fast: they fit 32 bits)
                for (int qq = (int)bl[nv.o_colptr + kl]; qq < (int)bl[nv.o_colptr + kl + 1]; ++qq) {
                    const uint32_t e = bl[nv.o_colent + qq];
                    const int m = ent_index(e);
                    const int64_t tm = (int64_t)Al * prow_l[m] + (int64_t)Cl * ent_coef(e);
                    const uint32_t rk = bl[nv.o_rank + m];
                    newp |= (tm > 0 ? 1ull : 0ull) << (rk & 0xFFu);
                    newn |= (tm < 0 ? 1ull : 0ull) << ((rk >> 8) & 0xFFu);
                    newu |= ((tm == 1 || tm == -1) ? 1ull : 0ull) << m;
                    newo |= (uint64_t)(tm & 1) << m;
                    const uint64_t am = (uint64_t)(tm < 0 ? -tm : tm);
                    tmax = am > tmax ? am : tmax;
                    if (am != 0 && gt != 1) gt = gt == 0 ? (uint32_t)am : gcd32(gt, (uint32_t)am);
                }
                sm.pm = (ps.pm & ~suppP) | newp;
                sm.nm = (ps.nm & ~suppN) | newn;
                const uint64_t uout = ps.um & ~suppR;  // parent's +-1 rows outside column k
                sm.um = (Al == 1 ? uout : 0ull) | newu;
                sm.om = ((Al & 1) ? (ps.om & ~suppR) : 0ull) | newo;  // odd rows (A p is odd iff both are)
                sm.rh = (uint64_t)(int64_t)Al * ps.rh + (uint64_t)(int64_t)Cl * blob_u64(bl, ox + 6);
                const uint64_t bound = (uint64_t)Al * pmaxp > tmax ? (uint64_t)Al * pmaxp : tmax;
                sm.pmax = bound > 2147483647ull ? 2147483647u : (uint32_t)bound;
                // gcd(t) = 1 without computing it: a +-1 entry in the child, a
                // parent +-1 outside column k with A = 1 or a coprime column, or
                // coprime changed entries (every common divisor divides them)
                cert = sm.um != 0 || (uout != 0 && (Al == 1 || gcd1 != 0)) || (fast && gt == 1) ||
                       (fast && gt != 0 && (gt & (gt - 1)) == 0 && sm.om != 0);  // gcd | 2^a, and an odd entry
                gtl = gt;  // 0: no changed entry is nonzero (the whole row decides)
            }
            const bool nzl = (sm.pm | sm.nm) != 0;
            const bool ball = okl && !nzl;
            if (ball) {
                ++n_bal;  // all metabolites stable: to the arbiter
                if (insert_support(a, W, pu_l, kl) < INS_DUP) fatal = true;
            }
            // ready: the child is final (no overflow possible, gcd 1): prune
            // test, key and fingerprint here.  verify: no overflow possible,
            // the gcd not certified; the lane group writing its row takes the
            // gcd of the whole row, and only a child whose gcd is above 1 (rare)
            // goes on to the settle pass.  slow: a possible overflow, settled.
            bool ready = okl && nzl && fast;
            const bool vfyl = ready && !cert;
            bool slowl = okl && nzl && !fast;
            // the superset rule through the sentinel index runs in the prune
            // pass over the reserved rows; the column buckets here otherwise
            if (ready && !inl && !(W <= 2 && a.cptr)) {
                const int64_t b1 = a.bptr[kl];
                const int64_t n = a.bptr[kl + 1] - b1;
                bool pr = false;
                if (n > 0) {
                    if (W <= 2) {
                        const uint64_t u0 = child_word(pu_l, 0, kl), u1 = W == 2 ? child_word(pu_l, 1, kl) : 0ull;
                        bool maybe = true;
                        if (a.band) {
                            const uint64_t i0 = __ldg(a.band + (size_t)kl * W), i1 = W == 2 ? __ldg(a.band + (size_t)kl * W + 1) : 0ull;
                            maybe = ((i0 & ~u0) | (i1 & ~u1)) == 0;
                        }
                        for (int64_t i = 0; i < n && !pr && maybe; ++i) {
                            const uint64_t *E = a.bres + (size_t)(b1 + i) * W;
                            const uint64_t e0 = __ldg(E), e1 = W == 2 ? __ldg(E + 1) : 0ull;
                            pr = ((e0 & ~u0) | (e1 & ~u1)) == 0;
                        }
                    } else {
                        for (int64_t i = 0; i < n && !pr; ++i) pr = result_inside_wide(a, pu_l, kl, b1 + i);
                    }
                }
                if (pr) {
                    ++n_pruned;
                    ready = false;
                }
            }
            // rows for the ready children of the pass, written per lane
            // except the extra-flux row (phase B, coalesced by lane groups)
            const unsigned rmask = __ballot_sync(FULL, ready);
            uint64_t myidx = 0;
            if (rmask) {
                myidx = reserve(__popc(rmask), __popc(rmask & ((1u << lane) - 1u)));
                if (ready) {
                    if ((int64_t)myidx < row_cap) {
                        uint64_t *du = a.child.U + (size_t)myidx * W;
                        for (int w = 0; w < W; ++w) du[w] = child_word(pu_l, w, kl);
                        a.child.meta[myidx] = pack_meta(mask_key(bl, nv, sm.pm, sm.nm), pcl + (inl ? 0 : 1));
                        put_summary(a.child.sum + (size_t)myidx * kSumWords, sm);
                    } else {
                        ++n_unwritten;
                    }
                    if ((int64_t)myidx < a.fp_cap) {
                        uint64_t f = sm.rh ^ mix64(support_hash(pu_l, W, kl) + 0x632BE59BD9B4E019ull);
                        if (f == kDeadFp) f = kDeadFp - 1;
                        a.fp[myidx] = f;
                        // the row itself is written by the row pass
                        a.wrec[myidx] = make_uint4((uint32_t)pl_, (uint32_t)kl | (vfyl ? 1u << 12 : 0u) |
                                                                      (inl ? 1u << 13 : 0u) | ((uint32_t)pcl << 14),
                                                   (uint32_t)Al, (uint32_t)Cl);
                    } else {
                        record_diag(a.ctr, ERR_BOUNDS, 7, (long long)myidx, a.fp_cap, a.level);
                        fatal = true;
                    }
                }
            }
            const uint32_t pl32 = (uint32_t)pl_;
            // === the slow children (no gcd certificate or a possible overflow)
            // go to the settle pass as records ===
            const unsigned smask = __ballot_sync(FULL, slowl);
            if (smask) {
                // record slots from this warp's pool (32 at a time, one atomic)
                const int scnt = __popc(smask), srank = __popc(smask & ((1u << lane) - 1u));
                uint64_t sfresh = 0;
                if (spool_left < scnt) {
                    if (lane == 0) sfresh = atomicAdd(&a.ctr[C_SLOW], 32ull);
                    sfresh = __shfl_sync(FULL, sfresh, 0);
                }
                const uint64_t si = srank < spool_left ? spool_next + (uint64_t)srank
                                                       : sfresh + (uint64_t)(srank - spool_left);
                if (spool_left < scnt) {
                    spool_next = sfresh + (uint64_t)(scnt - spool_left);
                    spool_left = 32 - (scnt - spool_left);
                } else {
                    spool_next += (uint64_t)scnt;
                    spool_left -= scnt;
                }
                if (slowl) {
                    if ((int64_t)si < a.slow_cap) {
                        uint64_t *r = a.slow + (size_t)si * kSlowWords;
                        const uint64_t w0 = (uint64_t)pl32 | ((uint64_t)kl << 32) | ((uint64_t)pcl << 44) |
                                            (inl ? 1ull << 51 : 0ull) | (fast ? 1ull << 52 : 0ull);
                        const uint64_t w1 = (uint64_t)(uint32_t)Al | ((uint64_t)(uint32_t)Cl << 32);
                        *reinterpret_cast<ulonglong2 *>(r) = make_ulonglong2(w0, w1);
                        *reinterpret_cast<ulonglong2 *>(r + 2) = make_ulonglong2(sm.rh, sm.pm);
                        *reinterpret_cast<ulonglong2 *>(r + 4) = make_ulonglong2(sm.nm, sm.um);
                        *reinterpret_cast<ulonglong2 *>(r + 6) = make_ulonglong2(sm.om, 0ull);
                    } else {
                        record_diag(a.ctr, ERR_BOUNDS, 9, (long long)si, a.slow_cap, a.level);
                        fatal = true;
                    }
                }
            }
        }
        if (__any_sync(FULL, fatal)) break;
    }
    for (int x = lane; x < pool_left; x += 32) {
        if ((int64_t)(pool_next + x) < a.fp_cap) {
            a.fp[pool_next + x] = kDeadFp;
            a.wrec[pool_next + x].x = kNoRecord;
        }
        if ((int64_t)(pool_next + x) < row_cap) a.child.meta[pool_next + x] = 0u;
    }
    // settle-record slots left unused: marked so that the settle pass skips them
    if (lane < spool_left && (int64_t)(spool_next + lane) < a.slow_cap) a.slow[(spool_next + lane) * kSlowWords] = ~0ull;
    if (n_exp) atomicAdd(&a.ctr[C_EXP], n_exp);
    if (n_ovf) atomicAdd(&a.ctr[C_OVF], n_ovf);
    if (n_bal) atomicAdd(&a.ctr[C_BAL], n_bal);
    if (n_pruned) atomicAdd(&a.ctr[C_PRUNED], n_pruned);
    if (n_unwritten) atomicAdd(&a.ctr[C_UNWRITTEN], n_unwritten);
}

template <int G>
__global__ void __launch_bounds__(kExpandWarps * 32, 6) generate_narrow_kernel(NetView nv, LevelArgs a, int staged)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int wid = threadIdx.x >> 5;
    const int blob_words = staged ? nv.blob_words : 0;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + blob_words);
    const uint32_t *bl = stage_blob(nv, smem, mbar, staged != 0, a.ctr);
    if (bl == nullptr) return;
    generate_narrow<G>(nv, a, bl, (int64_t)blockIdx.x * kExpandWarps + wid, (int64_t)gridDim.x * kExpandWarps);
}

// ---------------------------------------------------------------------------
// Prune pass (narrow networks, supports of at most 2 words): one thread per
// reserved row with a row-pass record that adds a new column.  The superset
// rule on the child's support (the parent's, plus the column); a pruned
// child gives its row up (no state, no fingerprint, no record).  A child
// without a written row is tested the same way, from its parent.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) prune_rows_kernel(NetView nv, LevelArgs a)
{
    const uint64_t begin = a.ctr[C_DEDUP_BEGIN];
    uint64_t end = a.ctr[C_WRITTEN];
    end = end < (uint64_t)a.fp_cap ? end : (uint64_t)a.fp_cap;
    const uint64_t row_cap = (uint64_t)a.child.cap;
    const int W = nv.W;
    unsigned long long n_pr = 0, n_unw = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = begin + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < end; i += stride) {
        const uint4 rc = a.wrec[i];
        if (rc.x == kNoRecord || ((rc.y >> 13) & 1u)) continue;  // nothing to write, or a secondary step
        const int k = (int)(rc.y & 0xFFFu);
        if (pruned_indexed(a, a.par.U + (size_t)rc.x * W, k, W, nv.N)) {
            a.fp[i] = kDeadFp;
            a.wrec[i].x = kNoRecord;
            if (i < row_cap)
                a.child.meta[i] = 0u;
            else
                ++n_unw;
            ++n_pr;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        n_pr += __shfl_xor_sync(FULL, n_pr, off);
        n_unw += __shfl_xor_sync(FULL, n_unw, off);
    }
    if ((threadIdx.x & 31) == 0) {
        if (n_pr) atomicAdd(&a.ctr[C_PRUNED], n_pr);
        if (n_unw) atomicAdd(&a.ctr[C_UNWRITTEN], (unsigned long long)(-(long long)n_unw));
    }
}

// ---------------------------------------------------------------------------
// Row pass (narrow networks): one lane group per reserved row of the level,
// in row order.  A row with a record gets t = A p + C s (32 bits: the
// generate pass recorded only children that cannot overflow); when the
// summaries did not certify its gcd, the group folds the row into its gcd
// first, and a row with a gcd above 1 (rare) is withdrawn and handed to the
// settle pass with its phase-A summaries.
// ---------------------------------------------------------------------------
template <int G, int CPL>
__global__ void __launch_bounds__(256) write_rows_kernel(NetView nv, LevelArgs a)
{
    constexpr int NG = 32 / G;
    const int lane = threadIdx.x & 31;
    const int gi = lane / G;
    const int gl = lane % G;
    const int Mpad = nv.Mpad;
    const int4 *dcol = reinterpret_cast<const int4 *>(nv.blob + nv.o_dcols);
    const uint64_t begin = a.ctr[C_DEDUP_BEGIN];
    uint64_t end = a.ctr[C_WRITTEN];
    end = end < (uint64_t)a.fp_cap ? end : (uint64_t)a.fp_cap;
    end = end < (uint64_t)a.child.cap ? end : (uint64_t)a.child.cap;
    const uint64_t wid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t r0 = begin + wid * NG; r0 < end; r0 += nwarps * NG) {
        const uint64_t idx = r0 + gi;
        uint4 rc = make_uint4(kNoRecord, 0u, 0u, 0u);
        if (idx < end) rc = a.wrec[idx];
        const bool has = rc.x != kNoRecord;
        const int k = (int)(rc.y & 0xFFFu);
        const bool vfy = has && ((rc.y >> 12) & 1u);
        const int32_t A = (int32_t)rc.z, C = (int32_t)rc.w;
        int4 t4[CPL];
        uint32_t gg = vfy ? 0u : 1u;
        if (has) {
            const int4 *prow4 = reinterpret_cast<const int4 *>(a.par.B + (size_t)rc.x * Mpad);
            const int4 *col4 = dcol + (size_t)k * (Mpad >> 2);
#pragma unroll
            for (int i = 0; i < CPL; ++i) {
                const int4 v = prow4[gl + G * i];
                const int4 w = col4[gl + G * i];
                t4[i] = make_int4(A * v.x + C * w.x, A * v.y + C * w.y, A * v.z + C * w.z, A * v.w + C * w.w);
            }
            if (vfy) {
#pragma unroll
                for (int i = 0; i < CPL; ++i) {
                    const int32_t xs[4] = {t4[i].x, t4[i].y, t4[i].z, t4[i].w};
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj)
                        if (gg != 1u && xs[jj] != 0) gg = gcd32(gg, (uint32_t)(xs[jj] < 0 ? -xs[jj] : xs[jj]));
                }
            }
        }
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) {
            const uint32_t og = __shfl_xor_sync(FULL, gg, off);
            if (gg != 1u || og != 1u) gg = gcd32(gg, og);
        }
        const bool bad = vfy && gg != 1u;
        if (has && !bad) {
            int4 *db = reinterpret_cast<int4 *>(a.child.B + (size_t)idx * Mpad);
#pragma unroll
            for (int i = 0; i < CPL; ++i) db[gl + G * i] = t4[i];
        }
        if (bad && gl == 0) {
            // withdrawn: the row carries no state; the settle pass makes the child
            a.child.meta[idx] = 0u;
            a.fp[idx] = kDeadFp;
            const uint64_t si = atomicAdd(&a.ctr[C_SLOW], 1ull);
            if ((int64_t)si < a.slow_cap) {
                const uint64_t *sm = a.child.sum + (size_t)idx * kSumWords;
                uint64_t *r = a.slow + (size_t)si * kSlowWords;
                const uint64_t w0 = (uint64_t)rc.x | ((uint64_t)k << 32) | ((uint64_t)((rc.y >> 14) & 0x7Fu) << 44) |
                                    (((rc.y >> 13) & 1u) ? 1ull << 51 : 0ull) | (1ull << 52);
                const uint64_t w1 = (uint64_t)rc.z | ((uint64_t)rc.w << 32);
                r[0] = w0;
                r[1] = w1;
                r[2] = sm[0];  // row hash
                r[3] = sm[1];  // positive entries (key-rank order)
                r[4] = sm[2];  // negative entries
                r[5] = sm[3];  // +-1 rows
                r[6] = sm[4];  // odd rows
                r[7] = 0ull;
            } else {
                record_diag(a.ctr, ERR_BOUNDS, 11, (long long)si, a.slow_cap, a.level);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Settle pass (narrow networks): the children whose gcd the summaries do not
// certify, or whose update may leave int32, listed by the generate pass as
// records (parent, column, |U|, flags, A, C and their phase-A summaries).
// A group of G lanes per record: the row in 32 or 64 bits, the exact gcd and
// int32 range over the whole row (the overflow rule comes before the
// superset rule, as in the definition), the superset rule, then a reserved
// row.  Keeping this rare, long path out of the generate kernel keeps that
// kernel's instruction footprint small.
// ---------------------------------------------------------------------------
template <int G>
__global__ void __launch_bounds__(kExpandWarps * 32) settle_kernel(NetView nv, LevelArgs a)
{
    constexpr int CPL = 2;
    constexpr int NG = 32 / G;
    constexpr int EPL = 4 * CPL;
    const int lane = threadIdx.x & 31;
    const int gi = lane / G;
    const int gl = lane % G;
    const int lead = gi * G;
    const int W = nv.W;
    const int Mpad = nv.Mpad;
    const uint32_t *bl = nv.blob;
    const int4 *dcol = reinterpret_cast<const int4 *>(bl + nv.o_dcols);
    const int64_t row_cap = a.child.cap;
    int64_t n_slow = (int64_t)a.ctr[C_SLOW];
    n_slow = n_slow < a.slow_cap ? n_slow : a.slow_cap;
    unsigned long long n_ovf = 0, n_pruned = 0, n_unwritten = 0;
    bool fatal = false;
    uint64_t pool_next = 0;
    int pool_left = 0;
    auto reserve = [&](int cnt, int rank) -> uint64_t {
        uint64_t fresh = 0;
        if (pool_left < cnt) {
            const int want = cnt;  // exactly what the round needs: no unused rows
            if (lane == 0) fresh = atomicAdd(&a.ctr[C_WRITTEN], (unsigned long long)want);
            fresh = __shfl_sync(FULL, fresh, 0);
            const uint64_t idx = rank < pool_left ? pool_next + (uint64_t)rank : fresh + (uint64_t)(rank - pool_left);
            pool_next = fresh + (uint64_t)(cnt - pool_left);
            pool_left = want - (cnt - pool_left);
            return idx;
        }
        const uint64_t idx = pool_next + (uint64_t)rank;
        pool_next += (uint64_t)cnt;
        pool_left -= cnt;
        return idx;
    };
    const int64_t wid = (int64_t)blockIdx.x * kExpandWarps + (threadIdx.x >> 5);
    const int64_t wstride = (int64_t)gridDim.x * kExpandWarps * NG;
    for (int64_t base = wid * NG; base < n_slow; base += wstride) {
        if (__any_sync(FULL, fatal)) break;
            const int64_t r = base + gi;
            bool slow = r < n_slow;
            // the record (every lane of the group reads it)
            uint64_t w0 = 0, w1 = 0, srh = 0, spm = 0, snm = 0, sum_ = 0, som = 0;
            if (slow) {
                const uint64_t *rec = a.slow + (size_t)r * kSlowWords;
                const ulonglong2 q0 = *reinterpret_cast<const ulonglong2 *>(rec);
                const ulonglong2 q1 = *reinterpret_cast<const ulonglong2 *>(rec + 2);
                const ulonglong2 q2 = *reinterpret_cast<const ulonglong2 *>(rec + 4);
                const ulonglong2 q3 = *reinterpret_cast<const ulonglong2 *>(rec + 6);
                w0 = q0.x;
                w1 = q0.y;
                srh = q1.x;
                spm = q1.y;
                snm = q2.x;
                sum_ = q2.y;
                som = q3.x;
                slow = w0 != ~0ull;  // an unused slot
            }
            const int64_t p = (int64_t)(uint32_t)w0;
            const int k = (int)((w0 >> 32) & 0xFFFu);
            const int pc = (int)((w0 >> 44) & 0x7Fu);
            const bool in_u = (w0 >> 51) & 1ull;
            const bool fst = (w0 >> 52) & 1ull;  // the update fits 32 bits
            const int32_t A = (int32_t)(uint32_t)w1;
            const int32_t C = (int32_t)(uint32_t)(w1 >> 32);
                const int4 *prow4 = reinterpret_cast<const int4 *>(a.par.B + (size_t)p * Mpad);
                const int4 *col4 = dcol + (size_t)k * (Mpad >> 2);
                int32_t t32[EPL];
                bool big = false;
                uint64_t gg = 0, amax = 0;
                if (slow && fst) {
                    uint32_t g32 = 0, m32 = 0;
#pragma unroll
                    for (int i = 0; i < CPL; ++i) {
                        const int4 v = prow4[gl + G * i];
                        const int4 w = col4[gl + G * i];
                        t32[4 * i + 0] = A * v.x + C * w.x;
                        t32[4 * i + 1] = A * v.y + C * w.y;
                        t32[4 * i + 2] = A * v.z + C * w.z;
                        t32[4 * i + 3] = A * v.w + C * w.w;
                    }
#pragma unroll
                    for (int e = 0; e < EPL; ++e) {
                        const uint32_t at = (uint32_t)(t32[e] < 0 ? -t32[e] : t32[e]);
                        if (at != 0 && g32 != 1) g32 = g32 == 0 ? at : gcd32(g32, at);
                        m32 = at > m32 ? at : m32;
                    }
                    gg = g32;
                    amax = m32;
                } else if (slow) {
#pragma unroll
                    for (int i = 0; i < CPL; ++i) {
                        const int4 v = prow4[gl + G * i];
                        const int4 w = col4[gl + G * i];
                        const int32_t pv[4] = {v.x, v.y, v.z, v.w}, cv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) {
                            const int64_t tt = (int64_t)A * pv[jj] + (int64_t)C * cv[jj];
                            const int32_t lo = (int32_t)tt;
                            big = big || tt != (int64_t)lo || lo == INT32_MIN;
                            t32[4 * i + jj] = lo;
                        }
                    }
                    if (!big) {
#pragma unroll
                        for (int e = 0; e < EPL; ++e) {
                            const uint32_t at = (uint32_t)(t32[e] < 0 ? -t32[e] : t32[e]);
                            if (at != 0 && gg != 1) gg = gg == 0 ? at : gcd32((uint32_t)gg, at);
                            amax = at > amax ? at : amax;
                        }
                    } else {
                        const GcdMax gmx = raw_gcd_max(prow4, col4, gl, G, CPL, A, C);
                        gg = gmx.g;
                        amax = gmx.m;
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < EPL; ++e) t32[e] = 0;
                }
                big = group_or<G>(big ? 1u : 0u) != 0;
                if (!__any_sync(FULL, big)) {
                    // every entry of every slow row of the round fits 32 bits
                    uint32_t g32 = (uint32_t)gg, m32 = (uint32_t)amax;
#pragma unroll
                    for (int off = G / 2; off > 0; off >>= 1) {
                        const uint32_t og = __shfl_xor_sync(FULL, g32, off);
                        g32 = (og == 0 || g32 == 1) ? g32 : (g32 == 0 ? og : gcd32(g32, og));
                        const uint32_t y = __shfl_xor_sync(FULL, m32, off);
                        m32 = y > m32 ? y : m32;
                    }
                    gg = g32;
                    amax = m32;
                } else {
#pragma unroll
                    for (int off = G / 2; off > 0; off >>= 1) {
                        const uint64_t og = __shfl_xor_sync(FULL, gg, off);
                        gg = og == 0 ? gg : (gg == 0 ? og : gcd64(gg, og));
                        const uint64_t y = __shfl_xor_sync(FULL, amax, off);
                        amax = y > amax ? y : amax;
                    }
                }
                if (gg == 0) gg = 1;
                const bool ovf = slow && amax / gg > 2147483647ull;
                if (slow && !ovf && gg > 1) {
                    if (!big) {
#pragma unroll
                        for (int e = 0; e < EPL; ++e) t32[e] = t32[e] / (int32_t)gg;
                    } else {
#pragma unroll
                        for (int i = 0; i < CPL; ++i) {
                            const int4 v = prow4[gl + G * i];
                            const int4 w = col4[gl + G * i];
                            const int32_t pv[4] = {v.x, v.y, v.z, v.w}, cv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                            for (int jj = 0; jj < 4; ++jj) {
                                const int64_t tt = (int64_t)A * pv[jj] + (int64_t)C * cv[jj];
                                t32[4 * i + jj] = (int32_t)(tt / (int64_t)gg);
                            }
                        }
                    }
                }
                if (ovf && gl == 0) ++n_ovf;
                const uint64_t *pu = a.par.U + (size_t)p * W;
                bool pr = false;
                const bool cand = slow && !ovf;
                if (cand && !in_u) {
                    const int64_t b1 = a.bptr[k];
                    const int64_t n = a.bptr[k + 1] - b1;
                    if (W <= 2 && a.cptr) {
                        if (gl == 0) pr = pruned_indexed(a, pu, k, W, nv.N);
                    } else if (W <= 2) {
                        const uint64_t u0 = child_word(pu, 0, k), u1 = W == 2 ? child_word(pu, 1, k) : 0ull;
                        bool maybe = n > 0;
                        if (maybe && a.band) {
                            const uint64_t i0 = __ldg(a.band + (size_t)k * W), i1 = W == 2 ? __ldg(a.band + (size_t)k * W + 1) : 0ull;
                            maybe = ((i0 & ~u0) | (i1 & ~u1)) == 0;
                        }
                        for (int64_t i = gl; i < n && !pr && maybe; i += G) {
                            const uint64_t *E = a.bres + (size_t)(b1 + i) * W;
                            const uint64_t e0 = __ldg(E), e1 = W == 2 ? __ldg(E + 1) : 0ull;
                            pr = ((e0 & ~u0) | (e1 & ~u1)) == 0;
                        }
                    } else {
                        for (int64_t i = gl; i < n && !pr; i += G) pr = result_inside_wide(a, pu, k, b1 + i);
                    }
                }
                pr = group_or<G>(pr ? 1u : 0u) != 0;
                if (pr && gl == 0) ++n_pruned;
                const bool keep = cand && !pr;
                // a row divided by its gcd: +-1 rows and hash over the row (the
                // signs do not change); otherwise phase A's values stand
                uint64_t um = sum_, om = som, rh = srh;
                if (__any_sync(FULL, keep && gg > 1)) {
                    uint64_t u2 = 0, o2 = 0, h2 = 0;
                    if (keep && gg > 1) {
#pragma unroll
                        for (int i = 0; i < CPL; ++i)
#pragma unroll
                            for (int jj = 0; jj < 4; ++jj) {
                                const int m = 4 * (gl + G * i) + jj;
                                const int32_t v = t32[4 * i + jj];
                                if (m < nv.M && v != 0) {
                                    if (v == 1 || v == -1) u2 |= 1ull << m;
                                    if (v & 1) o2 |= 1ull << m;
                                    h2 += (uint64_t)(int64_t)v * blob_u64(bl, nv.o_hrow + 2 * m);
                                }
                            }
                    }
#pragma unroll
                    for (int off = G / 2; off > 0; off >>= 1) {
                        u2 |= __shfl_xor_sync(FULL, u2, off);
                        o2 |= __shfl_xor_sync(FULL, o2, off);
                        h2 += __shfl_xor_sync(FULL, h2, off);
                    }
                    if (keep && gg > 1) {
                        um = u2;
                        om = o2;
                        rh = h2;
                    }
                }
                const unsigned km = __ballot_sync(FULL, keep && gl == 0);
                if (km) {
                    const uint64_t idx = reserve(__popc(km), __popc(km & ((1u << lead) - 1u)));
                    if (keep) {
                        if ((int64_t)idx < row_cap) {
                            int4 *db = reinterpret_cast<int4 *>(a.child.B + (size_t)idx * Mpad);
#pragma unroll
                            for (int i = 0; i < CPL; ++i)
                                db[gl + G * i] = make_int4(t32[4 * i + 0], t32[4 * i + 1], t32[4 * i + 2], t32[4 * i + 3]);
                            uint64_t *du = a.child.U + (size_t)idx * W;
                            for (int w = gl; w < W; w += G) du[w] = child_word(pu, w, k);
                            if (gl == 0) {
                                a.child.meta[idx] = pack_meta(mask_key(bl, nv, spm, snm), pc + (in_u ? 0 : 1));
                                put_summary(a.child.sum + (size_t)idx * kSumWords,
                                            NarrowSum{rh, spm, snm, um, om, (uint32_t)(amax / gg)});
                            }
                        } else if (gl == 0) {
                            ++n_unwritten;
                        }
                        if (gl == 0) {
                            if ((int64_t)idx < a.fp_cap) {
                                uint64_t f = rh ^ mix64(support_hash(pu, W, k) + 0x632BE59BD9B4E019ull);
                                if (f == kDeadFp) f = kDeadFp - 1;
                                a.fp[idx] = f;
                            } else {
                                record_diag(a.ctr, ERR_BOUNDS, 7, (long long)idx, a.fp_cap, a.level);
                                fatal = true;
                            }
                        }
                    }
                }
                fatal = group_or<G>(fatal ? 1u : 0u) != 0;
    }
    for (int x = lane; x < pool_left; x += 32)
        if ((int64_t)(pool_next + x) < a.fp_cap) a.fp[pool_next + x] = kDeadFp;
    if (n_ovf) atomicAdd(&a.ctr[C_OVF], n_ovf);
    if (n_pruned) atomicAdd(&a.ctr[C_PRUNED], n_pruned);
    if (n_unwritten) atomicAdd(&a.ctr[C_UNWRITTEN], n_unwritten);
}

// Are reserved rows i and j the same state (support and extra-flux row)?
__device__ __forceinline__ bool same_state(const Arena &ar, int Mpad, int W, uint64_t i, uint64_t j)
{
    const int4 *x = reinterpret_cast<const int4 *>(ar.B + (size_t)i * Mpad);
    const int4 *y = reinterpret_cast<const int4 *>(ar.B + (size_t)j * Mpad);
    bool eq = true;
    for (int c = 0; c < (Mpad >> 2) && eq; ++c) {
        const int4 u = __ldcg(x + c), v = __ldcg(y + c);
        eq = u.x == v.x && u.y == v.y && u.z == v.z && u.w == v.w;
    }
    const uint64_t *ux = ar.U + (size_t)i * W, *uy = ar.U + (size_t)j * W;
    for (int w = 0; w < W && eq; ++w) eq = __ldcg(ux + w) == __ldcg(uy + w);
    return eq;
}

// One thread per reserved row in [ctr[C_DEDUP_BEGIN], ctr[C_WRITTEN]).  The
// first row of every distinct state survives in place; a later copy gets a
// zero meta word (no branches), so the next level reads the arena's rows in
// order and no survivor list is built.  Survivors and their branch counts
// are summed per block, with one atomic per block.
__global__ void __launch_bounds__(256) dedup_kernel(LevelArgs a, int Mpad, int W)
{
    __shared__ unsigned long long s_keep[8], s_deg[8], s_unv[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint64_t begin = a.ctr[C_DEDUP_BEGIN];
    uint64_t end = a.ctr[C_WRITTEN];
    end = end < (uint64_t)a.fp_cap ? end : (uint64_t)a.fp_cap;
    const uint64_t row_cap = (uint64_t)a.child.cap;
    unsigned long long deg = 0, n_unv = 0, n_keep = 0;
    bool fatal = false;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i0 = begin + (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < end; i0 += stride) {
        const uint64_t i = i0 + lane;
        bool mine = i < end;
        const uint64_t f = mine ? a.fp[i] : kDeadFp;
        mine = mine && f != kDeadFp;
        if (mine) {
            uint64_t pos;
            uint32_t tag;
            slot_tag_pos(f, a.slot_mask, pos, tag);
            const bool written = i < row_cap;
            if (i >= 0xFFFFFFFEull) {
                record_diag(a.ctr, ERR_BOUNDS, 10, (long long)i, 0xFFFFFFFEll, a.level);
                fatal = true;
            }
            for (uint64_t probe = 0; !fatal; ++probe) {
                if (probe > a.slot_mask) {
                    record_diag(a.ctr, ERR_TABLE_FULL, 8, (long long)i, (long long)a.slot_mask, a.level);
                    fatal = true;
                    break;
                }
                const unsigned long long v = atomicCAS(&a.slots[pos], kEmpty, ((unsigned long long)tag << 32) | i);
                if (v == kEmpty) {  // first of its state
                    if (written) {
                        ++n_keep;
                        deg += (a.child.meta[i] >> 10) & 0x1FFFu;
                    } else {
                        ++n_unv;
                    }
                    break;
                }
                if ((uint32_t)(v >> 32) == tag) {
                    const uint64_t jrow = (uint32_t)v;
                    // a row without its state written cannot be compared: the
                    // level is then decided from the lower bound, or run again
                    if (!written || jrow >= row_cap) {
                        if (written) a.child.meta[i] = 0u;
                        break;
                    }
                    if (same_state(a.child, Mpad, W, i, jrow)) {  // a later copy
                        a.child.meta[i] = 0u;
                        break;
                    }
                }
                pos = (pos + 1) & a.slot_mask;
            }
        }
        if (__any_sync(FULL, fatal)) break;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        deg += __shfl_xor_sync(FULL, deg, off);
        n_unv += __shfl_xor_sync(FULL, n_unv, off);
        n_keep += __shfl_xor_sync(FULL, n_keep, off);
    }
    if (lane == 0) {
        s_keep[wid] = n_keep;
        s_deg[wid] = deg;
        s_unv[wid] = n_unv;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long k = 0, d = 0, u = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            k += s_keep[w];
            d += s_deg[w];
            u += s_unv[w];
        }
        if (k) atomicAdd(&a.ctr[C_NEXT], k);
        if (d) atomicAdd(&a.ctr[C_DEGSUM], d);
        if (u) atomicAdd(&a.ctr[C_UNV], u);
    }
}

// Surviving rows [0, n) of an arena (meta != 0: every state has |U| >= 1)
// appended to a list, for the passes that sample or order a frontier.
__global__ void live_list_kernel(const uint32_t *meta, int64_t n, uint32_t *live, unsigned long long *count)
{
    const int lane = threadIdx.x & 31;
    for (int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll; i0 < n;
         i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + lane;
        const bool keep = i < n && meta[i] != 0u;
        const unsigned m = __ballot_sync(FULL, keep);
        unsigned long long base = 0;
        if (lane == 0 && m) base = atomicAdd(count, (unsigned long long)__popc(m));
        base = __shfl_sync(FULL, base, 0);
        if (keep) live[base + __popc(m & ((1u << lane) - 1u))] = (uint32_t)i;
    }
}

__global__ void dedup_advance_kernel(unsigned long long *ctr) { ctr[C_DEDUP_BEGIN] = ctr[C_WRITTEN]; }

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

// shared memory of one minimality warp: basis 64x64, columns 64, pivots 64, row map 32
constexpr int kAcceptWarpWords = 64 * 64 + 64 + 64 + 32;

// Minimality test of the candidates [cand_begin, cand_end) by the warps
// gw = 0 .. nw-1; ws: this warp's shared-memory scratch (kAcceptWarpWords).
__device__ void accept_range(const NetView &nv, const AcceptArgs &a, uint32_t *ws, int64_t gw, int64_t nw)
{
    const int lane = threadIdx.x & 31;
    const int W = nv.W;
    uint32_t *basis = ws;
    int *cols = reinterpret_cast<int *>(ws + 64 * 64);
    int *pivcol = cols + 64;
    uint32_t *rowmap = reinterpret_cast<uint32_t *>(pivcol + 64);
    const uint32_t *bl = nv.blob;
    unsigned long long n_acc = 0;
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
                if (a.rcols) {
                    uint16_t *lst = a.rcols + (size_t)idx * kRcolStride;
                    for (int j = lane; j < n; j += 32) lst[1 + j] = (uint16_t)cols[j];
                    if (lane == 0) lst[0] = (uint16_t)n;
                }
            } else if (lane == 0) {
                atomicOr(&a.ctr[C_ERR], (unsigned long long)ERR_RES_CAP);
            }
            ++n_acc;
        }
        __syncwarp();
    }
    if (lane == 0 && n_acc) atomicAdd(&a.ctr[C_RES], n_acc);
}

__global__ void __launch_bounds__(kAcceptWarps * 32) accept_kernel(NetView nv, AcceptArgs a)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int wid = threadIdx.x >> 5;
    if (a.dev_range) {
        // the expansion launches before this one have finished: the range is stable
        a.cand_begin = (int64_t)a.ctr[C_ACC_BEGIN];
        const int64_t n = (int64_t)a.ctr[C_CAND_N];
        a.cand_end = n < a.cand_cap ? n : a.cand_cap;
    }
    accept_range(nv, a, smem + wid * kAcceptWarpWords, (int64_t)blockIdx.x * kAcceptWarps + wid,
                 (int64_t)gridDim.x * kAcceptWarps);
}

__global__ void accept_advance_kernel(unsigned long long *ctr, int64_t cand_cap)
{
    const unsigned long long n = ctr[C_CAND_N];
    ctr[C_ACC_BEGIN] = n < (unsigned long long)cand_cap ? n : (unsigned long long)cand_cap;
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
                                   uint64_t *bres, unsigned long long *band)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * W) return;
    const int w = (int)(i % W);
    const int64_t r = i / W;
    for (uint64_t x = res[i]; x; x &= x - 1) {
        const int k = w * 64 + __ffsll((long long)x) - 1;
        const int64_t pos = (int64_t)bptr[k] + atomicAdd(&bfill[k], 1);
        if (W > 2) {
            reinterpret_cast<int32_t *>(bres)[pos] = (int32_t)r;
        } else {
            for (int v = 0; v < W; ++v) {
                bres[pos * W + v] = res[r * W + v];
                // intersection of the results containing k
                if (band) atomicAnd(&band[(size_t)k * W + v], (unsigned long long)res[r * W + v]);
            }
        }
    }
}

// The superset rule's sentinel index (W <= 2, N <= 128): for each result E
// its two columns with the fewest results, (m1, m2), ties by column; for each
// k in E the sentinel is m1, or m2 when k = m1.
__device__ __forceinline__ void result_sentinels(const uint64_t *E, int W, const int32_t *bcnt, int &m1, int &m2)
{
    m1 = m2 = -1;
    long long k1 = 0x7FFFFFFFFFFFFFFFll, k2 = 0x7FFFFFFFFFFFFFFFll;
    for (int w = 0; w < W; ++w)
        for (uint64_t x = E[w]; x; x &= x - 1) {
            const int c = w * 64 + __ffsll((long long)x) - 1;
            const long long key = ((long long)bcnt[c] << 16) | c;
            if (key < k1) {
                k2 = k1;
                m2 = m1;
                k1 = key;
                m1 = c;
            } else if (key < k2) {
                k2 = key;
                m2 = c;
            }
        }
}

__global__ void sentinel_count_kernel(const uint64_t *res, int64_t n, int W, int N, const int32_t *bcnt, int32_t *ccnt,
                                      uint32_t *csingle)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const uint64_t *E = res + (size_t)r * W;
    int m1, m2;
    result_sentinels(E, W, bcnt, m1, m2);
    if (m2 < 0) {  // a one-column result: every child adding that column contains it
        if (m1 >= 0) csingle[m1] = 1u;
        return;
    }
    for (int w = 0; w < W; ++w)
        for (uint64_t x = E[w]; x; x &= x - 1) {
            const int k = w * 64 + __ffsll((long long)x) - 1;
            atomicAdd(&ccnt[(size_t)k * N + (k == m1 ? m2 : m1)], 1);
        }
}

__global__ void sentinel_scan_kernel(const int32_t *ccnt, int cells, int32_t *cptr)
{
    // one CTA of 1024 threads: exclusive scan over the cells
    __shared__ int32_t part[1024];
    const int per = (cells + 1023) / 1024;
    const int beg = threadIdx.x * per;
    int32_t s = 0;
    for (int i = beg; i < beg + per && i < cells; ++i) s += ccnt[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int32_t run = part[threadIdx.x] - s;
    for (int i = beg; i < beg + per && i < cells; ++i) {
        cptr[i] = run;
        run += ccnt[i];
    }
    if (threadIdx.x == 1023) cptr[cells] = part[1023];
}

__global__ void sentinel_mask_kernel(const int32_t *ccnt, int N, int W, uint64_t *cne)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    for (int w = 0; w < W; ++w) {
        uint64_t m = 0;
        for (int b = 0; b < 64 && w * 64 + b < N; ++b)
            if (ccnt[(size_t)k * N + w * 64 + b] > 0) m |= 1ull << b;
        cne[(size_t)k * W + w] = m;
    }
}

__global__ void sentinel_fill_kernel(const uint64_t *res, int64_t n, int W, int N, const int32_t *bcnt,
                                     const int32_t *cptr, int32_t *cfill, uint64_t *cent)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const uint64_t *E = res + (size_t)r * W;
    int m1, m2;
    result_sentinels(E, W, bcnt, m1, m2);
    if (m2 < 0) return;
    for (int w = 0; w < W; ++w)
        for (uint64_t x = E[w]; x; x &= x - 1) {
            const int k = w * 64 + __ffsll((long long)x) - 1;
            const size_t cell = (size_t)k * N + (k == m1 ? m2 : m1);
            const int32_t pos = cptr[cell] + atomicAdd(&cfill[cell], 1);
            for (int v = 0; v < W; ++v) cent[(size_t)pos * W + v] = E[v];
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

// ---------------------------------------------------------------------------
// Batched traversal: one persistent launch over many (network, target) jobs.
// Each CTA pulls jobs from a device queue and runs the whole level loop of a
// job (seed, expand, minimality test, buckets, sorted output) with CTA
// barriers between the steps, in its own slice of a scratch pool.  The level
// decisions (truncation, cap, counters) are those of the single-job host loop.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint64_t next_pow2_dev(uint64_t x)
{
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// CTA-level bucket rebuild over results [0, n_res)
__device__ void cta_buckets(const NetView &nv, const uint64_t *res, int64_t n_res, int32_t *bcnt, int32_t *bptr,
                            int32_t *bfill, uint64_t *bres)
{
    const int W = nv.W;
    for (int i = threadIdx.x; i < nv.N; i += blockDim.x) {
        bcnt[i] = 0;
        bfill[i] = 0;
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n_res * W; i += blockDim.x) {
        const int w = (int)(i % W);
        for (uint64_t x = res[i]; x; x &= x - 1) atomicAdd(&bcnt[w * 64 + __ffsll((long long)x) - 1], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t run = 0;
        for (int k = 0; k < nv.N; ++k) {
            bptr[k] = run;
            run += bcnt[k];
        }
        bptr[nv.N] = run;
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n_res * W; i += blockDim.x) {
        const int w = (int)(i % W);
        const int64_t r = i / W;
        for (uint64_t x = res[i]; x; x &= x - 1) {
            const int k = w * 64 + __ffsll((long long)x) - 1;
            const int64_t pos = (int64_t)bptr[k] + atomicAdd(&bfill[k], 1);
            if (W > 2)
                reinterpret_cast<int32_t *>(bres)[pos] = (int32_t)r;
            else
                for (int v = 0; v < W; ++v) bres[pos * W + v] = res[r * W + v];
        }
    }
    __syncthreads();
}

// CTA-level sort of results [0, n) into out (first n_keep rows)
__device__ void cta_sort(const uint64_t *res, int64_t n, int W, uint32_t *idx, uint64_t *out, int64_t n_keep)
{
    if (n <= 0 || n_keep <= 0) return;
    const int64_t n2 = (int64_t)next_pow2_dev((uint64_t)n);
    for (int64_t i = threadIdx.x; i < n2; i += blockDim.x) idx[i] = i < n ? (uint32_t)i : 0xFFFFFFFFu;
    __syncthreads();
    for (int64_t k = 2; k <= n2; k <<= 1)
        for (int64_t j = k >> 1; j > 0; j >>= 1) {
            for (int64_t i = threadIdx.x; i < n2; i += blockDim.x) {
                const int64_t l = i ^ j;
                if (l <= i) continue;
                const uint32_t x = idx[i], y = idx[l];
                const bool up = (i & k) == 0;
                if (support_greater(res, W, x, y) == up) {
                    idx[i] = y;
                    idx[l] = x;
                }
            }
            __syncthreads();
        }
    for (int64_t i = threadIdx.x; i < n_keep * W; i += blockDim.x) out[i] = res[(size_t)idx[i / W] * W + i % W];
    __syncthreads();
}

template <int G, int CPL>
__device__ void run_job(const BatchArgs &ba, const BatchJob &job, char *slice, uint32_t *sm)
{
    constexpr int EPL = G * CPL / 8;  // seed layout: Mpad = 32 EPL = 4 G CPL
    const NetView &nv = job.nv;
    unsigned long long *ctr = job.ctr;
    const int nwarps = blockDim.x >> 5;
    const int wid = threadIdx.x >> 5;
    const BatchLayout &L = ba.layout;
    __shared__ unsigned long long sh[C_COUNT];

    LevelArgs a{};
    a.slots = reinterpret_cast<unsigned long long *>(slice + L.o_slots);
    a.cslots = reinterpret_cast<unsigned long long *>(slice + L.o_cslots);
    a.cslot_mask = L.cslot_cap - 1;
    a.cand = reinterpret_cast<uint64_t *>(slice + L.o_cand);
    a.cand_cap = L.cand_cap;
    a.res = reinterpret_cast<const uint64_t *>(slice + L.o_res);
    a.bptr = reinterpret_cast<const int32_t *>(slice + L.o_bptr);
    a.bres = reinterpret_cast<const uint64_t *>(slice + L.o_bres);
    a.bids = reinterpret_cast<const int32_t *>(slice + L.o_bres);
    a.rcols = nv.W > 2 ? reinterpret_cast<const uint16_t *>(slice + L.o_rcols) : nullptr;
    a.max_len = job.max_len;
    a.max_sec = ba.max_sec;
    a.ctr = ctr;
    auto arena = [&](int i) {
        Arena r{};
        r.U = reinterpret_cast<uint64_t *>(slice + L.o_U[i]);
        r.B = reinterpret_cast<int32_t *>(slice + L.o_B[i]);
        r.meta = reinterpret_cast<uint32_t *>(slice + L.o_meta[i]);
        r.cap = L.cap;
        return r;
    };
    AcceptArgs acc{};
    acc.cand = a.cand;
    acc.res = reinterpret_cast<uint64_t *>(slice + L.o_res);
    acc.res_cap = L.res_cap;
    acc.rcols = nv.W > 2 ? reinterpret_cast<uint16_t *>(slice + L.o_rcols) : nullptr;
    acc.ctr = ctr;
    int32_t *bcnt = reinterpret_cast<int32_t *>(slice + L.o_bcnt);
    int32_t *bfill = reinterpret_cast<int32_t *>(slice + L.o_bfill);
    int32_t *bptr = reinterpret_cast<int32_t *>(slice + L.o_bptr);
    uint64_t *bres = reinterpret_cast<uint64_t *>(slice + L.o_bres);

    for (uint64_t i = threadIdx.x; i < L.cslot_cap; i += blockDim.x) a.cslots[i] = kEmpty;
    for (int i = threadIdx.x; i <= nv.N; i += blockDim.x) bptr[i] = 0;
    __syncthreads();
    auto read_ctr = [&]() {
        __syncthreads();
        for (int i = threadIdx.x; i < C_COUNT; i += blockDim.x) sh[i] = __ldcg(&ctr[i]);
        __syncthreads();
    };
    auto set_ctr = [&](int i, unsigned long long v) {
        if (threadIdx.x == 0) ctr[i] = v;
    };
    const int ERRMASK = ERR_TIMEOUT | ERR_CAND_CAP | ERR_RES_CAP | ERR_TABLE_FULL | ERR_PRIMES | ERR_LEN |
                        ERR_WATCHDOG | ERR_BOUNDS;

    // level 0: seeds, then the minimality test of balanced seeds
    int cur = 0;
    a.level = 0;
    a.child = arena(cur);
    seed_range<EPL>(nv, a, job.target, wid, nwarps);
    read_ctr();
    if (sh[C_ERR] & ERRMASK) return;
    acc.cand_begin = 0;
    acc.cand_end = (int64_t)sh[C_CAND_N];
    if (wid < kAcceptWarps) accept_range(nv, acc, sm + wid * kAcceptWarpWords, wid, kAcceptWarps);
    read_ctr();
    if (sh[C_ERR] & ERRMASK) return;
    int64_t cand_done = (int64_t)sh[C_CAND_N];
    int64_t res_n = (int64_t)min(sh[C_RES_N], (unsigned long long)L.res_cap);
    int64_t n_front = (int64_t)sh[C_NEXT];
    uint64_t deg_sum = sh[C_DEGSUM];
    unsigned long long status = 0, frontier = 0, frontier_max = 0, levels = 1;
    bool stop = false;
    if (ba.max_frontier > 0 && n_front > ba.max_frontier) {
        status |= EFM_TRUNCATED;
        stop = true;
    } else {
        frontier += n_front;
        frontier_max = max(frontier_max, (unsigned long long)n_front);
        if (ba.max_results > 0 && (int64_t)sh[C_RES] >= ba.max_results) {
            status |= EFM_CAPPED;
            stop = true;
        }
    }
    int64_t built_for = 0;
    for (int level = 1; !stop && n_front > 0; ++level) {
        if (level > a.max_len + a.max_sec + 1) {
            if (threadIdx.x == 0) atomicOr(&ctr[C_ERR], (unsigned long long)ERR_WATCHDOG);
            return;
        }
        if (res_n != built_for) {
            cta_buckets(nv, acc.res, res_n, bcnt, bptr, bfill, bres);
            built_for = res_n;
        }
        const uint64_t bound = min(deg_sum, (uint64_t)L.cap);
        const uint64_t nslots = min(L.slot_cap, next_pow2_dev(2 * bound + 64 * (uint64_t)nwarps));
        for (uint64_t i = threadIdx.x; i < nslots; i += blockDim.x) a.slots[i] = kEmpty;
        set_ctr(C_NEXT, 0);
        set_ctr(C_DEGSUM, 0);
        __syncthreads();
        a.par = arena(cur);
        a.n_par = n_front;
        a.child = arena(cur ^ 1);
        a.slot_mask = nslots - 1;
        a.level = level;
        a.cpw = (int)min((int64_t)ba.tile, max((int64_t)1, (n_front + nwarps - 1) / nwarps));
        expand_range<G, CPL>(nv, a, nv.blob, reinterpret_cast<char *>(sm) + (size_t)wid * BatchShape<G, CPL>::BYTES,
                             wid, nwarps);
        read_ctr();
        if (sh[C_ERR] & ERRMASK) return;
        acc.cand_begin = cand_done;
        acc.cand_end = (int64_t)sh[C_CAND_N];
        if (wid < kAcceptWarps) accept_range(nv, acc, sm + wid * kAcceptWarpWords, wid, kAcceptWarps);
        read_ctr();
        if (sh[C_ERR] & ERRMASK) return;
        cand_done = (int64_t)sh[C_CAND_N];
        res_n = (int64_t)min(sh[C_RES_N], (unsigned long long)L.res_cap);
        n_front = (int64_t)sh[C_NEXT];
        deg_sum = sh[C_DEGSUM];
        levels = level + 1;
        cur ^= 1;
        if (ba.max_frontier > 0 && n_front > ba.max_frontier) {
            status |= EFM_TRUNCATED;
            break;
        }
        frontier += n_front;
        frontier_max = max(frontier_max, (unsigned long long)n_front);
        if (ba.max_results > 0 && (int64_t)sh[C_RES] >= ba.max_results) {
            status |= EFM_CAPPED;
            break;
        }
    }
    if ((int64_t)sh[C_RES_N] > L.res_cap) {
        if (threadIdx.x == 0) atomicOr(&ctr[C_ERR], (unsigned long long)ERR_RES_CAP);
        return;
    }
    const int64_t n_keep = ba.max_results > 0 ? min(res_n, ba.max_results) : res_n;
    cta_sort(acc.res, res_n, nv.W, reinterpret_cast<uint32_t *>(slice + L.o_sort), job.out, n_keep);
    if (sh[C_OVF]) status |= EFM_OVERFLOW_DROPPED;
    set_ctr(C_LEVELS, levels);
    set_ctr(C_FRONTIER, frontier);
    set_ctr(C_FRONTIER_MAX, frontier_max);
    set_ctr(C_STATUS, status);
    set_ctr(C_OUT_N, (unsigned long long)n_keep);
    set_ctr(C_DONE, 1ull);
}

__global__ void __launch_bounds__(kBatchThreads) batch_kernel(BatchArgs ba)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ int s_job;
    char *slice = ba.pool + (size_t)blockIdx.x * ba.layout.slice_bytes;
    const int chunk = ba.chunk > 0 ? ba.chunk : 1;
    for (;;) {
        if (threadIdx.x == 0) s_job = (int)atomicAdd(ba.queue, (unsigned)chunk);
        __syncthreads();
        const int q0 = s_job;
        __syncthreads();
        if (q0 >= ba.n_jobs) break;
        for (int qi = q0; qi < q0 + chunk && qi < ba.n_jobs; ++qi) {
            const BatchJob &job = ba.jobs[ba.order[qi]];
            switch (job.nv.EPL) {
            case 1: run_job<4, 2>(ba, job, slice, smem); break;
            case 2: run_job<8, 2>(ba, job, slice, smem); break;
            case 4: run_job<16, 2>(ba, job, slice, smem); break;
            case 8: run_job<32, 2>(ba, job, slice, smem); break;
            default:
                if (threadIdx.x == 0) atomicOr(&job.ctr[C_ERR], (unsigned long long)ERR_LEN);
                break;
            }
            __syncthreads();
        }
    }
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


// The narrow kernel reads the static network through L1 rather than staging
// it: at four blocks per SM a staged copy per block would take shared memory
// that L1 then lacks for the parents' rows (measured: about 3 % faster).
inline bool narrow_staged(const NetView &) { return false; }

template <int G>
cudaError_t launch_generate_narrow_t(const NetView &nv, const LevelArgs &a, int grid, cudaStream_t s)
{
    const bool staged = narrow_staged(nv);
    const size_t sm = (size_t)(staged ? nv.blob_words : 0) * 4 + 16;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(generate_narrow_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kStageLimitBytes + 16);
        attr_set = true;
    }
    generate_narrow_kernel<G><<<grid, kExpandWarps * 32, sm, s>>>(nv, a, staged ? 1 : 0);
    return cudaGetLastError();
}

template <int G>
int generate_narrow_grid_t(const NetView &nv, int sm_count)
{
    const bool staged = narrow_staged(nv);
    const size_t sm = (size_t)(staged ? nv.blob_words : 0) * 4 + 16;
    cudaFuncSetAttribute(generate_narrow_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStageLimitBytes + 16);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, generate_narrow_kernel<G>, kExpandWarps * 32, sm) !=
            cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return sm_count * per_sm;
}

// the generic kernel stages the whole static network when it fits, else its
// sparse tables when those fit (the dense columns stay in global memory)
inline int generic_staging(const NetView &nv)
{
    if (nv.blob_words * 4 <= kStageLimitBytes) return 1;
    if ((nv.o_hbits - nv.o_consptr) * 4 <= kStageSparseLimitBytes && nv.o_consptr % 4 == 0 && nv.o_hbits % 4 == 0)
        return 2;
    return 0;
}
inline size_t generic_smem(const NetView &nv, int mode)
{
    return (size_t)(mode == 1 ? nv.blob_words : (mode == 2 ? nv.o_hbits - nv.o_consptr : 0)) * 4 + 16;
}

template <int G, int CPL>
cudaError_t launch_generate_t(const NetView &nv, const LevelArgs &a, int grid, cudaStream_t s)
{
    const int mode = generic_staging(nv);
    const size_t sm = generic_smem(nv, mode);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(generate_kernel<G, CPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (kStageLimitBytes > kStageSparseLimitBytes ? kStageLimitBytes : kStageSparseLimitBytes) + 16);
        attr_set = true;
    }
    generate_kernel<G, CPL><<<grid, kExpandWarps * 32, sm, s>>>(nv, a, mode);
    return cudaGetLastError();
}

template <int G, int CPL>
int generate_grid_t(const NetView &nv, int sm_count)
{
    const size_t sm = generic_smem(nv, generic_staging(nv));
    cudaFuncSetAttribute(generate_kernel<G, CPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (kStageLimitBytes > kStageSparseLimitBytes ? kStageLimitBytes : kStageSparseLimitBytes) + 16);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, generate_kernel<G, CPL>, kExpandWarps * 32, sm) !=
            cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return sm_count * per_sm;
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

// (lanes per child, 16-byte chunks per lane) for each row width Mpad = 32 EPL
#define EFM_GROUP_DISPATCH(EPLV, CALL) \
    switch (EPLV) {                    \
    case 1: return CALL(4, 2);         \
    case 2: return CALL(8, 2);         \
    case 4: return CALL(16, 2);        \
    case 8: return CALL(32, 2);        \
    case 16: return CALL(32, 4);       \
    case 28: return CALL(32, 7);       \
    case 32: return CALL(32, 8);       \
    default: break;                    \
    }


cudaError_t launch_generate(const NetView &nv, const LevelArgs &a, int grid, cudaStream_t s)
{
    // narrow networks: incremental summaries (needs the arenas' summary arrays)
    if (nv.narrow && a.par.sum && a.child.sum) {
        if (nv.EPL == 1) return launch_generate_narrow_t<4>(nv, a, grid, s);
        if (nv.EPL == 2) return launch_generate_narrow_t<8>(nv, a, grid, s);
    }
#define CALL_GEN(G, C) launch_generate_t<G, C>(nv, a, grid, s)
    EFM_GROUP_DISPATCH(nv.EPL, CALL_GEN)
#undef CALL_GEN
    return cudaErrorInvalidValue;
}

int generate_grid(const NetView &nv, int sm_count)
{
    if (nv.narrow && nv.EPL == 1) return generate_narrow_grid_t<4>(nv, sm_count);
    if (nv.narrow && nv.EPL == 2) return generate_narrow_grid_t<8>(nv, sm_count);
#define CALL_GGRID(G, C) generate_grid_t<G, C>(nv, sm_count)
    EFM_GROUP_DISPATCH(nv.EPL, CALL_GGRID)
#undef CALL_GGRID
    return sm_count;
}

cudaError_t launch_live_list(const uint32_t *meta, int64_t n, uint32_t *live, unsigned long long *count,
                             int sm_count, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)sm_count * 8);
    live_list_kernel<<<(unsigned)blocks, 256, 0, s>>>(meta, n, live, count);
    return cudaGetLastError();
}

cudaError_t launch_settle(const NetView &nv, const LevelArgs &a, int sm_count, cudaStream_t s)
{
    if (!(nv.narrow && a.par.sum && a.child.sum && a.slow)) return cudaSuccess;
    if (nv.EPL == 1)
        settle_kernel<4><<<sm_count * 4, kExpandWarps * 32, 0, s>>>(nv, a);
    else if (nv.EPL == 2)
        settle_kernel<8><<<sm_count * 4, kExpandWarps * 32, 0, s>>>(nv, a);
    return cudaGetLastError();
}

cudaError_t launch_prune_rows(const NetView &nv, const LevelArgs &a, int sm_count, cudaStream_t s)
{
    if (!(nv.narrow && a.par.sum && a.child.sum && a.wrec && nv.W <= 2 && a.cptr)) return cudaSuccess;
    prune_rows_kernel<<<sm_count * 8, 256, 0, s>>>(nv, a);
    return cudaGetLastError();
}

cudaError_t launch_write_rows(const NetView &nv, const LevelArgs &a, int sm_count, cudaStream_t s)
{
    if (!(nv.narrow && a.par.sum && a.child.sum && a.wrec)) return cudaSuccess;
    // G lanes per row of 32 EPL entries, CPL 16-byte chunks each
    if (nv.EPL == 1)
        write_rows_kernel<4, 2><<<sm_count * 8, 256, 0, s>>>(nv, a);
    else if (nv.EPL == 2)
        write_rows_kernel<8, 2><<<sm_count * 8, 256, 0, s>>>(nv, a);
    return cudaGetLastError();
}

cudaError_t launch_dedup(const LevelArgs &a, int Mpad, int W, int sm_count, cudaStream_t s)
{
    dedup_kernel<<<sm_count * 8, 256, 0, s>>>(a, Mpad, W);
    dedup_advance_kernel<<<1, 1, 0, s>>>(a.ctr);
    return cudaGetLastError();
}


cudaError_t launch_accept_new(const NetView &nv, const AcceptArgs &a, int sm_count, cudaStream_t s)
{
    const size_t sm = (size_t)kAcceptWarps * kAcceptWarpWords * 4;
    cudaFuncSetAttribute(accept_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    AcceptArgs d = a;
    d.dev_range = 1;
    accept_kernel<<<sm_count * 2, kAcceptWarps * 32, sm, s>>>(nv, d);
    accept_advance_kernel<<<1, 1, 0, s>>>(a.ctr, a.cand_cap);
    return cudaGetLastError();
}

cudaError_t launch_accept(const NetView &nv, const AcceptArgs &a, cudaStream_t s)
{
    const int64_t n = a.cand_end - a.cand_begin;
    if (n <= 0) return cudaSuccess;
    const size_t sm = (size_t)kAcceptWarps * kAcceptWarpWords * 4;
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
                           int32_t *bfill, uint64_t *bres, uint64_t *band, cudaStream_t s)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(bcnt, 0, sizeof(int32_t) * (size_t)nv.N, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(bfill, 0, sizeof(int32_t) * (size_t)nv.N, s)) != cudaSuccess) return e;
    if (band && (e = cudaMemsetAsync(band, 0xFF, sizeof(uint64_t) * (size_t)nv.N * nv.W, s)) != cudaSuccess) return e;
    const int64_t items = n_res * nv.W;
    const int tb = 256;
    if (items > 0) bucket_count_kernel<<<(int)((items + tb - 1) / tb), tb, 0, s>>>(res, n_res, nv.W, bcnt);
    bucket_scan_kernel<<<1, 1024, 0, s>>>(bcnt, nv.N, bptr);
    if (items > 0)
        bucket_fill_kernel<<<(int)((items + tb - 1) / tb), tb, 0, s>>>(res, n_res, nv.W, bptr, bfill, bres,
                                                                      reinterpret_cast<unsigned long long *>(band));
    return cudaGetLastError();
}

cudaError_t launch_sentinel_index(const NetView &nv, const uint64_t *res, int64_t n_res, const int32_t *bcnt,
                                  int32_t *ccnt, int32_t *cfill, int32_t *cptr, uint64_t *cent, uint64_t *cne,
                                  uint32_t *csingle, cudaStream_t s)
{
    const int N = nv.N, W = nv.W;
    const size_t cells = (size_t)N * N;
    cudaError_t e;
    if ((e = cudaMemsetAsync(ccnt, 0, cells * 4, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(cfill, 0, cells * 4, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(csingle, 0, (size_t)N * 4, s)) != cudaSuccess) return e;
    const int tb = 256;
    if (n_res > 0)
        sentinel_count_kernel<<<(int)((n_res + tb - 1) / tb), tb, 0, s>>>(res, n_res, W, N, bcnt, ccnt, csingle);
    sentinel_scan_kernel<<<1, 1024, 0, s>>>(ccnt, (int)cells, cptr);
    sentinel_mask_kernel<<<(N + 127) / 128, 128, 0, s>>>(ccnt, N, W, cne);
    if (n_res > 0)
        sentinel_fill_kernel<<<(int)((n_res + tb - 1) / tb), tb, 0, s>>>(res, n_res, W, N, bcnt, cptr, cfill, cent);
    return cudaGetLastError();
}

__global__ void iota_kernel(uint32_t *perm, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) perm[i] = (uint32_t)i;
}

cudaError_t launch_walks(const NetView &nv, const LevelArgs &a, int target, uint64_t seed, int64_t n_walks, int sm_count,
                         cudaStream_t s)
{
    if (n_walks <= 0) return cudaSuccess;
    const int64_t want = (n_walks + kExpandWarps - 1) / kExpandWarps;
    const int grid = (int)std::min<int64_t>(want, (int64_t)sm_count * 8);
    switch (nv.EPL) {
#define EFM_WALK(E)                                                                       \
    case E:                                                                               \
        walk_kernel<E><<<grid, kExpandWarps * 32, 0, s>>>(nv, a, target, seed, n_walks); \
        break;
        EFM_WALK(1) EFM_WALK(2) EFM_WALK(4) EFM_WALK(8) EFM_WALK(16) EFM_WALK(28) EFM_WALK(32)
#undef EFM_WALK
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_seedset(const NetView &nv, const LevelArgs &a, const int32_t *cols, int n_cols, cudaStream_t s)
{
    switch (nv.EPL) {
#define EFM_SEEDSET(E)                                                \
    case E:                                                           \
        seedset_kernel<E><<<1, 32, 0, s>>>(nv, a, cols, n_cols);      \
        break;
        EFM_SEEDSET(1) EFM_SEEDSET(2) EFM_SEEDSET(4) EFM_SEEDSET(8) EFM_SEEDSET(16) EFM_SEEDSET(28) EFM_SEEDSET(32)
#undef EFM_SEEDSET
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_iota(uint32_t *perm, int64_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    iota_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(perm, n);
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

int batch_blocks_per_sm(int warps)
{
    int per_sm = 0;
    const size_t sm = batch_smem_bytes(warps);
    cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem_bytes(kBatchThreads / 32));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, warps * 32, sm) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return per_sm;
}

size_t batch_smem_bytes(int warps)
{
    // union of the expansion batches of all warps (largest row class) and the
    // minimality scratch of kAcceptWarps warps
    size_t ex = (size_t)BatchShape<4, 2>::BYTES;
    ex = ex > (size_t)BatchShape<8, 2>::BYTES ? ex : (size_t)BatchShape<8, 2>::BYTES;
    ex = ex > (size_t)BatchShape<16, 2>::BYTES ? ex : (size_t)BatchShape<16, 2>::BYTES;
    ex = ex > (size_t)BatchShape<32, 2>::BYTES ? ex : (size_t)BatchShape<32, 2>::BYTES;
    ex *= (size_t)warps;
    const size_t ac = (size_t)kAcceptWarps * kAcceptWarpWords * 4;
    return ex > ac ? ex : ac;
}

cudaError_t launch_batch(const BatchArgs &ba, int grid, int warps, cudaStream_t s)
{
    if (warps < kAcceptWarps || warps > kBatchThreads / 32) return cudaErrorInvalidValue;
    const size_t sm = batch_smem_bytes(warps);
    cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem_bytes(kBatchThreads / 32));
    batch_kernel<<<grid, warps * 32, sm, s>>>(ba);
    return cudaGetLastError();
}

}  // namespace efm
