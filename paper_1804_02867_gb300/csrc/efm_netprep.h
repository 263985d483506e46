// efm_netprep.h -- the loader's host work: validate S and build the static
// network the kernels read (Alg. 1 "convert S to the MG graph").  Plain C++
// (no CUDA), so the same code is compiled into the library and into a
// host-only test.
//
// Split columns (the direction of Def. 6): reaction j gives its forward
// column, then, if reversible, its reverse column (-S[:, j]) right after it.
// The blob packs, as 32-bit words:
//  - S_int by column: per column, its internal rows (ascending) with their
//    coefficients;
//  - per internal row, the columns consuming it (S_int < 0) and producing it
//    (S_int > 0), ascending, with |coefficient| (the O and I arrays of Def. 5);
//  - per column, its twin column (the other direction of the same reaction)
//    or -1;
//  - per internal row, the pivot keys (consumers << 16 | row) and
//    (producers << 16 | row);
//  - per column, ceil(log2(|S_int[:, k]|^2)) (for the Hadamard bound of the
//    minimality test);
//  - networks with at most 64 internal rows ("narrow"), for the expansion's
//    incremental state summaries: per internal row its rank in the order of
//    the positive and of the negative pivot keys; per rank the key; per row
//    a 64-bit constant R[m] of the linear row hash sum_m EF_m R[m] (mod 2^64);
//    per column the rank-space masks of its rows (positive and negative
//    orders), its row-space mask, sum_m S_int[m][k] R[m], max |S_int[m][k]|
//    and whether the gcd of its entries is 1;
//  - wide networks: per column, the lane masks of the rows it consumes and
//    of the rows it produces (the first-K length-cap rule);
//  - a dense column-major copy of S_int: N rows of Mpad = 32 EPL int32,
//    16-byte aligned.
// Entries are packed as (index << 20) | (coefficient & 0xFFFFF).
#pragma once
#include <stdint.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "../../include/efmgraph.h"

namespace efm {

inline uint32_t ent_pack(int idx, int32_t coef) { return ((uint32_t)idx << 20) | ((uint32_t)coef & 0xFFFFFu); }

constexpr int kNarrowRows = 64;  // internal rows of a network with state summaries
constexpr int kColxWords = 10;   // per-column summary words (narrow networks)

// Constant of internal row m in the linear row hash: the SplitMix64
// finaliser (Steele, Lea, Flood 2014) of 0x9E3779B97F4A7C15 * (m + 1).
inline uint64_t row_hash_constant(int m)
{
    uint64_t z = 0x9E3779B97F4A7C15ull * (uint64_t)(m + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// balance entries per lane for M internal rows (a row holds 32 EPL entries),
// -1 beyond EFM_MAX_INTERNAL
inline int pick_epl(int M)
{
    const int need = std::max(1, (M + 31) / 32);
    const int opts[] = {1, 2, 4, 8, 16, 28, 32};
    for (int o : opts)
        if (o >= need) return o;
    return -1;
}

struct NetPrep {
    int N = 0, M = 0, W = 0, EPL = 0, Mpad = 0;
    std::vector<int32_t> col_rxn;  // reaction of each split column
    std::vector<int8_t> col_dir;   // +1 forward, -1 reverse
    std::vector<uint32_t> blob;
    int o_colptr = 0, o_colent = 0, o_consptr = 0, o_consent = 0, o_prodptr = 0, o_prodent = 0;
    int o_twin = 0, o_keypos = 0, o_keyneg = 0, o_hbits = 0, o_dcols = 0;
    bool narrow = false;                            // M <= kNarrowRows: the sections below exist
    int o_rank = 0, o_keyr = 0, o_hrow = 0, o_colx = 0;
    int o_fixc = 0, o_fixp = 0;  // wide networks: per-column lane masks of consumed / produced rows (0: none)
    std::vector<int32_t> mptr;  // full S rows over split columns (seeds): [n_met + 1]
    std::vector<uint32_t> ment;  // packed (column, coefficient)
};

// Validate the CSR of S (rows = metabolites) and build the static network.
// Returns EFM_OK or EFM_EINVAL (malformed CSR, index out of range, duplicate
// entry in a row, zero or out-of-range coefficient, more than
// EFM_MAX_COLUMNS split columns or EFM_MAX_INTERNAL internal metabolites).
// flux_rows: the view of the subtractive traversal (Eq. 5), whose states
// carry their flux vector after the extra flux: a row holds M + N entries
// and the dense copy of column k is S_int[:, k] followed by the unit vector
// e_k (flux 1 on k); EFM_EUNSUPPORTED when M + N exceeds EFM_MAX_INTERNAL.
inline int prepare_network(int32_t n_met, int32_t n_rxn, const int32_t *row_ptr, const int32_t *col_idx,
                           const int32_t *coef, const uint8_t *reversible, const uint8_t *external, NetPrep &out,
                           bool flux_rows = false)
{
    if (n_met <= 0 || n_rxn <= 0 || !row_ptr || !reversible || !external) return EFM_EINVAL;
    if (row_ptr[0] != 0) return EFM_EINVAL;
    const int64_t nnz = row_ptr[n_met];
    if (nnz > 0 && (!col_idx || !coef)) return EFM_EINVAL;
    std::vector<int32_t> mark(n_rxn, -1);
    for (int m = 0; m < n_met; ++m) {
        if (row_ptr[m + 1] < row_ptr[m]) return EFM_EINVAL;
        for (int p = row_ptr[m]; p < row_ptr[m + 1]; ++p) {
            const int j = col_idx[p];
            if (j < 0 || j >= n_rxn) return EFM_EINVAL;
            if (coef[p] == 0 || coef[p] > EFM_MAX_COEF || coef[p] < -EFM_MAX_COEF) return EFM_EINVAL;
            if (mark[j] == m) return EFM_EINVAL;  // duplicate entry in a row
            mark[j] = m;
        }
    }
    // split columns
    std::vector<int> first_col(n_rxn);
    int N = 0;
    out.col_rxn.clear();
    out.col_dir.clear();
    for (int j = 0; j < n_rxn; ++j) {
        first_col[j] = N;
        out.col_rxn.push_back(j);
        out.col_dir.push_back(1);
        ++N;
        if (reversible[j]) {
            out.col_rxn.push_back(j);
            out.col_dir.push_back(-1);
            ++N;
        }
    }
    std::vector<int> int_row(n_met, -1);
    int M = 0;
    for (int m = 0; m < n_met; ++m)
        if (!external[m]) int_row[m] = M++;
    if (N > EFM_MAX_COLUMNS || M > EFM_MAX_INTERNAL || pick_epl(M) < 0) return EFM_EINVAL;
    const int EPL = flux_rows ? pick_epl(M + N) : pick_epl(M);
    if (EPL < 0) return EFM_EUNSUPPORTED;
    // S_int by column (rows ascending) and by internal row (columns ascending)
    std::vector<std::vector<std::pair<int, int32_t>>> col(N), cons(M), prod(M);
    std::vector<std::vector<std::pair<int, int32_t>>> metrow(n_met);
    for (int m = 0; m < n_met; ++m) {
        for (int p = row_ptr[m]; p < row_ptr[m + 1]; ++p) {
            const int j = col_idx[p];
            const int f = first_col[j];
            metrow[m].push_back({f, coef[p]});
            if (reversible[j]) metrow[m].push_back({f + 1, -coef[p]});
            if (int_row[m] < 0) continue;
            col[f].push_back({int_row[m], coef[p]});
            if (reversible[j]) col[f + 1].push_back({int_row[m], -coef[p]});
        }
    }
    std::vector<uint32_t> hbits(N, 0);
    for (int k = 0; k < N; ++k) {
        std::sort(col[k].begin(), col[k].end());
        uint64_t nsq = 0;
        for (auto &e : col[k]) {
            nsq += (uint64_t)((int64_t)e.second * e.second);
            if (e.second < 0) cons[e.first].push_back({k, -e.second});
            if (e.second > 0) prod[e.first].push_back({k, e.second});
        }
        hbits[k] = nsq <= 1 ? 0u : (uint32_t)(64 - __builtin_clzll(nsq - 1));
    }
    // blob assembly
    std::vector<uint32_t> &blob = out.blob;
    blob.clear();
    auto put_csr = [&](std::vector<std::vector<std::pair<int, int32_t>>> &lists, int &o_ptr, int &o_ent) {
        o_ptr = (int)blob.size();
        uint32_t acc = 0;
        for (auto &l : lists) {
            blob.push_back(acc);
            acc += (uint32_t)l.size();
        }
        blob.push_back(acc);
        o_ent = (int)blob.size();
        for (auto &l : lists)
            for (auto &e : l) blob.push_back(ent_pack(e.first, e.second));
    };
    put_csr(col, out.o_colptr, out.o_colent);
    // [o_consptr, o_hbits): the expansion's sparse tables (branch lists, twins,
    // keys), 16-byte aligned so that one bulk copy can stage them
    while (blob.size() % 4) blob.push_back(0);
    put_csr(cons, out.o_consptr, out.o_consent);
    put_csr(prod, out.o_prodptr, out.o_prodent);
    out.o_twin = (int)blob.size();
    for (int k = 0; k < N; ++k) {
        int tw = -1;
        if (k + 1 < N && out.col_rxn[k + 1] == out.col_rxn[k]) tw = k + 1;
        if (k > 0 && out.col_rxn[k - 1] == out.col_rxn[k]) tw = k - 1;
        blob.push_back((uint32_t)tw);
    }
    out.o_keypos = (int)blob.size();
    for (int r = 0; r < M; ++r) blob.push_back(((uint32_t)cons[r].size() << 16) | (uint32_t)r);
    out.o_keyneg = (int)blob.size();
    for (int r = 0; r < M; ++r) blob.push_back(((uint32_t)prod[r].size() << 16) | (uint32_t)r);
    while (blob.size() % 4) blob.push_back(0);
    out.o_hbits = (int)blob.size();
    for (int k = 0; k < N; ++k) blob.push_back(hbits[k]);
    out.narrow = M <= kNarrowRows && !flux_rows;
    out.o_rank = out.o_keyr = out.o_hrow = out.o_colx = 0;
    if (out.narrow) {
        // ranks of the rows in the positive / negative key orders
        std::vector<std::pair<uint32_t, int>> kp, kn;
        for (int r = 0; r < M; ++r) {
            kp.push_back({((uint32_t)cons[r].size() << 16) | (uint32_t)r, r});
            kn.push_back({((uint32_t)prod[r].size() << 16) | (uint32_t)r, r});
        }
        std::sort(kp.begin(), kp.end());
        std::sort(kn.begin(), kn.end());
        std::vector<int> rp(M), rn(M);
        for (int i = 0; i < M; ++i) {
            rp[kp[i].second] = i;
            rn[kn[i].second] = i;
        }
        out.o_rank = (int)blob.size();
        for (int r = 0; r < M; ++r) blob.push_back((uint32_t)rp[r] | ((uint32_t)rn[r] << 8));
        out.o_keyr = (int)blob.size();
        for (int i = 0; i < kNarrowRows; ++i) blob.push_back(i < M ? kp[i].first : 0xFFFFFFFFu);
        for (int i = 0; i < kNarrowRows; ++i) blob.push_back(i < M ? kn[i].first : 0xFFFFFFFFu);
        while (blob.size() % 2) blob.push_back(0);
        out.o_hrow = (int)blob.size();
        std::vector<uint64_t> R(M);
        for (int r = 0; r < M; ++r) {
            R[r] = row_hash_constant(r);
            blob.push_back((uint32_t)R[r]);
            blob.push_back((uint32_t)(R[r] >> 32));
        }
        out.o_colx = (int)blob.size();
        for (int k = 0; k < N; ++k) {
            uint64_t sp = 0, sn = 0, sr = 0, hc = 0;
            uint32_t smax = 0, g = 0;
            for (auto &e : col[k]) {
                sp |= 1ull << rp[e.first];
                sn |= 1ull << rn[e.first];
                sr |= 1ull << e.first;
                hc += (uint64_t)(int64_t)e.second * R[e.first];
                const uint32_t a = (uint32_t)(e.second < 0 ? -e.second : e.second);
                smax = std::max(smax, a);
                uint32_t x = g, y = a;
                while (y) {
                    const uint32_t t = x % y;
                    x = y;
                    y = t;
                }
                g = x;
            }
            const uint64_t w[4] = {sp, sn, sr, hc};
            for (uint64_t v : w) {
                blob.push_back((uint32_t)v);
                blob.push_back((uint32_t)(v >> 32));
            }
            blob.push_back(smax);
            blob.push_back(g == 1 ? 1u : 0u);
        }
    }
    // wide networks (not narrow, additive rows): the rows column k consumes
    // and produces, as lane masks of the expansion's row layout.  Lane l of
    // a group of G = min(32, 4 EPL) lanes holds the rows 4 (l + G i) + j for
    // i < 8 EPL / G and j < 4, at bit 4 i + j of its mask word.
    out.o_fixc = out.o_fixp = 0;
    if (!out.narrow && !flux_rows) {
        const int G = std::min(32, 4 * EPL);
        const int CPL = EPL * 8 / G;
        out.o_fixc = (int)blob.size();
        blob.resize(blob.size() + (size_t)2 * N * G, 0u);
        out.o_fixp = out.o_fixc + N * G;
        for (int k = 0; k < N; ++k)
            for (auto &e : col[k]) {
                const int chunk = e.first / 4, j = e.first % 4;
                const int l = chunk % G, i = chunk / G;
                if (i >= CPL) continue;  // unreachable: rows < 32 EPL
                const int o = (e.second < 0 ? out.o_fixc : out.o_fixp) + k * G + l;
                blob[o] |= 1u << (4 * i + j);
            }
    }
    while (blob.size() % 4) blob.push_back(0);
    // dense column-major copy of S_int (row k = column k over Mpad rows)
    out.o_dcols = (int)blob.size();
    blob.resize(blob.size() + (size_t)N * 32 * EPL, 0u);
    for (int k = 0; k < N; ++k) {
        for (auto &e : col[k]) blob[(size_t)out.o_dcols + (size_t)k * 32 * EPL + e.first] = (uint32_t)e.second;
        if (flux_rows) blob[(size_t)out.o_dcols + (size_t)k * 32 * EPL + M + k] = 1u;
    }
    out.mptr.assign(n_met + 1, 0);
    out.ment.clear();
    for (int m = 0; m < n_met; ++m) {
        for (auto &e : metrow[m]) out.ment.push_back(ent_pack(e.first, e.second));
        out.mptr[m + 1] = (int32_t)out.ment.size();
    }
    if (out.ment.empty()) out.ment.push_back(0);
    out.N = N;
    out.M = M;
    out.W = (N + 63) / 64;
    out.EPL = EPL;
    out.Mpad = 32 * EPL;
    return EFM_OK;
}

}  // namespace efm
