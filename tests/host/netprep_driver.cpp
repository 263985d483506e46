// Host-only driver for efm::prepare_network (the loader's host work), used by
// tests/test_host_logic.py.  stdin: n_met n_rxn, row_ptr[n_met + 1],
// nnz = row_ptr[n_met], col_idx[nnz], coef[nnz], reversible[n_rxn],
// external[n_met].  stdout: the status, then (on success) the static network
// decoded from the blob, one labelled line per item.
#include <cstdio>
#include <vector>

#include "efm_netprep.h"

static int idx_of(uint32_t e) { return (int)(e >> 20); }
static int coef_of(uint32_t e) { return (e & 0x80000u) ? (int)(e & 0xFFFFFu) - (1 << 20) : (int)(e & 0xFFFFFu); }

static void print_csr(const char *name, const std::vector<uint32_t> &blob, int o_ptr, int o_ent, int n)
{
    for (int i = 0; i < n; ++i) {
        std::printf("%s %d", name, i);
        for (uint32_t q = blob[o_ptr + i]; q < blob[o_ptr + i + 1]; ++q)
            std::printf(" %d:%d", idx_of(blob[o_ent + q]), coef_of(blob[o_ent + q]));
        std::printf("\n");
    }
}

int main()
{
    int n_met = 0, n_rxn = 0;
    if (std::scanf("%d %d", &n_met, &n_rxn) != 2) return 2;
    std::vector<int32_t> row_ptr(n_met + 1);
    for (auto &x : row_ptr)
        if (std::scanf("%d", &x) != 1) return 2;
    const int nnz = row_ptr[n_met];
    std::vector<int32_t> col_idx(nnz > 0 ? nnz : 1), coef(nnz > 0 ? nnz : 1);
    for (int i = 0; i < nnz; ++i)
        if (std::scanf("%d", &col_idx[i]) != 1) return 2;
    for (int i = 0; i < nnz; ++i)
        if (std::scanf("%d", &coef[i]) != 1) return 2;
    std::vector<uint8_t> rev(n_rxn), ext(n_met);
    for (auto &x : rev) {
        int v = 0;
        if (std::scanf("%d", &v) != 1) return 2;
        x = (uint8_t)v;
    }
    for (auto &x : ext) {
        int v = 0;
        if (std::scanf("%d", &v) != 1) return 2;
        x = (uint8_t)v;
    }
    efm::NetPrep p;
    const int rc = efm::prepare_network(n_met, n_rxn, row_ptr.data(), col_idx.data(), coef.data(), rev.data(),
                                        ext.data(), p);
    std::printf("status %d\n", rc);
    if (rc != 0) return 0;
    std::printf("shape %d %d %d %d %d\n", p.N, p.M, p.W, p.EPL, p.Mpad);
    for (int k = 0; k < p.N; ++k) std::printf("colmap %d %d %d\n", k, p.col_rxn[k], p.col_dir[k]);
    print_csr("col", p.blob, p.o_colptr, p.o_colent, p.N);
    print_csr("cons", p.blob, p.o_consptr, p.o_consent, p.M);
    print_csr("prod", p.blob, p.o_prodptr, p.o_prodent, p.M);
    for (int k = 0; k < p.N; ++k) std::printf("twin %d %d\n", k, (int)(int32_t)p.blob[p.o_twin + k]);
    for (int r = 0; r < p.M; ++r) std::printf("key %d %u %u\n", r, p.blob[p.o_keypos + r], p.blob[p.o_keyneg + r]);
    for (int k = 0; k < p.N; ++k) std::printf("hbits %d %u\n", k, p.blob[p.o_hbits + k]);
    std::printf("narrow %d\n", p.narrow ? 1 : 0);
    if (p.narrow) {
        auto u64 = [&](int o) { return (unsigned long long)p.blob[o] | ((unsigned long long)p.blob[o + 1] << 32); };
        for (int r = 0; r < p.M; ++r)
            std::printf("rank %d %u %u\n", r, p.blob[p.o_rank + r] & 0xFFu, (p.blob[p.o_rank + r] >> 8) & 0xFFu);
        for (int i = 0; i < efm::kNarrowRows; ++i)
            std::printf("keyr %d %u %u\n", i, p.blob[p.o_keyr + i], p.blob[p.o_keyr + efm::kNarrowRows + i]);
        for (int r = 0; r < p.M; ++r) std::printf("hrow %d %llu\n", r, u64(p.o_hrow + 2 * r));
        for (int k = 0; k < p.N; ++k) {
            const int o = p.o_colx + efm::kColxWords * k;
            std::printf("colx %d %llu %llu %llu %llu %u %u\n", k, u64(o), u64(o + 2), u64(o + 4), u64(o + 6),
                        p.blob[o + 8], p.blob[o + 9]);
        }
        std::printf("align64 %d %d\n", p.o_hrow % 2, p.o_colx % 2);
    }
    std::printf("fixtab %d\n", p.o_fixc > 0 ? 1 : 0);
    if (p.o_fixc > 0) {
        const int G = p.EPL >= 8 ? 32 : 4 * p.EPL;
        for (int k = 0; k < p.N; ++k)
            for (int l = 0; l < G; ++l)
                std::printf("fix %d %d %u %u\n", k, l, p.blob[p.o_fixc + k * G + l], p.blob[p.o_fixp + k * G + l]);
    }
    std::printf("dense_offset_mod4 %d\n", p.o_dcols % 4);
    for (int k = 0; k < p.N; ++k) {
        std::printf("dense %d", k);
        for (int r = 0; r < p.Mpad; ++r) std::printf(" %d", (int)(int32_t)p.blob[(size_t)p.o_dcols + (size_t)k * p.Mpad + r]);
        std::printf("\n");
    }
    for (int m = 0; m < n_met; ++m) {
        std::printf("met %d", m);
        for (int q = p.mptr[m]; q < p.mptr[m + 1]; ++q) std::printf(" %d:%d", idx_of(p.ment[q]), coef_of(p.ment[q]));
        std::printf("\n");
    }
    return 0;
}
