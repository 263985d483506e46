// Host-only driver for efm::TopK (the first-K search's host bound), used by
// tests/test_host_logic.py.  stdin: K W, then batches "n" followed by n rows
// of W words; a batch of size -1 ends the input.  stdout after each batch:
// "pc" followed by the kth row (or nothing while fewer than K rows were
// seen), then the kept rows at the end.
#include <cstdio>
#include <vector>

#include "efm_topk.h"

int main()
{
    int K = 0, W = 0;
    if (std::scanf("%d %d", &K, &W) != 2 || K <= 0 || W <= 0) return 2;
    efm::TopK top;
    top.K = K;
    top.W = W;
    for (;;) {
        long long n = 0;
        if (std::scanf("%lld", &n) != 1) return 2;
        if (n < 0) break;
        std::vector<uint64_t> batch((size_t)n * W);
        for (auto &x : batch)
            if (std::scanf("%llu", reinterpret_cast<unsigned long long *>(&x)) != 1) return 2;
        top.add(batch.data(), n);
        std::printf("bound %d", top.pc);
        for (uint64_t x : top.kth) std::printf(" %llu", (unsigned long long)x);
        std::printf("\n");
    }
    const size_t rows = top.rows.size() / (size_t)W;
    for (size_t i = 0; i < rows; ++i) {
        std::printf("row");
        for (int w = 0; w < W; ++w) std::printf(" %llu", (unsigned long long)top.rows[i * W + w]);
        std::printf("\n");
    }
    return 0;
}
