// efm_topk.h -- host side of the first-K search: the K smallest supports
// seen so far in the output order (|U|, then the ascending column list).
// Plain C++ (no CUDA), so the same code is compiled into the library and
// into a host-only test.
#pragma once
#include <stdint.h>

#include <algorithm>
#include <vector>

namespace efm {

// Supports are rows of W uint64 words (column k at bit k % 64 of word
// k / 64).  add() appends a batch; once K rows were seen, only the K
// smallest are kept, kth is the largest of them and pc its size: a support
// that follows kth cannot be among the K smallest.
struct TopK {
    int K = 0, W = 0;
    std::vector<uint64_t> rows;  // at most K rows once K were found
    int pc = 0;                  // |U| of the K-th (0 while fewer than K)
    std::vector<uint64_t> kth;

    static int popc(const uint64_t *r, int W)
    {
        int c = 0;
        for (int w = 0; w < W; ++w) c += __builtin_popcountll(r[w]);
        return c;
    }
    static bool less(const uint64_t *x, const uint64_t *y, int W)
    {
        const int cx = popc(x, W), cy = popc(y, W);
        if (cx != cy) return cx < cy;
        for (int w = 0; w < W; ++w) {
            const uint64_t d = x[w] ^ y[w];
            if (d) return (x[w] & (d & (~d + 1))) != 0;
        }
        return false;
    }
    // rows: supports (W words each); a support already kept counts once, so
    // the K kept rows are the K smallest distinct supports seen
    void add(const uint64_t *r, int64_t n)
    {
        rows.insert(rows.end(), r, r + (size_t)n * W);
        const int64_t have = (int64_t)(rows.size() / W);
        std::vector<int64_t> idx((size_t)have);
        for (int64_t i = 0; i < have; ++i) idx[i] = i;
        const uint64_t *base = rows.data();
        const int Wl = W;
        std::sort(idx.begin(), idx.end(), [&](int64_t i, int64_t j) { return less(base + i * Wl, base + j * Wl, Wl); });
        std::vector<uint64_t> keep;
        keep.reserve((size_t)std::min<int64_t>(have, K) * W);
        int64_t kept = 0;
        for (int64_t t = 0; t < have && kept < K; ++t) {
            const uint64_t *x = base + idx[t] * W;
            if (kept > 0 && std::equal(x, x + W, keep.end() - W)) continue;  // the same support again
            keep.insert(keep.end(), x, x + W);
            ++kept;
        }
        rows.swap(keep);
        if (kept == K) {
            kth.assign(rows.end() - W, rows.end());
            pc = popc(kth.data(), W);
        } else {
            kth.clear();
            pc = 0;
        }
    }
};

}  // namespace efm
