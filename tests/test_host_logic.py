"""Host logic of the library, without a GPU.

The first-K search keeps, on the host, the K smallest results seen so far in
the output order (|U|, then the ascending column list) and hands the K-th of
them to the kernels as the bound (efm::TopK, csrc/efm_topk.h).  Here that
code is compiled alone with g++ and fed random batches of distinct supports;
after every batch its bound must be the K-th smallest of all supports seen,
by the order's definition written out in Python, and at the end it must keep
exactly the K smallest."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1804_02867_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("topk") / "topk_driver")
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, os.path.join(ROOT, "tests", "host", "topk_driver.cpp"),
                    "-o", exe], check=True)
    return exe


def columns(row):
    return [64 * w + b for w, x in enumerate(row) for b in range(64) if (int(x) >> b) & 1]


def order_key(row):
    cols = columns(row)
    return (len(cols), cols)


@pytest.mark.parametrize("seed,K,W", [(0, 1, 1), (1, 5, 1), (2, 40, 2), (3, 100, 3), (4, 7, 64)])
def test_topk_keeps_the_k_smallest(driver, seed, K, W):
    rng = np.random.default_rng(seed)
    n_cols = 64 * W
    seen = set()
    while len(seen) < 6 * K + 20:
        size = int(rng.integers(1, min(12, n_cols) + 1))
        cols = rng.choice(n_cols, size=size, replace=False)
        row = [0] * W
        for c in cols:
            row[c // 64] |= 1 << int(c % 64)
        seen.add(tuple(row))
    rows = list(seen)
    rng.shuffle(rows)
    cuts = sorted(rng.choice(np.arange(1, len(rows)), size=5, replace=False).tolist()) + [len(rows)]
    text = [f"{K} {W}"]
    batches, lo = [], 0
    for hi in cuts:
        batches.append(rows[lo:hi])
        text.append(str(hi - lo))
        text.extend(" ".join(str(x) for x in r) for r in rows[lo:hi])
        lo = hi
    text.append("-1")
    out = subprocess.run([driver], input="\n".join(text) + "\n", capture_output=True, text=True,
                         check=True).stdout.splitlines()
    bounds = [ln.split()[1:] for ln in out if ln.startswith("bound")]
    kept = [tuple(int(x) for x in ln.split()[1:]) for ln in out if ln.startswith("row")]
    so_far = []
    for b, line in zip(batches, bounds):
        so_far += b
        if len(so_far) < K:
            assert line == ["0"]
            continue
        kth = sorted(so_far, key=order_key)[K - 1]
        assert int(line[0]) == len(columns(kth))
        assert tuple(int(x) for x in line[1:]) == kth
    assert sorted(kept, key=order_key) == sorted(rows, key=order_key)[:K]
