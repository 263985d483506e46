"""Host logic of the library, without a GPU.

The loader's host work (csrc/efm_netprep.h) validates S and builds the
static network the kernels read; compiled alone with g++, its decoded output
must equal what the definitions give on seeded networks: split columns
(forward, then reverse for a reversible reaction), S_int by column, the
consumers and producers of each internal metabolite, twins, pivot keys,
Hadamard bits, the dense copy and the full rows over split columns; and it
must refuse every malformed input.

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


def _compile(tmp_path_factory, name):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp(name) / name)
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, os.path.join(ROOT, "tests", "host", name + ".cpp"),
                    "-o", exe], check=True)
    return exe


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    return _compile(tmp_path_factory, "topk_driver")


@pytest.fixture(scope="module")
def netprep(tmp_path_factory):
    return _compile(tmp_path_factory, "netprep_driver")


def run_netprep(exe, n_met, n_rxn, row_ptr, col_idx, coef, reversible, external):
    vals = [n_met, n_rxn, *row_ptr, *col_idx, *coef, *reversible, *external]
    out = subprocess.run([exe], input=" ".join(str(int(v)) for v in vals) + "\n", capture_output=True, text=True,
                         check=True).stdout.splitlines()
    status = int(out[0].split()[1])
    items = {}
    for ln in out[1:]:
        f = ln.split()
        items.setdefault(f[0], []).append(f[1:])
    return status, items


def expected_static(net):
    """The static network by its definitions, from the dense S."""
    S = net.dense()
    cols, cmap = [], []
    for j in range(net.n_rxn):
        cols.append(S[:, j])
        cmap.append((j, 1))
        if net.reversible[j]:
            cols.append(-S[:, j])
            cmap.append((j, -1))
    Ss = np.stack(cols, axis=1)
    internal = [m for m in range(net.n_met) if not net.external[m]]
    Si = Ss[internal]
    M, N = Si.shape
    epl = min(e for e in (1, 2, 4, 8, 16, 28, 32) if e >= max(1, -(-M // 32)))
    exp = {"shape": [N, M, -(-N // 64), epl, 32 * epl], "colmap": cmap}
    exp["col"] = [[(r, int(Si[r, k])) for r in range(M) if Si[r, k]] for k in range(N)]
    exp["cons"] = [[(k, int(-Si[r, k])) for k in range(N) if Si[r, k] < 0] for r in range(M)]
    exp["prod"] = [[(k, int(Si[r, k])) for k in range(N) if Si[r, k] > 0] for r in range(M)]
    exp["twin"] = [next((q for q in (k - 1, k + 1) if 0 <= q < N and cmap[q][0] == cmap[k][0]), -1)
                   for k in range(N)]
    exp["key"] = [((len(exp["cons"][r]) << 16) | r, (len(exp["prod"][r]) << 16) | r) for r in range(M)]
    nsq = [int(sum(int(x) ** 2 for x in Si[:, k])) for k in range(N)]
    exp["hbits"] = [(q - 1).bit_length() if q > 1 else 0 for q in nsq]  # ceil(log2(q))
    exp["dense"] = [list(Si[:, k]) + [0] * (32 * epl - M) for k in range(N)]
    exp["met"] = [[(k, int(Ss[m, k])) for k in range(N) if Ss[m, k]] for m in range(net.n_met)]
    if M > 64:
        # wide networks: lane masks in the expansion's row layout.  Lane l of a
        # group of G lanes reads the 4-entry chunks l, l + G, ... of a row, so
        # bit 4 i + j of its word stands for row 4 (l + G i) + j.
        G = min(32, 4 * epl)
        cpl = 8 * epl // G
        exp["fix"] = []
        for k in range(N):
            for lane in range(G):
                c = p = 0
                for i in range(cpl):
                    for j in range(4):
                        r = 4 * (lane + G * i) + j
                        if r < M and Si[r, k] < 0:
                            c |= 1 << (4 * i + j)
                        if r < M and Si[r, k] > 0:
                            p |= 1 << (4 * i + j)
                exp["fix"].append((k, lane, c, p))
    if M <= 64:
        # narrow networks: ranks in the key orders, keys by rank, row hash
        # constants (SplitMix64 finaliser of 0x9E3779B97F4A7C15 (m + 1)), and
        # per column: rank-space and row-space masks, sum S R, max |S|, gcd == 1
        import math

        mask = (1 << 64) - 1

        def splitmix_fin(z):
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9 & mask
            z = (z ^ (z >> 27)) * 0x94D049BB133111EB & mask
            return z ^ (z >> 31)

        kp = sorted((exp["key"][r][0], r) for r in range(M))
        kn = sorted((exp["key"][r][1], r) for r in range(M))
        rp = {r: i for i, (_, r) in enumerate(kp)}
        rn = {r: i for i, (_, r) in enumerate(kn)}
        exp["rank"] = [(rp[r], rn[r]) for r in range(M)]
        big = 0xFFFFFFFF
        exp["keyr"] = [(kp[i][0] if i < M else big, kn[i][0] if i < M else big) for i in range(64)]
        R = [splitmix_fin(0x9E3779B97F4A7C15 * (r + 1) & mask) for r in range(M)]
        exp["hrow"] = R
        exp["colx"] = []
        for k in range(N):
            rows = [r for r in range(M) if Si[r, k]]
            g = 0
            for r in rows:
                g = math.gcd(g, abs(int(Si[r, k])))
            exp["colx"].append((sum(1 << rp[r] for r in rows), sum(1 << rn[r] for r in rows), sum(1 << r for r in rows),
                                sum(int(Si[r, k]) * R[r] for r in rows) & mask,
                                max((abs(int(Si[r, k])) for r in rows), default=0), 1 if g == 1 else 0))
    return exp


def _pairs(fields):
    return [tuple(int(x) for x in f.split(":")) for f in fields]


@pytest.mark.parametrize("which", ["tiny-0", "tiny-5", "core", "batched-7", "type1-3", "mid-40", "wide-150"])
def test_network_preparation_matches_the_definitions(netprep, which):
    from paper_1804_02867_gb300 import synth

    net = {"tiny-0": lambda: synth.tiny(0), "tiny-5": lambda: synth.tiny(5), "core": synth.core,
           "batched-7": lambda: synth.batched_member(7), "type1-3": lambda: synth.type1(3),
           "mid-40": lambda: synth.generate(n_int=40, n_targets=3, n_hubs=2, n_substrates=1, n_rxn=70, n_rev=20,
                                            coef_probs={1: 0.5, 3: 0.3, 524287: 0.2}, seed=7),
           "wide-150": lambda: synth.generate(n_int=150, n_targets=3, n_hubs=4, n_substrates=2, n_rxn=260, n_rev=60,
                                              seed=9)}[which]()
    status, got = run_netprep(netprep, net.n_met, net.n_rxn, net.row_ptr, net.col_idx, net.coef, net.reversible,
                              net.external)
    assert status == 0
    exp = expected_static(net)
    N, M = exp["shape"][0], exp["shape"][1]
    assert [int(x) for x in got["shape"][0]] == exp["shape"]
    assert [(int(f[1]), int(f[2])) for f in got["colmap"]] == exp["colmap"]
    for name, n in (("col", N), ("cons", M), ("prod", M)):
        rows = got.get(name, [])
        assert [int(f[0]) for f in rows] == list(range(n))
        assert [_pairs(f[1:]) for f in rows] == exp[name], name
    assert [int(f[1]) for f in got["twin"]] == exp["twin"]
    assert [(int(f[1]), int(f[2])) for f in got.get("key", [])] == exp["key"]
    assert [int(f[1]) for f in got["hbits"]] == exp["hbits"]
    assert got["dense_offset_mod4"] == [["0"]]
    assert got["narrow"] == [["1" if M <= 64 else "0"]]
    if M <= 64:
        assert [(int(f[1]), int(f[2])) for f in got["rank"]] == exp["rank"]
        assert [(int(f[1]), int(f[2])) for f in got["keyr"]] == exp["keyr"]
        assert [int(f[1]) for f in got["hrow"]] == exp["hrow"]
        assert [tuple(int(x) for x in f[1:]) for f in got["colx"]] == exp["colx"]
        assert got["align64"] == [["0", "0"]]
    assert got["fixtab"] == [["1" if M > 64 else "0"]]
    if M > 64:
        assert [tuple(int(x) for x in f) for f in got["fix"]] == exp["fix"]
    assert [[int(x) for x in f[1:]] for f in got["dense"]] == exp["dense"]
    assert [_pairs(f[1:]) for f in got["met"]] == exp["met"]


def test_network_preparation_refuses_malformed_input(netprep):
    from paper_1804_02867_gb300 import synth

    net = synth.tiny(1)
    args = [net.n_met, net.n_rxn, net.row_ptr, net.col_idx, net.coef, net.reversible, net.external]

    def status(**change):
        a = dict(zip(("n_met", "n_rxn", "row_ptr", "col_idx", "coef", "reversible", "external"), args))
        a.update(change)
        return run_netprep(netprep, *a.values())[0]

    assert status() == 0
    coef = net.coef.copy()
    coef[3] = 0
    assert status(coef=coef) == -1  # explicit zero
    coef[3] = 524288
    assert status(coef=coef) == -1  # beyond the coefficient limit
    col = net.col_idx.copy()
    col[2] = net.n_rxn
    assert status(col_idx=col) == -1  # reaction index out of range
    col = net.col_idx.copy()
    r0 = next(m for m in range(net.n_met) if net.row_ptr[m + 1] - net.row_ptr[m] >= 2)
    col[net.row_ptr[r0] + 1] = col[net.row_ptr[r0]]
    assert status(col_idx=col) == -1  # duplicate entry in a row
    rp = net.row_ptr.copy()
    rp[2], rp[3] = rp[3], rp[2]
    assert status(row_ptr=rp) == -1 or rp[2] == rp[3]  # decreasing row pointer
    rp = net.row_ptr.copy()
    rp[0] = 1
    assert status(row_ptr=rp) == -1  # row_ptr[0] != 0


def columns(row):
    return [64 * w + b for w, x in enumerate(row) for b in range(64) if (int(x) >> b) & 1]


def order_key(row):
    cols = columns(row)
    return (len(cols), cols)


@pytest.mark.parametrize("seed,K,W,dup", [(0, 1, 1, False), (1, 5, 1, False), (2, 40, 2, False), (3, 100, 3, False),
                                         (4, 7, 64, False), (5, 30, 2, True), (6, 3, 1, True)])
def test_topk_keeps_the_k_smallest(driver, seed, K, W, dup):
    """The K smallest distinct supports seen, after every batch; with dup,
    later batches repeat supports of earlier ones (as the merged answers of
    several searches do), and a repeat counts once."""
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
    if dup:  # every third support appears a second time, later
        rows = rows + [rows[i] for i in range(0, len(rows), 3)]
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
    so_far = set()
    for b, line in zip(batches, bounds):
        so_far |= set(b)
        if len(so_far) < K:
            assert line == ["0"]
            continue
        kth = sorted(so_far, key=order_key)[K - 1]
        assert int(line[0]) == len(columns(kth))
        assert tuple(int(x) for x in line[1:]) == kth
    assert sorted(kept, key=order_key) == sorted(set(rows), key=order_key)[:K]
