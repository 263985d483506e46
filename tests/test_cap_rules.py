"""The first-K length-cap rules drop only states without results.

In a run capped at P (first-K deepening), the GPU drops
  * a child of size P whose support touches an internal row with one sign
    only (a surplus with no consumer, a deficit with no producer in U), or
    that has no secondary step left;
  * a child of size P - 1 whose support has such one-sided rows when no
    single column c (twin rule kept) gives each of them the missing sign and
    finds the opposite sign in U for every row of its own.
Both follow from balance: S_int v = 0 with v > 0 on the support needs both
signs in every row the support touches.  This test restates the traversal
in plain Python with and without the rules and requires the same result
set, on the tiny networks and short core runs.  No GPU is needed.
"""
from math import gcd

import pytest

from oracle import reference as R
from paper_1804_02867_gb300 import synth


def _traverse(net, target, max_len, max_sec, rules):
    S, twin, full, cols = R.split_network(net)
    M, N = len(S), len(cols)
    deg_out = [sum(1 for k in range(N) if S[i][k] < 0) for i in range(M)]
    deg_in = [sum(1 for k in range(N) if S[i][k] > 0) for i in range(M)]
    signs = [({i for i in range(M) if S[i][k] < 0}, {i for i in range(M) if S[i][k] > 0}) for k in range(N)]

    def one_sided(U):
        cons, prod = set(), set()
        for k in range(N):
            if (U >> k) & 1:
                cons |= signs[k][0]
                prod |= signs[k][1]
        return cons, prod, (cons ^ prod)

    res, dropped = set(), 0
    front = {}
    for j in range(N):
        if target >= 0 and full[target][j] <= 0:
            continue
        ef, zero = R._normalise([S[i][j] for i in range(M)])
        if zero:
            if R.nullity_one(S, 1 << j, N):
                res.add(1 << j)
        else:
            front[(1 << j, ef)] = 0
    while front:
        nxt = {}
        for (U, ef), sec in front.items():
            pc = bin(U).count("1")
            _, piv = min((deg_out[i] if ef[i] > 0 else deg_in[i], i) for i in range(M) if ef[i] != 0)
            e = ef[piv]
            for k in range(N):
                s = S[piv][k]
                if not ((s < 0) if e > 0 else (s > 0)):
                    continue
                if twin[k] >= 0 and (U >> twin[k]) & 1:
                    continue
                inu = (U >> k) & 1
                if (not inu and pc + 1 > max_len) or (inu and sec + 1 > max_sec):
                    continue
                g = gcd(abs(e), abs(s))
                nef, zero = R._normalise([abs(s) // g * ef[i] + abs(e) // g * S[i][k] for i in range(M)])
                if any(abs(x) > 2**31 - 1 for x in nef):
                    continue
                U2 = U | (1 << k)
                if zero:
                    if R.nullity_one(S, U2, N):
                        res.add(U2)
                    continue
                pc2, sec2 = pc + (0 if inu else 1), sec + inu
                if rules and pc2 >= max_len - 1:
                    cons, prod, lonely = one_sided(U2)
                    dead = False
                    if pc2 >= max_len:
                        dead = sec2 >= max_sec or bool(lonely)
                    elif lonely:
                        dead = True
                        for c in range(N):
                            if (U2 >> c) & 1 or (twin[c] >= 0 and (U2 >> twin[c]) & 1):
                                continue
                            c_cons, c_prod = signs[c]
                            if all(((i in cons) or (i in c_cons)) and ((i in prod) or (i in c_prod))
                                   for i in (lonely | c_cons | c_prod)):
                                dead = False
                                break
                    if dead:
                        dropped += 1
                        continue
                key = (U2, nef)
                if key not in nxt:
                    nxt[key] = sec2
        front = nxt
    return res, dropped


@pytest.mark.parametrize("seed", range(6))
def test_cap_rules_keep_every_result_on_tiny_networks(seed):
    net = synth.tiny(seed)
    dropped = 0
    for t in list(net.targets) + [-1]:
        for L, S in ((3, 1), (4, 2), (5, 1), (6, 2), (8, 1)):
            plain, _ = _traverse(net, t, L, S, False)
            ruled, d = _traverse(net, t, L, S, True)
            assert plain == ruled, (seed, t, L, S)
            dropped += d
    assert dropped > 0


def test_cap_rules_keep_every_result_on_the_core_network():
    net = synth.core()
    dropped = 0
    for t in (63, 58):
        for L in (6, 8):
            plain, _ = _traverse(net, t, L, 4, False)
            ruled, d = _traverse(net, t, L, 4, True)
            assert plain == ruled, (t, L)
            dropped += d
    assert dropped > 100
