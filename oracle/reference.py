"""Pure-Python restatement of the traversal for tiny inputs.

TEST INFRASTRUCTURE ONLY.  A second, independent spelling of the same
definition as ``efm_oracle.c`` (Python integers, Fraction elimination,
dictionaries instead of sorted arrays).  It additionally carries the explicit
flux vector v of one path (with the integer scale s, S_int v = s * EF) to
every state and checks, at every step, that the stored extra-flux vector EF is
a positive multiple of S_int v (Eq. 2) and that v is positive exactly on U --
the invariant the integer ray update (Eq. 3) relies on.
"""
from __future__ import annotations

from fractions import Fraction
from math import gcd

INT32_MAX = 2**31 - 1
TRUNCATED, CAPPED, OVERFLOW_DROPPED = 1, 2, 4


def split_network(net):
    """Columns: forward then reverse (if reversible) per reaction (Def. 6
    direction).  Returns (S_int as list of rows over columns, twin, full S
    rows, internal row indices)."""
    S = net.dense()
    cols = []  # (reaction, direction)
    for j in range(net.n_rxn):
        cols.append((j, 1))
        if net.reversible[j]:
            cols.append((j, -1))
    N = len(cols)
    twin = [-1] * N
    for k in range(N - 1):
        if cols[k][0] == cols[k + 1][0]:
            twin[k], twin[k + 1] = k + 1, k
    full = [[int(S[m, j]) * d for (j, d) in cols] for m in range(net.n_met)]
    internal = [m for m in range(net.n_met) if not net.external[m]]
    S_int = [full[m] for m in internal]
    return S_int, twin, full, cols


def rank_fraction(rows):
    """Rank over Q by Gaussian elimination on Fractions."""
    A = [[Fraction(x) for x in r] for r in rows]
    if not A:
        return 0
    n_r, n_c = len(A), len(A[0])
    r = 0
    for c in range(n_c):
        piv = next((i for i in range(r, n_r) if A[i][c] != 0), None)
        if piv is None:
            continue
        A[r], A[piv] = A[piv], A[r]
        for i in range(n_r):
            if i != r and A[i][c] != 0:
                f = A[i][c] / A[r][c]
                A[i] = [x - f * y for x, y in zip(A[i], A[r])]
        r += 1
        if r == n_r:
            break
    return r


def nullity_one(S_int, U, N):
    """Def. 3 for a balanced support U: nullity over Q of S_int[:, U] is 1."""
    cols = [k for k in range(N) if (U >> k) & 1]
    sub = [[row[k] for k in cols] for row in S_int if any(row[k] for k in cols)]
    return len(cols) - rank_fraction(sub) == 1


def _normalise(ef):
    g = 0
    for x in ef:
        g = gcd(g, abs(x))
    if g == 0:
        return tuple(ef), True
    return tuple(x // g for x in ef), False


def enumerate_reference(net, target, max_len=64, max_secondary=4, max_results=0, max_frontier=0, fluxes=None,
                        prune=True):
    """The traversal in pure Python.  Returns (sorted result supports as
    int bitmasks, counters).  fluxes: optional dict, filled with support ->
    the flux vector {column: flux} of the first path reaching each balanced
    support (S_int v = 0 there).  prune=False skips the superset rule, which
    leaves only the definition (Def. 3: nullity 1 decides)."""
    S_int, twin, full, cols = split_network(net)
    M = len(S_int)
    N = len(cols)
    deg_out = [sum(1 for k in range(N) if S_int[i][k] < 0) for i in range(M)]
    deg_in = [sum(1 for k in range(N) if S_int[i][k] > 0) for i in range(M)]
    ctr = dict(levels=0, seeds=0, expansions=0, overflow=0, balanced=0, candidates=0, results=0,
               pruned=0, frontier=0, frontier_max=0, status=0, zero_flux=0)
    seen = set()
    results = []  # (U, level)

    def col_of(k):
        return [S_int[i][k] for i in range(M)]

    def judge(U, level):
        if U in seen:
            return
        seen.add(U)
        ctr["candidates"] += 1
        if nullity_one(S_int, U, N):
            results.append((U, level))
            ctr["results"] += 1

    def check_invariant(U, ef, v):
        b = [sum(S_int[i][k] * v.get(k, 0) for k in v) for i in range(M)]
        assert all(x > 0 for x in v.values())
        assert set(v) == {k for k in range(N) if (U >> k) & 1}
        # b is a positive multiple of ef
        nz = [i for i in range(M) if b[i] != 0]
        if not nz:
            assert not any(ef)
            return
        i0 = nz[0]
        assert ef[i0] != 0 and (b[i0] > 0) == (ef[i0] > 0)
        assert all(b[i] * ef[i0] == ef[i] * b[i0] for i in range(M))

    # level 0: seeds
    F = {}  # (U, ef) -> (sec, v)
    for j in range(N):
        if target >= 0 and full[target][j] <= 0:
            continue
        ctr["seeds"] += 1
        raw = col_of(j)
        ef, zero = _normalise(raw)
        U = 1 << j
        v = {j: 1}
        scale = max((abs(x) for x in raw), default=0) and gcd(*[abs(x) for x in raw])
        check_invariant(U, ef, v)
        if zero:
            ctr["balanced"] += 1
            if fluxes is not None and U not in fluxes:
                fluxes[U] = v
            judge(U, 0)
        else:
            F[(U, ef)] = (0, v, scale)

    def finish():
        if ctr["overflow"]:
            ctr["status"] |= OVERFLOW_DROPPED
        res = sorted((U for U, _ in results), key=lambda U: (bin(U).count("1"),
                                                             [k for k in range(N) if (U >> k) & 1]))
        if max_results > 0:
            res = res[:max_results]
        return res, ctr

    ctr["levels"] = 1
    if max_frontier > 0 and len(F) > max_frontier:
        ctr["status"] |= TRUNCATED
        return finish()
    ctr["frontier"] += len(F)
    ctr["frontier_max"] = max(ctr["frontier_max"], len(F))
    if max_results > 0 and ctr["results"] >= max_results:
        ctr["status"] |= CAPPED
        return finish()

    level = 0
    while F:
        level += 1
        C = {}
        for (U, ef), (sec, v, scale) in F.items():
            pc = bin(U).count("1")
            cand = [(deg_out[i] if ef[i] > 0 else deg_in[i], i) for i in range(M) if ef[i] != 0]
            _, piv = min(cand)
            e = ef[piv]
            for k in range(N):
                s = S_int[piv][k]
                if not ((s < 0) if e > 0 else (s > 0)):
                    continue
                if twin[k] >= 0 and (U >> twin[k]) & 1:
                    continue
                in_u = (U >> k) & 1
                if not in_u and pc + 1 > max_len:
                    continue
                if in_u and sec + 1 > max_secondary:
                    continue
                ctr["expansions"] += 1
                g = gcd(abs(e), abs(s))
                a, c = abs(s) // g, abs(e) // g
                raw = [a * ef[i] + c * S_int[i][k] for i in range(M)]
                nef, zero = _normalise(raw)
                if any(abs(x) > INT32_MAX for x in nef):
                    ctr["overflow"] += 1
                    continue
                U2 = U | (1 << k)
                # S_int v = scale * EF, so flux c on k is c * scale in v's units
                v2 = {kk: a * vv for kk, vv in v.items()}
                v2[k] = v2.get(k, 0) + c * scale
                g2 = gcd(*[abs(x) for x in raw]) if any(raw) else 1
                check_invariant(U2, nef, v2)
                if zero:
                    ctr["balanced"] += 1
                    if fluxes is not None and U2 not in fluxes:
                        fluxes[U2] = v2
                    judge(U2, level)
                    continue
                # the new column completes a result accepted at an earlier level
                if prune and not in_u and any((E >> k) & 1 and (E & ~U2) == 0 for E, lv in results if lv < level):
                    ctr["pruned"] += 1
                    continue
                key = (U2, nef)
                if key not in C or C[key][0] > sec + in_u:
                    C[key] = (sec + in_u, v2, scale * g2)
        F = C
        ctr["levels"] = level + 1
        if max_frontier > 0 and len(F) > max_frontier:
            ctr["status"] |= TRUNCATED
            break
        ctr["frontier"] += len(F)
        ctr["frontier_max"] = max(ctr["frontier_max"], len(F))
        if max_results > 0 and ctr["results"] >= max_results:
            ctr["status"] |= CAPPED
            break
    return finish()


def enumerate_subtractive(net, target, max_len=64, max_secondary=4, max_results=0, max_frontier=0, prune=True):
    """The traversal with the subtractive steps of Eq. 5 as well, in pure
    Python.  A state is (U, v): the support and its flux vector, a primitive
    integer vector positive on U.  Its extra flux is recomputed from v at
    every step, EF = S_int v (Eq. 2), instead of being updated.  Branches of
    the acting metabolite i (fewest reactions able to fix it, then index):
      * additive (Eq. 3 / Eq. 4): every k with S_ik of the opposite sign to
        EF_i, twin not in U, v' = a v + c e_k;
      * subtractive (Eq. 5): every k in U with S_ik of the same sign as EF_i,
        v' = a v - c e_k, discarded when v'_k <= 0 (Prop. 3);
    with g = gcd(|EF_i|, |S_ik|), a = |S_ik| / g, c = |EF_i| / g, so that
    EF'_i = 0.  Secondary steps (k already in U, either kind) cost one unit of
    max_secondary.  Returns (sorted result supports as int bitmasks, counters)
    like enumerate_reference."""
    S_int, twin, full, cols = split_network(net)
    M = len(S_int)
    N = len(cols)
    deg_out = [sum(1 for k in range(N) if S_int[i][k] < 0) for i in range(M)]
    deg_in = [sum(1 for k in range(N) if S_int[i][k] > 0) for i in range(M)]
    ctr = dict(levels=0, seeds=0, expansions=0, overflow=0, balanced=0, candidates=0, results=0,
               pruned=0, frontier=0, frontier_max=0, status=0, zero_flux=0)
    seen = set()
    results = []  # (U, level)

    def extra_flux(v):
        return [sum(S_int[i][k] * x for k, x in v) for i in range(M)]

    def primitive(vd):
        g = 0
        for x in vd.values():
            g = gcd(g, abs(x))
        return tuple(sorted((k, x // g) for k, x in vd.items() if x != 0))

    def judge(U, level):
        if U in seen:
            return
        seen.add(U)
        ctr["candidates"] += 1
        if nullity_one(S_int, U, N):
            results.append((U, level))
            ctr["results"] += 1

    def finish():
        if ctr["overflow"]:
            ctr["status"] |= OVERFLOW_DROPPED
        res = sorted((U for U, _ in results), key=lambda U: (bin(U).count("1"),
                                                             [k for k in range(N) if (U >> k) & 1]))
        if max_results > 0:
            res = res[:max_results]
        return res, ctr

    def child(U, v, level, sec, F, new_col=-1):
        """Place the child state (U, v) (v primitive) at `level`; new_col: the
        column an additive step added to the support (superset rule)."""
        ef = extra_flux(v)
        if any(abs(x) > INT32_MAX for x in ef) or any(abs(x) > INT32_MAX for _, x in v):
            ctr["overflow"] += 1
            return
        if not any(ef):
            ctr["balanced"] += 1
            judge(U, level)
            return
        if prune and new_col >= 0 and any((E >> new_col) & 1 and (E & ~U) == 0 for E, lv in results if lv < level):
            ctr["pruned"] += 1
            return
        key = (U, v)
        if key not in F or F[key] > sec:
            F[key] = sec

    F = {}  # (U, v) -> sec
    for j in range(N):
        if target >= 0 and full[target][j] <= 0:
            continue
        ctr["seeds"] += 1
        child(1 << j, ((j, 1),), 0, 0, F)
    ctr["levels"] = 1
    if max_frontier > 0 and len(F) > max_frontier:
        ctr["status"] |= TRUNCATED
        return finish()
    ctr["frontier"] += len(F)
    ctr["frontier_max"] = max(ctr["frontier_max"], len(F))
    if max_results > 0 and ctr["results"] >= max_results:
        ctr["status"] |= CAPPED
        return finish()
    level = 0
    while F:
        level += 1
        C = {}
        for (U, v), sec in F.items():
            pc = bin(U).count("1")
            ef = extra_flux(v)
            _, piv = min((deg_out[i] if ef[i] > 0 else deg_in[i], i) for i in range(M) if ef[i] != 0)
            e = ef[piv]
            vd = dict(v)
            for k in range(N):
                s = S_int[piv][k]
                in_u = (U >> k) & 1
                add = (s < 0) if e > 0 else (s > 0)
                take = bool(in_u) and ((s > 0) if e > 0 else (s < 0))
                if not add and not take:
                    continue
                if add and twin[k] >= 0 and (U >> twin[k]) & 1:
                    continue
                if (in_u and sec + 1 > max_secondary) or (not in_u and pc + 1 > max_len):
                    continue
                ctr["expansions"] += 1
                g = gcd(abs(e), abs(s))
                a, c = abs(s) // g, abs(e) // g
                nv = {kk: a * x for kk, x in vd.items()}
                nv[k] = nv.get(k, 0) + (c if add else -c)
                if take and nv[k] <= 0:
                    ctr["zero_flux"] += 1
                    continue
                nvt = primitive(nv)
                assert extra_flux(nvt)[piv] == 0  # Eq. 3 / Eq. 5 zero the acting metabolite
                child(U | (1 << k), nvt, level, sec + in_u, C, k if not in_u else -1)
        F = C
        ctr["levels"] = level + 1
        if max_frontier > 0 and len(F) > max_frontier:
            ctr["status"] |= TRUNCATED
            break
        ctr["frontier"] += len(F)
        ctr["frontier_max"] = max(ctr["frontier_max"], len(F))
        if max_results > 0 and ctr["results"] >= max_results:
            ctr["status"] |= CAPPED
            break
    return finish()


def _splitmix_at(seed, c):
    """First output of SplitMix64 started from state seed + c * golden."""
    m = (1 << 64) - 1
    z = (seed + (c + 1) * 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def sample_reference(net, target, max_len, max_secondary, seed, n_walks):
    """The Monte-Carlo walks in pure Python (exact integers): walk w draws
    counter 128 w for its seed column and 128 w + s for step s; one random
    valid branch per step.  Returns (sorted result bitmasks, counters)."""
    S_int, twin, full, cols = split_network(net)
    M = len(S_int)
    N = len(cols)
    deg_out = [sum(1 for k in range(N) if S_int[i][k] < 0) for i in range(M)]
    deg_in = [sum(1 for k in range(N) if S_int[i][k] > 0) for i in range(M)]
    ctr = dict(levels=0, seeds=0, expansions=0, overflow=0, balanced=0, candidates=0, results=0,
               pruned=0, frontier=0, frontier_max=0, status=0, zero_flux=0)
    seeds = [j for j in range(N) if target < 0 or full[target][j] > 0]
    seen, results = set(), []
    for w in range(n_walks if seeds else 0):
        c0 = 128 * w
        j = seeds[_splitmix_at(seed, c0) % len(seeds)]
        ctr["seeds"] += 1
        U, sec, steps = 1 << j, 0, 0
        ef, zero = _normalise([S_int[i][j] for i in range(M)])
        if any(abs(x) > INT32_MAX for x in ef):
            ctr["overflow"] += 1
            continue
        s = 1
        while True:
            if zero:
                ctr["balanced"] += 1
                if U not in seen:
                    seen.add(U)
                    ctr["candidates"] += 1
                    if nullity_one(S_int, U, N):
                        results.append(U)
                        ctr["results"] += 1
                break
            _, piv = min((deg_out[i] if ef[i] > 0 else deg_in[i], i) for i in range(M) if ef[i] != 0)
            e = ef[piv]
            pc = bin(U).count("1")
            valid = []
            for k in range(N):
                sk = S_int[piv][k]
                if not ((sk < 0) if e > 0 else (sk > 0)):
                    continue
                if twin[k] >= 0 and (U >> twin[k]) & 1:
                    continue
                in_u = (U >> k) & 1
                if (not in_u and pc + 1 > max_len) or (in_u and sec + 1 > max_secondary):
                    continue
                valid.append(k)
            if not valid:
                ctr["pruned"] += 1
                break
            k = valid[_splitmix_at(seed, c0 + s) % len(valid)]
            sk = S_int[piv][k]
            g = gcd(abs(e), abs(sk))
            a, c = abs(sk) // g, abs(e) // g
            ctr["expansions"] += 1
            steps += 1
            if (U >> k) & 1:
                sec += 1
            U |= 1 << k
            ef, zero = _normalise([a * ef[i] + c * S_int[i][k] for i in range(M)])
            if any(abs(x) > INT32_MAX for x in ef):
                ctr["overflow"] += 1
                break
            s += 1
        ctr["levels"] = max(ctr["levels"], steps)
    if ctr["overflow"]:
        ctr["status"] |= OVERFLOW_DROPPED
    res = sorted(results, key=lambda U: (bin(U).count("1"), [k for k in range(N) if (U >> k) & 1]))
    return res, ctr
