"""Pins of the CPU oracle to things other than itself (no GPU needed).

* hand-worked networks (tests/golden/handworked.json, derived by hand from
  Def. 2-3, Eq. 2-4 and the exhaustive restatement of Alg. 3);
* the exact rank routine against sympy, including the arbitrary-precision
  fallback;
* Type I networks (Lemma 2): results equal the simple paths and simple
  cycles of the reaction digraph, enumerated by networkx;
* tiny random networks: every result is an elementary flux mode (exact
  sympy null space), and results are a subset of the brute-force EFM set;
* the overflow rule on a chain whose flux grows by 4 per step;
* the maximal network (the library's size limits): its chain target's
  pathways and flux vectors in closed form.
"""
import json
import os

import numpy as np
import pytest

from paper_1804_02867_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _handworked():
    with open(os.path.join(HERE, "golden", "handworked.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _handworked(), ids=lambda c: c["name"])
def test_handworked(oracle_lib, case):
    net = synth.Network.from_dense(case["S"], case["reversible"], case["external"])
    lim = oracle_lib.Limits(case["max_len"], case["max_secondary"], 0, 0, subtractive=case.get("subtractive", False))
    sup, ctr = oracle_lib.enumerate_pathways(net, case["target"], lim)
    assert oracle_lib.supports_to_lists(sup) == [tuple(x) for x in case["expected"]]
    for k, v in case.get("counters", {}).items():
        assert ctr[k] == v, (k, ctr)


def test_handworked_python_reference_agrees(oracle_lib):
    from oracle import reference

    for case in _handworked():
        net = synth.Network.from_dense(case["S"], case["reversible"], case["external"])
        run = reference.enumerate_subtractive if case.get("subtractive") else reference.enumerate_reference
        res, ctr = run(net, case["target"], case["max_len"], case["max_secondary"])
        got = [tuple(k for k in range(64) if (U >> k) & 1) for U in res]
        assert got == [tuple(x) for x in case["expected"]], case["name"]
        for k, v in case.get("counters", {}).items():
            assert ctr[k] == v, (case["name"], k)


def test_rank_matches_sympy(oracle_lib):
    import sympy

    rng = np.random.default_rng(7)
    for trial in range(300):
        r, c = int(rng.integers(1, 9)), int(rng.integers(1, 9))
        k = int(rng.integers(1, min(r, c) + 1))
        A = rng.integers(-3, 4, size=(r, k)) @ rng.integers(-3, 4, size=(k, c))
        if trial % 3 == 0:
            A = rng.integers(-2, 3, size=(r, c))
        want = sympy.Matrix(A.tolist()).rank()
        assert oracle_lib.rank(A) == want
        assert oracle_lib.rank(A, force_big=True) == want


def test_rank_bigint_fallback_on_huge_minors(oracle_lib):
    """Entries near 2^30 make 12x12 minors far exceed 2^127, so the __int128
    elimination overflows and the arbitrary-precision path decides."""
    import sympy

    rng = np.random.default_rng(11)
    for trial in range(6):
        n = 12
        k = 12 if trial % 2 == 0 else 9
        B = rng.integers(-(2**15), 2**15, size=(n, k))
        C = rng.integers(-(2**14), 2**14, size=(k, n))
        A = B @ C
        want = sympy.Matrix(A.tolist()).rank()
        assert oracle_lib.rank(A) == want


def _type1_expected(net, target, max_len):
    """Simple source-to-sink paths and simple cycles of the bipartite
    metabolite/column digraph that contain a column producing the target."""
    import networkx as nx

    from oracle import bruteforce

    S_int, twin, full = bruteforce.split(net)
    M, N = S_int.shape
    G = nx.DiGraph()
    G.add_node("src")
    G.add_node("snk")
    for k in range(N):
        subs = [i for i in range(M) if S_int[i, k] < 0]
        prods = [i for i in range(M) if S_int[i, k] > 0]
        assert len(subs) <= 1 and len(prods) <= 1
        G.add_edge(("m", subs[0]) if subs else "src", ("c", k))
        G.add_edge(("c", k), ("m", prods[0]) if prods else "snk")
    found = set()
    for path in nx.all_simple_paths(G, "src", "snk"):
        found.add(tuple(sorted(n[1] for n in path if isinstance(n, tuple) and n[0] == "c")))
    H = G.copy()
    H.remove_nodes_from(["src", "snk"])
    for cyc in nx.simple_cycles(H):
        found.add(tuple(sorted(n[1] for n in cyc if n[0] == "c")))
    seeds = bruteforce.seeds_of(net, target)
    out = []
    for cols in found:
        if len(cols) > max_len:
            continue
        if any(twin[a] in cols for a in cols if twin[a] >= 0):
            continue
        if not seeds.intersection(cols):
            continue
        out.append(cols)
    return sorted(out, key=lambda c: (len(c), c))


@pytest.mark.parametrize("seed", range(12))
def test_type1_equals_simple_paths_and_cycles(oracle_lib, seed):
    net = synth.type1(seed)
    for t in list(net.targets) + [-1]:
        for L in (3, 6, 40):
            sup, ctr = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(L, 0, 0, 0))
            assert oracle_lib.supports_to_lists(sup) == _type1_expected(net, t, L), (t, L)


@pytest.mark.parametrize("seed", range(4))
def test_tiny_results_are_efms_and_within_bruteforce(oracle_lib, seed):
    from oracle import bruteforce

    net = synth.tiny(seed)
    S_int, twin, full = bruteforce.split(net)
    efms = set(bruteforce.efm_supports(net))
    recall = []
    for t in list(net.targets) + [-1]:
        L = 8
        sup, ctr = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(L, 2, 0, 0))
        res = oracle_lib.supports_to_lists(sup)
        seeds = bruteforce.seeds_of(net, t)
        truth = {e for e in efms if len(e) <= L and seeds.intersection(e)}
        for cols in res:
            # precision: each result is an EFM (exact), within limits
            assert bruteforce.is_efm_support(S_int, cols)
            assert len(cols) <= L and seeds.intersection(cols)
            assert not any(twin[a] in cols for a in cols if twin[a] >= 0)
            assert cols in truth
        recall.append((len(res), len(truth)))
    assert sum(r for r, _ in recall) > 0
    print("recall (found, true) per target:", recall)


def test_overflow_chain(oracle_lib):
    """Chain t <- X0 <- 4 X1 <- 16 X2 ...: the shortfall on X_i is 4^i while a
    second shortfall (W, two inputs) keeps the gcd at 1, so the child
    reaching X16 (4^16 > 2^31 - 1) is dropped as overflow."""
    n = 17  # X0..X16
    mets = n + 1 + 3  # X*, W, t, S, S2
    W_, t, Sx, S2 = n, n + 1, n + 2, n + 3
    cols = []
    c = np.zeros(mets, dtype=np.int64)
    c[0], c[W_], c[t] = -1, -1, 1  # r0: X0 + W -> t
    cols.append(c)
    for i in range(1, n):  # r_i: 4 X_i -> X_{i-1}
        c = np.zeros(mets, dtype=np.int64)
        c[i], c[i - 1] = -4, 1
        cols.append(c)
    c = np.zeros(mets, dtype=np.int64)
    c[Sx], c[n - 1] = -1, 1  # S -> X16
    cols.append(c)
    for src in (Sx, S2):  # two inputs of W
        c = np.zeros(mets, dtype=np.int64)
        c[src], c[W_] = -1, 1
        cols.append(c)
    S = np.stack(cols, axis=1)
    ext = np.zeros(mets, dtype=np.uint8)
    ext[[t, Sx, S2]] = 1
    net = synth.Network.from_dense(S, np.zeros(S.shape[1], np.uint8), ext)
    sup, ctr = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(40, 0, 0, 0))
    assert ctr["overflow"] == 1 and ctr["status"] & 4
    assert ctr["expansions"] == 16 and len(sup) == 0
    # a shorter length limit stops before the overflowing step
    sup, ctr = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(10, 0, 0, 0))
    assert ctr["overflow"] == 0 and ctr["expansions"] == 9


def test_truncation_and_cap_are_level_granular(oracle_lib):
    net = synth.tiny(3)
    full, cf = oracle_lib.enumerate_pathways(net, -1, oracle_lib.Limits(8, 1, 0, 0))
    assert cf["status"] == 0
    # cap: stop after the level where the count reaches the cap, keep the smallest
    cap = 5
    sup, c = oracle_lib.enumerate_pathways(net, -1, oracle_lib.Limits(8, 1, cap, 0))
    assert c["status"] & 2 and len(sup) == cap
    got = oracle_lib.supports_to_lists(sup)
    assert got == sorted(got, key=lambda x: (len(x), x))
    # truncation: stop before expanding a frontier larger than the budget
    sup, t = oracle_lib.enumerate_pathways(net, -1, oracle_lib.Limits(8, 1, 0, 50))
    assert t["status"] & 1 and t["frontier_max"] <= 50
    assert set(oracle_lib.supports_to_lists(sup)) <= set(oracle_lib.supports_to_lists(full))


def test_invalid_inputs_rejected(oracle_lib):
    net = synth.tiny(0)
    bad = synth.Network(net.n_met, net.n_rxn, net.row_ptr.copy(), net.col_idx.copy(), net.coef.copy(),
                        net.reversible, net.external)
    bad.coef[0] = 0
    with pytest.raises(RuntimeError):
        oracle_lib.enumerate_pathways(bad, -1, oracle_lib.Limits(8, 1, 0, 0))
    with pytest.raises(RuntimeError):
        oracle_lib.enumerate_pathways(net, net.n_met, oracle_lib.Limits(8, 1, 0, 0))
    with pytest.raises(RuntimeError):
        oracle_lib.enumerate_pathways(net, -1, oracle_lib.Limits(65, 1, 0, 0))


def test_first_k_is_prefix_of_full_enumeration(oracle_lib):
    """first_k by popcount deepening equals the k smallest of the complete
    enumeration (no budget, no cap)."""
    for seed in range(6):
        net = synth.tiny(seed)
        for t in list(net.targets) + [-1]:
            full, _ = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(9, 1, 0, 0))
            for k in (1, 3, 10, 1000):
                got, _ = oracle_lib.first_k(net, t, k, 9, 1)
                assert np.array_equal(got, full[:k]), (seed, t, k)


def test_budgeted_first_k_is_certified_only_when_exact(oracle_lib):
    """first_k_within: a certified answer is the k smallest of the complete
    enumeration; an answer is uncertified exactly when the deepening run it
    stopped at overflowed the budget somewhere."""
    seen_uncertified = seen_certified = 0
    for seed in range(6):
        net = synth.tiny(seed)
        for t in list(net.targets) + [-1]:
            full, _ = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(9, 1, 0, 0))
            for k in (1, 3, 10):
                for budget in (2, 5, 40):
                    got, P, ok = oracle_lib.first_k_within(net, t, k, 9, 1, budget)
                    _, ctr = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(P, 1, 0, budget))
                    assert ok == (not ctr["status"] & oracle_lib.TRUNCATED), (seed, t, k, budget)
                    if ok:
                        assert np.array_equal(got, full[:k]), (seed, t, k, budget)
                        seen_certified += 1
                    else:
                        seen_uncertified += 1
    assert seen_certified > 0 and seen_uncertified > 0


def test_splitmix_published_outputs(oracle_lib):
    """The walks' counter-based generator is SplitMix64: from state 0 its
    first outputs are the published 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4,
    0x06c45d188009454f."""
    assert [oracle_lib.splitmix_at(0, c) for c in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                                0x06C45D188009454F]


def test_sampled_results_are_exhaustive_results(oracle_lib):
    """Every walk follows one branch sequence of the traversal, so the
    sampled results lie inside the exhaustive result set; each walk ends in
    exactly one way; enough walks find every result of a tiny network."""
    for seed in range(6):
        net = synth.tiny(seed)
        for t in list(net.targets) + [-1]:
            full, _ = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(9, 1, 0, 0))
            sup, c = oracle_lib.sample_pathways(net, t, oracle_lib.Limits(9, 1), 11, 3000)
            assert set(oracle_lib.supports_to_lists(sup)) <= set(oracle_lib.supports_to_lists(full))
            assert c["balanced"] + c["overflow"] + c["pruned"] == c["seeds"]
            assert c["results"] == len(sup) <= c["candidates"] <= c["balanced"]
    net = synth.tiny(3)
    full, _ = oracle_lib.enumerate_pathways(net, -1, oracle_lib.Limits(9, 1, 0, 0))
    sup, _ = oracle_lib.sample_pathways(net, -1, oracle_lib.Limits(9, 1), 5, 200000)
    assert np.array_equal(sup, full)
    net = synth.core()
    full, _ = oracle_lib.enumerate_pathways(net, 63, oracle_lib.Limits(16, 4, 0, 0))
    sup, _ = oracle_lib.sample_pathways(net, 63, oracle_lib.Limits(16, 4), 3, 20000)
    assert set(oracle_lib.supports_to_lists(sup)) <= set(oracle_lib.supports_to_lists(full)) and len(sup) > 0


def test_sampling_a_chain_is_deterministic(oracle_lib):
    """On the hand-worked chain every step has one valid branch, so every
    walk reaches the one pathway."""
    case = next(c for c in _handworked() if c["name"] == "chain")
    net = synth.Network.from_dense(case["S"], case["reversible"], case["external"])
    sup, c = oracle_lib.sample_pathways(net, case["target"], oracle_lib.Limits(case["max_len"], case["max_secondary"]),
                                        1, 50)
    assert oracle_lib.supports_to_lists(sup) == [tuple(x) for x in case["expected"]]
    assert c["balanced"] == 50 and c["candidates"] == 1


def test_flux_vectors_hand_worked(oracle_lib):
    from oracle import flux

    for case in _handworked():
        if "flux" not in case:
            continue
        net = synth.Network.from_dense(case["S"], case["reversible"], case["external"])
        sup, _ = oracle_lib.enumerate_pathways(net, case["target"],
                                               oracle_lib.Limits(case["max_len"], case["max_secondary"], 0, 0,
                                                                 subtractive=case.get("subtractive", False)))
        assert flux.flux_vectors(net, sup) == case["flux"], case["name"]


def test_flux_vectors_match_the_walked_flux(oracle_lib):
    """The null-space vector of each result equals, up to scale, the flux
    vector the pure-Python traversal carries along the path that reached it
    (a different computation: accumulated AND updates, Eq. 3 / Eq. 4)."""
    from math import gcd

    from oracle import bruteforce, flux, reference

    for seed in range(6):
        net = synth.tiny(seed)
        S_int, _, _ = bruteforce.split(net)
        for t in list(net.targets) + [-1]:
            walked = {}
            res, _ = reference.enumerate_reference(net, t, 9, 1, fluxes=walked)
            for U in res:
                cols = [k for k in range(64) if (U >> k) & 1]
                v = [walked[U][k] for k in cols]
                g = 0
                for x in v:
                    g = gcd(g, x)
                want = [x // g for x in v]
                got = flux.flux_vector(S_int, cols)
                assert got == want, (seed, t, cols)
                assert not np.any(S_int[:, cols] @ np.array(got, dtype=np.int64))


def test_seed_sets(oracle_lib):
    """Traversal from a seed set R_in (Prop. 1): the union over single
    columns j of the results from {j} is the result set of the all-column
    run; every result from R_in contains R_in and is an EFM; a seed set that
    is itself balanced with unit fluxes is its own result; twin pairs and
    repeated columns are rejected."""
    from oracle import bruteforce

    for seed in range(5):
        net = synth.tiny(seed)
        S_int, twin, _ = bruteforce.split(net)
        full, _ = oracle_lib.enumerate_pathways(net, -1, oracle_lib.Limits(9, 1, 0, 0))
        union = set()
        for j in range(S_int.shape[1]):
            sup, c = oracle_lib.enumerate_from(net, [j], oracle_lib.Limits(9, 1, 0, 0))
            got = oracle_lib.supports_to_lists(sup)
            assert all(j in cols for cols in got)
            union |= set(got)
        assert union == set(oracle_lib.supports_to_lists(full)), seed
        rng = np.random.default_rng(seed)
        for _ in range(10):
            R = sorted(int(x) for x in rng.choice(S_int.shape[1], size=2, replace=False))
            if twin[R[0]] == R[1]:
                continue
            sup, _ = oracle_lib.enumerate_from(net, R, oracle_lib.Limits(9, 2, 0, 0))
            for cols in oracle_lib.supports_to_lists(sup):
                assert set(R) <= set(cols) and bruteforce.is_efm_support(S_int, cols)
    case = next(c for c in _handworked() if c["name"] == "chain")
    net = synth.Network.from_dense(case["S"], case["reversible"], case["external"])
    sup, c = oracle_lib.enumerate_from(net, [0, 1], oracle_lib.Limits(4, 0, 0, 0))
    assert oracle_lib.supports_to_lists(sup) == [(0, 1)] and c["balanced"] == 1 and c["levels"] == 1
    net = synth.tiny(0)
    _, twin, _ = bruteforce.split(net)
    a = next(k for k in range(len(twin)) if twin[k] >= 0)
    for bad in ([a, twin[a]], [1, 1], [], [10**6]):
        with pytest.raises(RuntimeError):
            oracle_lib.enumerate_from(net, bad, oracle_lib.Limits(9, 1, 0, 0))


def _dep_from_cycles(net, L):
    """Flux-dependent pairs from the simple cycles through each metabolite
    of the bipartite metabolite / column digraph (networkx), at most L
    columns long: a first-return walk shortens to a simple cycle with the
    same leaving and returning columns."""
    import networkx as nx

    from oracle import bruteforce

    S_int, _, _ = bruteforce.split(net)
    M, N = S_int.shape
    G = nx.DiGraph()
    for k in range(N):
        for m in range(M):
            if S_int[m, k] < 0:
                G.add_edge(("m", m), ("c", k))
            if S_int[m, k] > 0:
                G.add_edge(("c", k), ("m", m))
    dep_out = np.zeros((M, N), dtype=bool)
    dep_in = np.zeros((M, N), dtype=bool)
    for cyc in nx.simple_cycles(G, length_bound=2 * L):
        for pos, node in enumerate(cyc):
            if node[0] != "m":
                continue
            i = node[1]
            dep_out[i, cyc[(pos + 1) % len(cyc)][1]] = True
            dep_in[i, cyc[pos - 1][1]] = True
    return dep_out, dep_in


def test_dependent_reactions_match_simple_cycles():
    from oracle import depthy

    for seed in range(4):
        for net in (synth.tiny(seed), synth.type1(seed)):
            for L in (1, 2, 3, 4):
                a_out, a_in = depthy.dependent_reactions(net, L)
                b_out, b_in = _dep_from_cycles(net, L)
                assert np.array_equal(a_out, b_out) and np.array_equal(a_in, b_in), (seed, net.name, L)


def test_dependent_reactions_hand_worked():
    """Internal A, B; columns c0: A -> B, c1: B -> A, c2: B -> (out), c3:
    (in) -> A.  The only cycle is A -c0-> B -c1-> A: for A, c0 leaves and c1
    returns; for B, c1 leaves and c0 returns.  Depth 1 finds nothing."""
    from oracle import depthy

    S = [[-1, 1, 0, 1], [1, -1, -1, 0], [0, 0, 1, 0], [0, 0, 0, -1]]
    net = synth.Network.from_dense(S, [0, 0, 0, 0], [0, 0, 1, 1])
    o, i = depthy.dependent_reactions(net, 2)
    assert o.tolist() == [[True, False, False, False], [False, True, False, False]]
    assert i.tolist() == [[False, True, False, False], [True, False, False, False]]
    o, i = depthy.dependent_reactions(net, 1)
    assert not o.any() and not i.any()


@pytest.mark.parametrize("seed", range(6))
def test_python_reference_agrees_on_tiny_networks(oracle_lib, seed):
    """Two independent restatements of the traversal (plain C with rays; pure
    Python with exact fractions and explicit flux vectors) give the same
    results and counters on random tiny networks, for every target."""
    from oracle import reference

    net = synth.tiny(seed)
    for t in list(net.targets) + [-1]:
        for L, S in ((6, 0), (8, 1), (9, 2)):
            sup, ctr = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(L, S, 0, 0))
            res, rctr = reference.enumerate_reference(net, t, L, S)
            got = [tuple(k for k in range(64) if (U >> k) & 1) for U in res]
            assert got == oracle_lib.supports_to_lists(sup), (seed, t, L, S)
            for key in ("levels", "seeds", "expansions", "overflow", "balanced", "candidates", "results", "pruned",
                        "frontier", "frontier_max", "status"):
                assert ctr[key] == rctr[key], (seed, t, L, S, key)


def test_python_walks_agree_with_c_walks(oracle_lib):
    """The Monte-Carlo walks restated in pure Python give the C oracle's
    results and counters."""
    from oracle import reference

    for seed in range(4):
        net = synth.tiny(seed)
        for t in list(net.targets) + [-1]:
            sup, ctr = oracle_lib.sample_pathways(net, t, oracle_lib.Limits(9, 2), 100 + seed, 300)
            res, rctr = reference.sample_reference(net, t, 9, 2, 100 + seed, 300)
            got = [tuple(k for k in range(64) if (U >> k) & 1) for U in res]
            assert got == oracle_lib.supports_to_lists(sup), (seed, t)
            assert ctr == rctr, (seed, t, ctr, rctr)


def test_maximal_network_chain_in_closed_form(oracle_lib):
    """At the library's size limits (1024 internal metabolites, 4096 split
    columns, 64-word supports, coefficients up to 524287) the target T of
    the maximal network ends a linear chain, so its pathways are known by
    construction: r_0..r_i closed by the side uptake of m_i (i = 10, 20, 30,
    40, 50), and the whole chain r_0..r_62 closed by the uptake r_63.  Along
    a chain each intermediate m_{j-1} balances its producer r_j against its
    consumer r_{j-1}, so v_j = v_{j-1} * |S[m_{j-1}, r_{j-1}]| / S[m_{j-1}, r_j]
    (Def. 3), scaled to the primitive integer vector."""
    from fractions import Fraction
    from math import gcd, lcm

    from oracle import bruteforce, flux

    net = synth.maximal()
    S = net.dense()
    T = net.targets[0]
    rx, d = oracle_lib.column_map(net)
    col = {(int(r), int(s)): k for k, (r, s) in enumerate(zip(rx, d))}
    side = {10: 64, 20: 65, 30: 66, 40: 67, 50: 68}  # reactions of the side uptakes
    closes = [(i, side[i]) for i in (10, 20, 30, 40, 50)] + [(62, 63)]
    want_sup, want_flux = [], []
    for i, last in closes:
        rxns = list(range(i + 1)) + [last]
        v = {0: Fraction(1)}
        for j in range(1, i + 1):
            v[j] = v[j - 1] * -S[j - 1, j - 1] / S[j - 1, j]
        v[last] = v[i] * -S[i, i] / S[i, last]
        den = lcm(*(x.denominator for x in v.values()))
        ints = {r: int(x * den) for r, x in v.items()}
        g = 0
        for x in ints.values():
            g = gcd(g, x)
        cols = sorted(col[(r, 1)] for r in rxns)
        by_col = {col[(r, 1)]: ints[r] // g for r in rxns}
        want_sup.append(tuple(cols))
        want_flux.append([by_col[c] for c in cols])
    sup, ctr = oracle_lib.enumerate_pathways(net, T, oracle_lib.Limits(64, 4, 0, 0))
    got = oracle_lib.supports_to_lists(sup)
    assert [tuple(c) for c in got] == want_sup
    assert ctr["status"] == 0 and ctr["results"] == 6
    S_int, _, _ = bruteforce.split(net)
    for cols, w in zip(got, want_flux):
        rows = np.nonzero(np.any(S_int[:, list(cols)] != 0, axis=1))[0]
        assert flux.flux_vector(S_int[rows], cols) == w
    assert max(want_flux[-1]) == 6 * synth.MAX_COEF


def test_walks_choose_uniformly_among_valid_branches(oracle_lib):
    """The Monte-Carlo mode takes one valid OR branch per step, each with the
    same probability (Alg. 3's random input, Theorem 1).  On a chain with
    side uptakes the probability of each result is a closed form: target T
    is made from m_0 by r0; m_{i-1} from m_i by r_i (i = 1..5); m_5 from the
    uptake X by r6; m_1 and m_3 each have one more producer (an uptake of Y),
    m_4 two more.  A walk ends at m_1 with probability 1/2, at m_3 with 1/4,
    and at m_4 with 1/12 for each of its three producers (two uptakes, and
    r5 followed by the forced r6).  6000 walks, one generator key each, must
    fit these probabilities (chi-square, 4 degrees of freedom, p > 1e-4)."""
    n_int, T, X, Y = 6, 6, 7, 8
    cols = []

    def rxn(*entries):
        c = np.zeros(9, dtype=np.int64)
        for m, v in entries:
            c[m] = v
        cols.append(c)

    rxn((0, -1), (T, 1))
    for i in range(1, 6):
        rxn((i, -1), (i - 1, 1))
    rxn((X, -1), (5, 1))
    for m in (1, 3, 4, 4):
        rxn((Y, -1), (m, 1))
    S = np.stack(cols, axis=1)
    ext = np.zeros(9, dtype=np.uint8)
    ext[n_int:] = 1
    net = synth.Network.from_dense(S, np.zeros(S.shape[1], np.uint8), ext)
    lists = {(0, 1, 7): 0, (0, 1, 2, 3, 8): 1, (0, 1, 2, 3, 4, 9): 2, (0, 1, 2, 3, 4, 10): 3,
             (0, 1, 2, 3, 4, 5, 6): 4}
    probs = np.array([1 / 2, 1 / 4, 1 / 12, 1 / 12, 1 / 12])
    counts = np.zeros(5)
    n = 6000
    for seed in range(n):
        sup, ctr = oracle_lib.sample_pathways(net, T, oracle_lib.Limits(20, 0), seed, 1)
        assert ctr["balanced"] == 1 and len(sup) == 1
        counts[lists[tuple(oracle_lib.supports_to_lists(sup)[0])]] += 1
    expected = n * probs
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    assert chi2 < 23.5, (counts, expected, chi2)  # 23.5 = chi-square(4) quantile at 1 - 1e-4
