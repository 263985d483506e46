"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Supports must be bit-identical and in the same order; every counter must
match (the definitions are shared; the implementations are not).  Sizes run
from hand-worked networks through seeded tiny networks to the core-shaped
network at reduced and full frontier budgets.
"""
import json
import os

import numpy as np
import pytest

from paper_1804_02867_gb300 import synth

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def efm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_02867_gb300 import build, efmgraph

    build.build()
    efmgraph.load_library()
    return efmgraph


def run_gpu(efm, net, targets, L, S, max_results=0, max_frontier=0):
    with efm.Network(net) as nw:
        return efm.enumerate_targets(nw, targets, L, S, max_results, max_frontier)


def run_oracle(oracle_lib, net, t, L, S, max_results=0, max_frontier=0):
    return oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(L, S, max_results, max_frontier))


def assert_same(oracle_lib, efm, net, targets, L, S, max_results=0, max_frontier=0, check_counters=True):
    got = run_gpu(efm, net, targets, L, S, max_results, max_frontier)
    for t, (sup, ctr) in zip(targets, got):
        osup, octr = run_oracle(oracle_lib, net, t, L, S, max_results, max_frontier)
        assert sup.shape == osup.shape, (net.name, t, sup.shape, osup.shape, ctr, octr)
        assert np.array_equal(sup, osup), (net.name, t)
        if check_counters:
            assert ctr == octr, (net.name, t, ctr, octr)
    return got


def test_handworked(oracle_lib, efm):
    with open(os.path.join(HERE, "golden", "handworked.json")) as f:
        cases = json.load(f)["cases"]
    for case in cases:
        if case.get("subtractive"):
            continue  # the Eq. 5 variant: tests/test_gpu_subtractive.py
        net = synth.Network.from_dense(case["S"], case["reversible"], case["external"], name=case["name"])
        (sup, ctr), = run_gpu(efm, net, [case["target"]], case["max_len"], case["max_secondary"])
        assert [tuple(c) for c in __import__("oracle").supports_to_lists(sup)] == \
            [tuple(x) for x in case["expected"]], case["name"]
        for k, v in case.get("counters", {}).items():
            assert ctr[k] == v, (case["name"], k, ctr)


@pytest.mark.parametrize("seed", range(24))
def test_tiny_networks(oracle_lib, efm, seed):
    net = synth.tiny(seed)
    targets = list(net.targets) + [-1]
    for L, S in ((8, 1), (6, 0), (12, 2)):
        assert_same(oracle_lib, efm, net, targets, L, S)


@pytest.mark.parametrize("seed", range(8))
def test_type1_networks(oracle_lib, efm, seed):
    net = synth.type1(seed)
    assert_same(oracle_lib, efm, net, list(net.targets) + [-1], 40, 0)


@pytest.mark.parametrize("budget", [2**10, 2**14, 2**17])
def test_core_network_budgets(oracle_lib, efm, budget):
    """Core-shaped network (72 metabolites, 95 reactions, 114 columns, two
    64-bit words per support): all 8 targets, L = 30, 4 secondary steps,
    truncation at several frontier budgets (multi-tile frontiers with a
    ragged tail, hash tables of many sizes)."""
    net = synth.core()
    assert_same(oracle_lib, efm, net, net.targets, 30, 4, 0, budget)


def test_core_network_cap(oracle_lib, efm):
    net = synth.core()
    got = assert_same(oracle_lib, efm, net, net.targets[:4], 30, 4, 5, 2**16)
    assert any(c["status"] & 2 for _, c in got)


def test_batched_members(oracle_lib, efm):
    """Uneven networks of the batched workload (10-120 metabolites)."""
    for i in range(12):
        net = synth.batched_member(i)
        L = min(30, net.split_columns())
        assert_same(oracle_lib, efm, net, net.targets, L, 4, 0, 2**12)


def test_overflow_chain(oracle_lib, efm):
    n = 17
    mets = n + 4
    W_, t, Sx, S2 = n, n + 1, n + 2, n + 3
    cols = []
    c = np.zeros(mets, dtype=np.int64)
    c[0], c[W_], c[t] = -1, -1, 1
    cols.append(c)
    for i in range(1, n):
        c = np.zeros(mets, dtype=np.int64)
        c[i], c[i - 1] = -4, 1
        cols.append(c)
    c = np.zeros(mets, dtype=np.int64)
    c[Sx], c[n - 1] = -1, 1
    cols.append(c)
    for src in (Sx, S2):
        c = np.zeros(mets, dtype=np.int64)
        c[src], c[W_] = -1, 1
        cols.append(c)
    S = np.stack(cols, axis=1)
    ext = np.zeros(mets, dtype=np.uint8)
    ext[[t, Sx, S2]] = 1
    net = synth.Network.from_dense(S, np.zeros(S.shape[1], np.uint8), ext, name="overflow")
    got = assert_same(oracle_lib, efm, net, [t], 40, 0)
    assert got[0][1]["overflow"] == 1 and got[0][1]["status"] & 4


def test_empty_and_degenerate(oracle_lib, efm):
    # a target nothing produces: no seeds, no results
    net = synth.tiny(1)
    S = net.dense()
    cons_only = [m for m in range(net.n_met) if net.external[m] and not (S[m] > 0).any()
                 and not any(S[m, j] < 0 and net.reversible[j] for j in range(net.n_rxn))]
    for t in cons_only:
        (sup, ctr), = run_gpu(efm, net, [t], 8, 1)
        assert sup.shape[0] == 0 and ctr["seeds"] == 0
    # max_len 1: only single-column balanced seeds can be results
    assert_same(oracle_lib, efm, net, list(net.targets) + [-1], 1, 0)
    # frontier budget 1: truncation right after the seeds
    assert_same(oracle_lib, efm, synth.core(), synth.core().targets[:2], 30, 4, 0, 1)


def test_invalid_inputs(efm):
    net = synth.tiny(0)
    coef = net.coef.copy()
    coef[0] = 0
    with pytest.raises(efm.EfmError) as e:
        efm.efm_load_network(net.n_met, net.n_rxn, net.row_ptr, net.col_idx, coef, net.reversible, net.external)
    assert e.value.code == -1
    col = net.col_idx.copy()
    col[0] = net.n_rxn
    with pytest.raises(efm.EfmError):
        efm.efm_load_network(net.n_met, net.n_rxn, net.row_ptr, col, net.coef, net.reversible, net.external)
    with efm.Network(net) as nw:
        with pytest.raises(efm.EfmError):
            efm.efm_find_pathways(nw.handle, [net.n_met], 8, 1)
        with pytest.raises(efm.EfmError):
            efm.efm_find_pathways(nw.handle, [-1], 65, 1)
        with pytest.raises(efm.EfmError):
            efm.efm_find_pathways(nw.handle, [-1], 8, -1)


def test_column_map_matches_split(oracle_lib, efm):
    net = synth.core()
    with efm.Network(net) as nw:
        rx, d = efm.efm_column_map(nw.handle)
        assert nw.n_columns == net.split_columns() and nw.words == 2 and nw.n_internal == 58
    orx, od = oracle_lib.column_map(net)
    assert np.array_equal(rx, orx) and np.array_equal(d.astype(np.int32), od)


def test_core_full_budget_properties(oracle_lib, efm):
    """The benchmark's launch: core network, 8 targets, L = 30, 4 secondary
    steps, frontier budget 2^26.  Checked via properties that hold at any
    size and on sampled outputs the oracle computes one by one:
      * each result is elementary (exact oracle rank: nullity of
        S_int[:, U] is 1), within L, without a reversible pair, and contains
        a column producing the target;
      * results of the oracle at a smaller budget are a subset (truncation
        is level-granular, a larger budget never stops earlier).
    """
    from oracle import bruteforce

    net = synth.core()
    S_int, twin, full = bruteforce.split(net)
    got = run_gpu(efm, net, net.targets, 30, 4, 0, 2**26)
    rng = np.random.default_rng(0)
    for t, (sup, ctr) in zip(net.targets, got):
        lists = oracle_lib.supports_to_lists(sup)
        assert lists == sorted(lists, key=lambda c: (len(c), c))
        seeds = bruteforce.seeds_of(net, t)
        pick = rng.choice(len(lists), size=min(len(lists), 40), replace=False) if lists else []
        for i in pick:
            cols = list(lists[i])
            A = S_int[:, cols]
            A = A[np.any(A != 0, axis=1)]
            assert len(cols) - (oracle_lib.rank(A) if A.size else 0) == 1
            assert len(cols) <= 30 and seeds.intersection(cols)
            assert not any(twin[a] in cols for a in cols if twin[a] >= 0)
        small, _ = run_oracle(oracle_lib, net, t, 30, 4, 0, 2**14)
        assert set(oracle_lib.supports_to_lists(small)) <= set(lists)
        assert ctr["expansions"] > 0
