"""The subtractive variant (Eq. 5 with the zero-flux discard of Prop. 3),
pinned without a GPU.

* hand-worked: tests/golden/handworked.json, cases "subtractive_step_needed"
  (a result only a subtractive step reaches, three children discarded by
  Prop. 3) and "subtractive_network_additive_only" (the same network without
  the variant finds nothing) -- run by test_oracle_pins.py;
* two spellings agree: the C oracle (extra flux updated with the step,
  (EF, v) rays) and the pure-Python restatement (extra flux recomputed as
  S_int v from the explicit flux vector at every step) give the same results
  and every counter;
* the additive steps are a subset of the variant's, so with no frontier
  budget every additive result is also a result of the variant;
* precision: every result of the variant is an elementary mode (exact null
  space), and is inside the brute-force EFM set of the network.
"""
import pytest

from paper_1804_02867_gb300 import synth


def _lists(res):
    return [tuple(k for k in range(64) if (U >> k) & 1) for U in res]


@pytest.mark.parametrize("seed", range(6))
def test_two_spellings_of_the_variant_agree(oracle_lib, seed):
    from oracle import reference

    net = synth.tiny(seed)
    for t in list(net.targets) + [-1]:
        for L, S in ((7, 1), (9, 2)):
            sup, ctr = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(L, S, 0, 0, subtractive=True))
            res, rctr = reference.enumerate_subtractive(net, t, L, S)
            assert _lists(res) == oracle_lib.supports_to_lists(sup), (seed, t, L, S)
            assert ctr == rctr, (seed, t, L, S)


def test_two_spellings_agree_with_budget_cap_and_no_rule(oracle_lib):
    from oracle import reference

    net = synth.tiny(3)
    for t in list(net.targets) + [-1]:
        for kw in (dict(max_frontier=20), dict(max_results=2), dict(prune=False)):
            lim = oracle_lib.Limits(9, 2, kw.get("max_results", 0), kw.get("max_frontier", 0),
                                    prune=kw.get("prune", True), subtractive=True)
            sup, ctr = oracle_lib.enumerate_pathways(net, t, lim)
            res, rctr = reference.enumerate_subtractive(net, t, 9, 2, **kw)
            assert _lists(res) == oracle_lib.supports_to_lists(sup), (t, kw)
            assert ctr == rctr, (t, kw)


@pytest.mark.parametrize("seed", range(8))
def test_additive_results_are_variant_results(oracle_lib, seed):
    net = synth.tiny(seed)
    grew = 0
    for t in list(net.targets) + [-1]:
        for L, S in ((8, 1), (9, 2)):
            add, _ = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(L, S, 0, 0))
            sub, ctr = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(L, S, 0, 0, subtractive=True))
            a, b = set(oracle_lib.supports_to_lists(add)), set(oracle_lib.supports_to_lists(sub))
            assert a <= b, (seed, t, L, S)
            grew += len(b - a)
            assert ctr["zero_flux"] >= 0


def test_variant_reaches_more_and_discards(oracle_lib):
    """Across the tiny networks the variant finds results the additive
    traversal cannot, and Prop. 3 discards children."""
    more = discarded = 0
    for seed in range(8):
        net = synth.tiny(seed)
        for t in list(net.targets) + [-1]:
            add, _ = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(9, 2, 0, 0))
            sub, ctr = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(9, 2, 0, 0, subtractive=True))
            more += len(set(oracle_lib.supports_to_lists(sub)) - set(oracle_lib.supports_to_lists(add)))
            discarded += ctr["zero_flux"]
    assert more > 0 and discarded > 0


@pytest.mark.parametrize("seed", range(4))
def test_variant_results_are_efms(oracle_lib, seed):
    from oracle import bruteforce

    net = synth.tiny(seed)
    S_int, twin, full = bruteforce.split(net)
    efms = set(bruteforce.efm_supports(net))
    for t in list(net.targets) + [-1]:
        sup, _ = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(9, 2, 0, 0, subtractive=True))
        seeds = bruteforce.seeds_of(net, t)
        for cols in oracle_lib.supports_to_lists(sup):
            assert bruteforce.is_efm_support(S_int, cols)
            assert cols in efms and seeds.intersection(cols)
            assert not any(twin[a] in cols for a in cols if twin[a] >= 0)


def test_variant_on_the_core_network(oracle_lib):
    """Core-shaped network, short pathways: the variant keeps every additive
    result and its own results are elementary (exact rank)."""
    import numpy as np

    from oracle import bruteforce

    net = synth.core()
    S_int, _, _ = bruteforce.split(net)
    for t in net.targets[:4]:
        add, _ = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(10, 2, 0, 0))
        sub, ctr = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(10, 2, 0, 0, subtractive=True))
        a, b = set(oracle_lib.supports_to_lists(add)), set(oracle_lib.supports_to_lists(sub))
        assert a <= b, t
        for cols in b - a:
            sub_m = np.asarray(S_int)[:, list(cols)]
            assert len(cols) - oracle_lib.rank(sub_m) == 1
