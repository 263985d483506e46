"""The superset rule is an optimisation, not part of the definition.

The traversal's result set is defined without it: every support some
sequence of valid expansions reaches that is balanced and has nullity 1
(Def. 3).  The rule drops an unbalanced child whose new column completes a
result accepted at an earlier level; it is exact because any balanced
support strictly containing an elementary mode has nullity at least 2.
These tests run the oracles with and without the rule, with no frontier
budget (truncation depends on frontier sizes, which the rule changes), and
require the same supports and status.  Only the pruned counter and the
counters of the extra states it saves (frontier, expansions, balanced,
candidates) may differ.  No GPU is needed.
"""
import numpy as np
import pytest

from paper_1804_02867_gb300 import synth


def _both(oracle_lib, net, t, L, S):
    on = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(L, S, 0, 0))
    off = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(L, S, 0, 0, prune=False))
    return on, off


def _same_results(on, off, where):
    (a, ca), (b, cb) = on, off
    assert np.array_equal(a, b), where
    assert ca["results"] == cb["results"] and ca["status"] == cb["status"], where
    assert cb["pruned"] == 0, where
    # the rule only removes work
    assert cb["frontier"] >= ca["frontier"] and cb["expansions"] >= ca["expansions"], where


@pytest.mark.parametrize("seed", range(8))
def test_prune_free_tiny_networks_give_the_same_results(oracle_lib, seed):
    net = synth.tiny(seed)
    for t in list(net.targets) + [-1]:
        for L, S in ((8, 1), (9, 2), (12, 2)):
            _same_results(*_both(oracle_lib, net, t, L, S), (seed, t, L, S))


@pytest.mark.parametrize("seed", range(6))
def test_prune_free_type1_networks_with_secondary_steps(oracle_lib, seed):
    net = synth.type1(seed)
    for t in list(net.targets) + [-1]:
        for L, S in ((6, 1), (40, 2)):
            _same_results(*_both(oracle_lib, net, t, L, S), (seed, t, L, S))


def test_prune_free_core_network(oracle_lib):
    """The core-shaped network (58 internal metabolites, 114 columns) at
    max_len 15, every target: the rule fires thousands of times and the
    results do not move."""
    net = synth.core()
    fired = 0
    for t in net.targets:
        on, off = _both(oracle_lib, net, t, 15, 4)
        _same_results(on, off, t)
        fired += on[1]["pruned"]
    assert fired > 1000


def test_rule_fires_on_the_small_cases(oracle_lib):
    """The pins above are not vacuous: the rule prunes children there."""
    fired = 0
    for seed in range(8):
        net = synth.tiny(seed)
        for t in list(net.targets) + [-1]:
            fired += _both(oracle_lib, net, t, 12, 2)[0][1]["pruned"]
    assert fired > 0


@pytest.mark.parametrize("seed", range(4))
def test_python_reference_without_the_rule_agrees(oracle_lib, seed):
    """Both spellings of the definition without the rule (C rays; Python with
    explicit flux vectors) agree on results and every counter."""
    from oracle import reference

    net = synth.tiny(seed)
    for t in list(net.targets) + [-1]:
        for L, S in ((8, 1), (9, 2)):
            sup, ctr = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(L, S, 0, 0, prune=False))
            res, rctr = reference.enumerate_reference(net, t, L, S, prune=False)
            got = [tuple(k for k in range(64) if (U >> k) & 1) for U in res]
            assert got == oracle_lib.supports_to_lists(sup), (seed, t, L, S)
            assert ctr == rctr, (seed, t, L, S)


def test_extreme_coefficients_agree_with_unbounded_integers(oracle_lib):
    """Coefficients up to 2^31 - 1 (the largest the oracle accepts): the C
    oracle's 64-bit update must give what unbounded Python integers give,
    overflow drops included."""
    from oracle import reference

    big = 2**31 - 1
    rng = np.random.default_rng(11)
    checked = 0
    for trial in range(30):
        net = synth.tiny(100 + trial)
        coef = np.asarray(net.coef, dtype=np.int64)
        pick = rng.random(len(coef)) < 0.35
        mag = rng.choice([big, big - 1, 3 * 5 * 7 * 11 * 13 * 17 * 19 * 23, 2**30 + 7], size=len(coef))
        coef = np.where(pick, np.sign(coef) * mag, coef).astype(np.int32)
        net.coef = coef
        for t in list(net.targets) + [-1]:
            sup, ctr = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(8, 2, 0, 0))
            res, rctr = reference.enumerate_reference(net, t, 8, 2)
            got = [tuple(k for k in range(64) if (U >> k) & 1) for U in res]
            assert got == oracle_lib.supports_to_lists(sup), (trial, t)
            assert ctr == rctr, (trial, t)
            checked += ctr["overflow"]
    assert checked > 0  # the int32 rule is exercised


@pytest.mark.parametrize("seed", range(4))
def test_budgeted_levels_match_the_python_reference(oracle_lib, seed):
    """Small frontier budgets make the C oracle compact (deduplicate) a
    level's children before the level ends and stop storing them once the
    budget is exceeded; results and every counter still equal the pure-Python
    restatement, which never does either."""
    from oracle import reference

    net = synth.tiny(seed)
    for t in list(net.targets) + [-1]:
        for budget in (3, 7, 20, 60):
            sup, ctr = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(10, 2, 0, budget))
            res, rctr = reference.enumerate_reference(net, t, 10, 2, max_frontier=budget)
            got = [tuple(k for k in range(64) if (U >> k) & 1) for U in res]
            assert got == oracle_lib.supports_to_lists(sup), (seed, t, budget)
            assert ctr == rctr, (seed, t, budget)
