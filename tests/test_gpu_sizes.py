"""Parity at every balance-row width and at the library's size limits.

The expansion kernel is compiled once per row width (Mpad = 32 EPL int32
entries; EPL = 1, 2, 4, 8, 16, 28, 32).  The tiny, core, batched and genome
networks cover EPL 1, 2, 4 and 28; the networks here cover the rest:

* 200 and 400 internal metabolites (EPL 8 and 16), genome-like degree laws,
  truncated at two frontier budgets;
* the maximal network: 1024 internal metabolites (EPL 32), 4096 split
  columns (64-word supports), a 64-column pathway at max_len 64 with
  coefficients up to the loader's limit, a reversible chain step (twin
  rule), a cycle that needs secondary steps and yields a non-elementary
  balanced support, and a random filler whose target overflows int32 on
  some branches.

Supports and every counter must equal the oracle's, and so must first-K,
seed-set traversal, Monte-Carlo walks and flux vectors at the maximal size.
"""
import numpy as np
import pytest

from paper_1804_02867_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def efm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_02867_gb300 import build, efmgraph

    build.build()
    efmgraph.load_library()
    return efmgraph


def mid_network(n_int):
    """Genome-like network with n_int internal metabolites."""
    shapes = {
        200: dict(n_targets=6, n_hubs=6, n_substrates=2, n_rxn=500, n_rev=100, hub_degree=(40, 100)),
        400: dict(n_targets=6, n_hubs=10, n_substrates=3, n_rxn=1000, n_rev=250, hub_degree=(80, 200)),
    }
    return synth.generate(n_int=n_int, size_range=(2, 6), coef_probs=synth.CORE_COEFS, gamma=2.2,
                          seed=5_000_000 + n_int, name=f"mid-{n_int}", **shapes[n_int])


@pytest.fixture(scope="module")
def maximal():
    return synth.maximal()


@pytest.mark.parametrize("n_int", [200, 400])
def test_row_widths_8_and_16(oracle_lib, efm, n_int):
    net = mid_network(n_int)
    targets = net.targets[:4]
    with efm.Network(net) as nw:
        assert nw.n_internal == n_int
        for budget in (1 << 12, 1 << 16):
            got = efm.enumerate_targets(nw, targets, 40, 4, 0, budget)
            for t, (sup, ctr) in zip(targets, got):
                osup, octr = oracle_lib.enumerate_pathways(net, t, oracle_lib.Limits(40, 4, 0, budget))
                assert np.array_equal(sup, osup), (n_int, t, budget)
                assert ctr == octr, (n_int, t, budget, ctr, octr)


def test_maximal_network_shape(efm, maximal):
    with efm.Network(maximal) as nw:
        assert (nw.n_columns, nw.words, nw.n_internal) == (4096, 64, 1024)
    assert int(np.abs(maximal.coef).max()) == synth.MAX_COEF


def test_maximal_chain_target(oracle_lib, efm, maximal):
    """Target T: six pathways of 12, 22, 32, 42, 52 and 64 columns, one
    non-elementary balanced support; the last pathway sits at max_len 64."""
    T = maximal.targets[0]
    B = 1 << 12  # frontier budget: the chain's levels hold at most 3 states
    lim = oracle_lib.Limits(64, 4, 0, B)
    with efm.Network(maximal) as nw:
        (sup, ctr), = efm.enumerate_targets(nw, [T], 64, 4, 0, B)
        osup, octr = oracle_lib.enumerate_pathways(maximal, T, lim)
        assert np.array_equal(sup, osup) and ctr == octr, (ctr, octr)
        assert [len(c) for c in oracle_lib.supports_to_lists(sup)] == [12, 22, 32, 42, 52, 64]
        assert ctr["balanced"] - ctr["results"] == 1 and ctr["status"] == 0
        # one column less: the 64-column pathway is out of reach
        (sup63, _), = efm.enumerate_targets(nw, [T], 63, 4, 0, B)
        assert np.array_equal(sup63, osup[:5])
        # first-K in the output order
        (fk, _), = efm.enumerate_targets(nw, [T], 64, 4, 0, B, first_k=3)
        want, _ = oracle_lib.first_k(maximal, T, 3, 64, 4)
        assert np.array_equal(fk, want) and np.array_equal(fk, osup[:3])
        # seed set R_in = {r_0, r_1}
        sup_from, ctr_from = efm.enumerate_from(nw, [0, 1], 64, 4, 0, B)
        osup_from, octr_from = oracle_lib.enumerate_from(maximal, [0, 1], lim)
        assert np.array_equal(sup_from, osup_from) and ctr_from == octr_from


def test_maximal_flux_vectors(oracle_lib, efm, maximal):
    """Flux vectors at 64 columns with coefficients up to the loader's limit."""
    from oracle import bruteforce, flux

    T = maximal.targets[0]
    S_int, _, _ = bruteforce.split(maximal)
    osup, _ = oracle_lib.enumerate_pathways(maximal, T, oracle_lib.Limits(64, 4, 0, 0))
    with efm.Network(maximal) as nw:
        fl, st = efm.efm_flux_vectors(nw.handle, osup)
    for i, cols in enumerate(oracle_lib.supports_to_lists(osup)):
        rows = np.nonzero(np.any(S_int[:, list(cols)] != 0, axis=1))[0]
        want = flux.flux_vector(S_int[rows], cols)
        assert st[i] == 1 and list(fl[i, :len(cols)]) == want, (i, len(cols))
        assert not fl[i, len(cols):].any()
    assert max(int(x) for x in fl[-1]) == 6 * synth.MAX_COEF


def test_maximal_walks(oracle_lib, efm, maximal):
    T = maximal.targets[0]
    with efm.Network(maximal) as nw:
        sup, ctr = efm.sample_target(nw, T, 64, 4, 11, 4096)
    osup, octr = oracle_lib.sample_pathways(maximal, T, oracle_lib.Limits(64, 4), 11, 4096)
    assert np.array_equal(sup, osup) and ctr == octr, (ctr, octr)


@pytest.mark.parametrize("budget", [1 << 10, 1 << 14])
def test_maximal_filler_target(oracle_lib, efm, maximal, budget):
    """The random filler at 1024-entry rows and 64-word supports, truncated
    at the budget; some branches leave int32 and are dropped."""
    t = maximal.targets[1]
    with efm.Network(maximal) as nw:
        (sup, ctr), = efm.enumerate_targets(nw, [t], 64, 2, 0, budget)
    osup, octr = oracle_lib.enumerate_pathways(maximal, t, oracle_lib.Limits(64, 2, 0, budget))
    assert np.array_equal(sup, osup) and ctr == octr, (ctr, octr)
    assert ctr["overflow"] > 0 and ctr["status"] & 1
