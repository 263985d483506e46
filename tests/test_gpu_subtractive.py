"""The subtractive variant (Eq. 5 with the zero-flux discard of Prop. 3) on
the GPU against the oracle, through the C-ABI: supports bit-identical and
every counter equal, zero_flux included."""
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


def _same(oracle_lib, efm, nw, net, targets, L, S, max_results=0, max_frontier=0):
    got = efm.enumerate_targets(nw, targets, L, S, max_results, max_frontier, variant=efm.EFM_SUBTRACTIVE)
    for t, (sup, ctr) in zip(targets, got):
        osup, octr = oracle_lib.enumerate_pathways(
            net, t, oracle_lib.Limits(L, S, max_results, max_frontier, subtractive=True))
        assert np.array_equal(sup, osup), (net.name, t, L, S)
        assert ctr == octr, (net.name, t, L, S, ctr, octr)
    return got


def test_hand_worked(oracle_lib, efm):
    with open(os.path.join(HERE, "golden", "handworked.json")) as f:
        cases = [c for c in json.load(f)["cases"] if c.get("subtractive")]
    assert cases
    for case in cases:
        net = synth.Network.from_dense(case["S"], case["reversible"], case["external"], name=case["name"])
        with efm.Network(net) as nw:
            (sup, ctr), = efm.enumerate_targets(nw, [case["target"]], case["max_len"], case["max_secondary"],
                                                variant=efm.EFM_SUBTRACTIVE)
        assert [tuple(c) for c in oracle_lib.supports_to_lists(sup)] == [tuple(x) for x in case["expected"]]
        for k, v in case["counters"].items():
            assert ctr[k] == v, (case["name"], k, ctr)


@pytest.mark.parametrize("seed", range(12))
def test_tiny_networks(oracle_lib, efm, seed):
    net = synth.tiny(seed)
    with efm.Network(net) as nw:
        for L, S in ((8, 1), (9, 2), (12, 3)):
            _same(oracle_lib, efm, nw, net, list(net.targets) + [-1], L, S)


def test_budget_and_cap(oracle_lib, efm):
    net = synth.tiny(3)
    with efm.Network(net) as nw:
        _same(oracle_lib, efm, nw, net, list(net.targets) + [-1], 9, 2, max_frontier=20)
        _same(oracle_lib, efm, nw, net, list(net.targets) + [-1], 9, 2, max_results=2)


def test_core_network(oracle_lib, efm):
    """Core-shaped network (58 internal, 114 columns: rows of 172 entries) at
    short pathway lengths, every target; the variant discards children."""
    net = synth.core()
    with efm.Network(net) as nw:
        got = _same(oracle_lib, efm, nw, net, list(net.targets), 12, 2)
    assert sum(c["zero_flux"] for _, c in got) > 0


def test_batched_members(oracle_lib, efm):
    for i in (0, 3, 11):
        net = synth.batched_member(i)
        if net.n_met - int(np.asarray(net.external).sum()) + net.split_columns() > 1024:
            continue
        with efm.Network(net) as nw:
            _same(oracle_lib, efm, nw, net, [net.targets[0]], min(14, net.split_columns()), 2, max_frontier=1 << 14)


def test_seed_sets(oracle_lib, efm):
    net = synth.tiny(4)
    with efm.Network(net) as nw:
        for R in ([0], [2, 5], [1, 4, 9]):
            sup, ctr = efm.enumerate_from(nw, R, 9, 2, variant=efm.EFM_SUBTRACTIVE)
            osup, octr = oracle_lib.enumerate_from(net, R, oracle_lib.Limits(9, 2, 0, 0, subtractive=True))
            assert np.array_equal(sup, osup), R
            assert ctr == octr, (R, ctr, octr)


def test_rejected_arguments(efm):
    genome = synth.genome()  # 850 internal + 3125 columns: rows too wide
    with efm.Network(genome) as nw:
        with pytest.raises(efm.EfmError) as e:
            efm.enumerate_targets(nw, [genome.targets[0]], 10, 2, variant=efm.EFM_SUBTRACTIVE)
        assert e.value.code == -6
    net = synth.tiny(0)
    with efm.Network(net) as nw:
        with pytest.raises(efm.EfmError) as e:
            efm.enumerate_targets(nw, [-1], 8, 1, first_k=5, variant=efm.EFM_SUBTRACTIVE)
        assert e.value.code == -1
        with pytest.raises(efm.EfmError) as e:
            efm.enumerate_targets(nw, [-1], 8, 1, variant=7)
        assert e.value.code == -1
