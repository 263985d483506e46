"""Monte-Carlo mode on the GPU against the oracle's walks.

The walks are a pure function of (network, target, limits, seed, walk
count): the same counter-based generator picks the same seed column and
branches on both sides, so the sampled result set and every counter must be
identical.  Sampled results also lie inside the exhaustive result set.
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


def same(oracle_lib, efm, nw, net, t, L, S, seed, n):
    sup, ctr = efm.sample_target(nw, t, L, S, seed, n)
    osup, octr = oracle_lib.sample_pathways(net, t, oracle_lib.Limits(L, S), seed, n)
    assert np.array_equal(sup, osup), (net.name, t, seed, n)
    assert ctr == octr, (net.name, t, ctr, octr)
    return sup, ctr


@pytest.mark.parametrize("seed", range(8))
def test_tiny_walks(oracle_lib, efm, seed):
    net = synth.tiny(seed)
    with efm.Network(net) as nw:
        for t in list(net.targets) + [-1]:
            for n in (0, 1, 37, 5000):
                same(oracle_lib, efm, nw, net, t, 9, 1 + seed % 3, 1000 + seed, n)


def test_core_walks(oracle_lib, efm):
    net = synth.core()
    with efm.Network(net) as nw:
        for t in net.targets:
            same(oracle_lib, efm, nw, net, int(t), 30, 4, 17, 100000)
        sup, _ = same(oracle_lib, efm, nw, net, 63, 16, 4, 5, 300000)
        (full, _), = efm.enumerate_targets(nw, [63], 16, 4)
    assert set(map(bytes, sup)) <= set(map(bytes, full)) and len(sup) > 0


def test_genome_walks(oracle_lib, efm):
    net = synth.genome()
    with efm.Network(net) as nw:
        for t in (705, 924, -1):
            same(oracle_lib, efm, nw, net, t, 40, 4, 99, 1500)


def test_batched_member_walks(oracle_lib, efm):
    for i in range(12):
        net = synth.batched_member(i)
        with efm.Network(net) as nw:
            same(oracle_lib, efm, nw, net, int(net.targets[0]), min(30, nw.n_columns), 4, 7, 4000)


def test_walk_argument_rules(efm):
    net = synth.tiny(0)
    with efm.Network(net) as nw:
        with pytest.raises(efm.EfmError):
            efm.efm_sample_pathways(nw.handle, -1, 9, 64, 1, 10)     # max_secondary > 63
        with pytest.raises(efm.EfmError):
            efm.efm_sample_pathways(nw.handle, net.n_met, 9, 1, 1, 10)
        with pytest.raises(efm.EfmError):
            efm.efm_sample_pathways(nw.handle, -1, 9, 1, 1, -1)
