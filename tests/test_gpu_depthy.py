"""DEPTHy (flux-dependent reactions, Def. 11) on the GPU against the oracle's
depth-first enumeration: tags bit-identical, r equal."""
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


def same(efm, net, depths):
    from oracle import depthy

    with efm.Network(net) as nw:
        for L in depths:
            o, i, r, _ = efm.efm_dependent_reactions(nw, L)
            wo, wi = depthy.dependent_reactions(net, L)
            assert r == depthy.r_max(net)
            assert np.array_equal(o, wo) and np.array_equal(i, wi), (net.name, L)


@pytest.mark.parametrize("seed", range(6))
def test_tiny_and_type1(efm, seed):
    same(efm, synth.tiny(seed), (1, 2, 3, 4, 5))
    same(efm, synth.type1(seed), (1, 2, 3, 4))


def test_core(efm):
    same(efm, synth.core(), (1, 2, 3))


def test_genome_depth_one(efm):
    same(efm, synth.genome(), (1,))


def test_depth_rules(efm):
    net = synth.genome()
    with efm.Network(net) as nw:
        with pytest.raises(efm.EfmError):
            efm.efm_dependent_reactions(nw, 0)
        with pytest.raises(efm.EfmError):   # 804^5 walks per metabolite: over 2^40
            efm.efm_dependent_reactions(nw, 5)
