"""Traversal from a seed set R_in (Prop. 1) on the GPU against the oracle:
supports bit-identical and every counter equal."""
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


def same(oracle_lib, efm, nw, net, R, L, S):
    sup, ctr = efm.enumerate_from(nw, R, L, S)
    osup, octr = oracle_lib.enumerate_from(net, R, oracle_lib.Limits(L, S, 0, 0))
    assert np.array_equal(sup, osup), (net.name, R)
    assert ctr == octr, (net.name, R, ctr, octr)


def _sets(rng, twin, N, sizes, count):
    out = []
    while len(out) < count:
        size = int(rng.choice(sizes))
        R = sorted(int(x) for x in rng.choice(N, size=min(size, N), replace=False))
        if any(twin[a] in R for a in R if twin[a] >= 0):
            continue
        out.append(R)
    return out


@pytest.mark.parametrize("seed", range(6))
def test_tiny_seed_sets(oracle_lib, efm, seed):
    from oracle import bruteforce

    net = synth.tiny(seed)
    _, twin, _ = bruteforce.split(net)
    N = len(twin)
    rng = np.random.default_rng(seed)
    with efm.Network(net) as nw:
        for j in range(N):
            same(oracle_lib, efm, nw, net, [j], 9, 1)
        for R in _sets(rng, twin, N, (2, 3), 12):
            same(oracle_lib, efm, nw, net, R, 9, 2)


def test_core_seed_sets(oracle_lib, efm):
    from oracle import bruteforce

    net = synth.core()
    _, twin, _ = bruteforce.split(net)
    rng = np.random.default_rng(1)
    with efm.Network(net) as nw:
        (res, _), = efm.enumerate_targets(nw, [63], 16, 4)
        cols = __import__("oracle").supports_to_lists(res)
        # subsets of known results, and random sets
        sets = [list(c[:2]) for c in cols[:6]] + [list(c[::3]) for c in cols[6:10]]
        sets += _sets(rng, twin, len(twin), (1, 2), 6)
        for R in sets:
            same(oracle_lib, efm, nw, net, R, 14, 4)


def test_seed_set_rules(efm):
    from oracle import bruteforce

    net = synth.tiny(0)
    _, twin, _ = bruteforce.split(net)
    a = next(k for k in range(len(twin)) if twin[k] >= 0)
    with efm.Network(net) as nw:
        for bad in ([a, int(twin[a])], [1, 1], [], [len(twin)], list(range(10))):
            with pytest.raises(efm.EfmError):
                efm.efm_find_pathways_from(nw.handle, bad, 9, 1)


def test_seed_set_first_k_and_fluxes(oracle_lib, efm):
    """Features combined: a first-K search from a seed set returns the K
    smallest of the seed set's results, and their flux vectors are exact."""
    from oracle import flux

    net = synth.core()
    with efm.Network(net) as nw:
        (res, _), = efm.enumerate_targets(nw, [63], 16, 4)
        R = list(__import__("oracle").supports_to_lists(res)[3][:2])
        full, _ = oracle_lib.enumerate_from(net, R, oracle_lib.Limits(16, 4, 0, 0))
        for k in (1, 5, len(full)):
            sup, _ = efm.enumerate_from(nw, R, 16, 4, first_k=k)
            assert np.array_equal(sup, full[:k]), (R, k)
        fl, st = efm.efm_flux_vectors(nw.handle, full)
        for i, v in enumerate(flux.flux_vectors(net, full)):
            assert st[i] == 1 and list(fl[i, :len(v)]) == v
