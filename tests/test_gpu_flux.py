"""Exact flux vectors on the GPU against the oracle (sympy null space).

Each result's flux vector is the primitive positive kernel vector of
S_int[:, U]; the GPU computes it by integer elimination on the device and
must agree entry for entry.
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


def check(efm, nw, net, sup):
    from oracle import flux

    got, st = efm.efm_flux_vectors(nw.handle, sup)
    want = flux.flux_vectors(net, sup)
    for i, w in enumerate(want):
        assert w is not None
        assert st[i] == 1, (i, st[i])
        assert list(got[i, :len(w)]) == w and not got[i, len(w):].any(), (i, got[i, :len(w)], w)


def test_hand_worked(efm):
    with open(os.path.join(HERE, "golden", "handworked.json")) as f:
        cases = json.load(f)["cases"]
    for case in cases:
        if "flux" not in case:
            continue
        net = synth.Network.from_dense(case["S"], case["reversible"], case["external"])
        variant = efm.EFM_SUBTRACTIVE if case.get("subtractive") else efm.EFM_ADDITIVE
        with efm.Network(net) as nw:
            (sup, _), = efm.enumerate_targets(nw, [case["target"]], case["max_len"], case["max_secondary"],
                                              variant=variant)
            got, st = efm.efm_flux_vectors(nw.handle, sup)
        for i, w in enumerate(case["flux"]):
            assert st[i] == 1 and list(got[i, :len(w)]) == w, case["name"]


@pytest.mark.parametrize("seed", range(8))
def test_tiny_results(efm, seed):
    net = synth.tiny(seed)
    with efm.Network(net) as nw:
        for (sup, _) in efm.enumerate_targets(nw, list(net.targets) + [-1], 9, 2):
            if len(sup):
                check(efm, nw, net, sup)


def test_core_and_genome_results(efm):
    net = synth.core()
    with efm.Network(net) as nw:
        for sup, _ in efm.enumerate_targets(nw, [63, 65, 42, 5], 16, 4):
            check(efm, nw, net, sup)
    net = synth.genome()
    with efm.Network(net) as nw:
        for t, k in [(924, 200), (883, 80)]:
            (sup, _), = efm.enumerate_targets(nw, [t], 40, 4, 0, 1 << 21, first_k=k)
            check(efm, nw, net, sup)


def test_non_rays_are_flagged(efm):
    """A union of two results has nullity 2; a single column that is not
    balanced has nullity 0; no columns at all: all are status -1."""
    net = synth.tiny(3)
    with efm.Network(net) as nw:
        (sup, _), = efm.enumerate_targets(nw, [-1], 9, 1)
        from oracle import bruteforce

        S_int, _, _ = bruteforce.split(net)
        lists = __import__("oracle").supports_to_lists(sup)
        a, b = next((x, y) for i, x in enumerate(lists) for y in lists[i + 1:] if not set(x) & set(y))
        union = np.zeros((1, sup.shape[1]), dtype=np.uint64)
        for c in set(a) | set(b):
            union[0, c // 64] |= np.uint64(1 << (c % 64))
        unbalanced = next(k for k in range(S_int.shape[1]) if S_int[:, k].any())
        single = np.zeros((1, sup.shape[1]), dtype=np.uint64)
        single[0, unbalanced // 64] |= np.uint64(1 << (unbalanced % 64))
        empty = np.zeros((1, sup.shape[1]), dtype=np.uint64)
        got, st = efm.efm_flux_vectors(nw.handle, np.vstack([union, single, empty, sup[:1]]))
    assert list(st) == [-1, -1, -1, 1]
    assert not got[:3].any()
