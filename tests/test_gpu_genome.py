"""Genome-scale shape (1000 metabolites, 2500 reactions, 3125 split columns,
49-word supports, 850-entry balance rows): parity with the oracle on a fixed
subset of the 256 targets (external products and internal metabolites) at
budgets small enough for the oracle, and properties at a larger budget."""
import numpy as np
import pytest

from paper_1804_02867_gb300 import synth

pytestmark = pytest.mark.gpu
SUBSET = [0, 1, 2, 3, 60, 119, 140, 200, 255]


@pytest.fixture(scope="module")
def efm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_02867_gb300 import build, efmgraph

    build.build()
    efmgraph.load_library()
    return efmgraph


@pytest.fixture(scope="module")
def genome():
    return synth.genome()


@pytest.mark.parametrize("budget", [2**10, 2**13])
def test_genome_subset_matches_oracle(oracle_lib, efm, genome, budget):
    targets = [genome.targets[i] for i in SUBSET]
    with efm.Network(genome) as nw:
        assert nw.n_columns == 3125 and nw.words == 49 and nw.n_internal == 850
        got = efm.enumerate_targets(nw, targets, 40, 4, 0, budget)
    for t, (sup, ctr) in zip(targets, got):
        osup, octr = oracle_lib.enumerate_pathways(genome, t, oracle_lib.Limits(40, 4, 0, budget))
        assert np.array_equal(sup, osup), t
        assert ctr == octr, (t, ctr, octr)


def test_genome_larger_budget_properties(oracle_lib, efm, genome):
    from oracle import bruteforce

    S_int, twin, full = bruteforce.split(genome)
    targets = [genome.targets[i] for i in SUBSET[:4]]
    with efm.Network(genome) as nw:
        got = efm.enumerate_targets(nw, targets, 40, 4, 0, 2**17)
    rng = np.random.default_rng(1)
    for t, (sup, ctr) in zip(targets, got):
        lists = oracle_lib.supports_to_lists(sup)
        small, _ = oracle_lib.enumerate_pathways(genome, t, oracle_lib.Limits(40, 4, 0, 2**13))
        assert set(oracle_lib.supports_to_lists(small)) <= set(lists)
        seeds = bruteforce.seeds_of(genome, t)
        for i in (rng.choice(len(lists), size=min(10, len(lists)), replace=False) if lists else []):
            cols = list(lists[i])
            A = S_int[:, cols]
            A = A[np.any(A != 0, axis=1)]
            assert len(cols) - oracle_lib.rank(A) == 1 and seeds.intersection(cols)
