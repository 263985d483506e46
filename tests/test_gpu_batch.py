"""Batched traversal (one persistent, graph-captured launch over many uneven
networks): every job's supports and counters equal the CPU oracle's and the
single-job path's."""
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


def _batch(efm, nets, L, S, budget, max_results=0):
    handles = [efm.Network(n) for n in nets]
    try:
        targets = [n.targets[0] for n in nets]
        job, _ = efm.efm_find_pathways_batch([h.handle for h in handles], targets, L, S, max_results, budget)
        out = []
        for i in range(len(nets)):
            sup, ctr, _ = efm.efm_fetch_results(job, i)
            out.append((sup, ctr))
        efm.efm_free_job(job)
        return out
    finally:
        for h in handles:
            h.close()


@pytest.mark.parametrize("budget", [2**10, 2**12])
def test_batch_matches_oracle(oracle_lib, efm, budget):
    nets = [synth.batched_member(i) for i in range(96)]
    got = _batch(efm, nets, 30, 4, budget)
    for net, (sup, ctr) in zip(nets, got):
        L = min(30, net.split_columns())
        osup, octr = oracle_lib.enumerate_pathways(net, net.targets[0], oracle_lib.Limits(L, 4, 0, budget))
        assert np.array_equal(sup, osup), net.name
        assert ctr == octr, (net.name, ctr, octr)


def test_batch_matches_single_job_path(efm):
    nets = [synth.batched_member(1000 + i) for i in range(40)] + [synth.tiny(i) for i in range(8)]
    got = _batch(efm, nets, 12, 2, 2**11)
    for net, (sup, ctr) in zip(nets, got):
        L = min(12, net.split_columns())
        with efm.Network(net) as nw:
            (ssup, sctr), = efm.enumerate_targets(nw, [net.targets[0]], L, 2, 0, 2**11)
        assert np.array_equal(sup, ssup) and ctr == sctr, net.name


def test_batch_autotuner_reports_choice(efm):
    efm.efm_batch_set_tuning(None)
    nets = [synth.batched_member(2000 + i) for i in range(80)]
    _batch(efm, nets, 20, 2, 2**9)
    t = efm.efm_batch_tuning()
    assert t is not None and t["ctas_per_sm"] >= 1 and t["largest_first"] in (0, 1) and t["pinned"] == 0
    assert t["warps_per_job"] in (4, 8) and 1 <= t["tile"] <= 32 and t["queue_chunk"] >= 1
    # the search keeps the untuned configuration unless something beat it
    assert 0 < t["sample_tuned_ms"] <= t["sample_default_ms"]


@pytest.mark.parametrize("cfg", [dict(ctas_per_sm=0, largest_first=0, warps_per_job=8, tile=32, queue_chunk=1),
                                 dict(ctas_per_sm=1, largest_first=1, warps_per_job=4, tile=8, queue_chunk=4),
                                 dict(ctas_per_sm=0, largest_first=1, warps_per_job=4, tile=1, queue_chunk=3),
                                 dict(ctas_per_sm=2, largest_first=0, warps_per_job=8, tile=16, queue_chunk=64)])
def test_every_launch_configuration_gives_the_oracle_answers(oracle_lib, efm, cfg):
    """The autotuner's search space (CTAs per SM, queue order, warps per job,
    tile, queue chunk) changes only the schedule: pinned to any point of it,
    the batch gives the oracle's supports and counters."""
    nets = [synth.batched_member(4000 + i) for i in range(70)] + [synth.tiny(i) for i in range(4)]
    efm.efm_batch_set_tuning(cfg)
    try:
        got = _batch(efm, nets, 30, 4, 2**10)
        t = efm.efm_batch_tuning()
        assert t["pinned"] == 1 and t["warps_per_job"] == cfg["warps_per_job"] and t["tile"] == cfg["tile"]
    finally:
        efm.efm_batch_set_tuning(None)
    for net, (sup, ctr) in zip(nets, got):
        L = min(30, net.split_columns())
        osup, octr = oracle_lib.enumerate_pathways(net, net.targets[0], oracle_lib.Limits(L, 4, 0, 2**10))
        assert np.array_equal(sup, osup), net.name
        assert ctr == octr, (net.name, ctr, octr)


def test_tuning_pin_is_validated(efm):
    for bad in (dict(warps_per_job=6), dict(tile=0), dict(tile=33), dict(queue_chunk=0), dict(largest_first=2),
                dict(ctas_per_sm=-1), dict(ctas_per_sm=10_000)):
        cfg = dict(ctas_per_sm=1, largest_first=0, warps_per_job=8, tile=32, queue_chunk=1, **{})
        cfg.update(bad)
        with pytest.raises(efm.EfmError):
            efm.efm_batch_set_tuning(cfg)


def wide_member(i):
    """A batched-call member with 129-256 internal metabolites (8 balance
    entries per lane, the widest row the batched kernel takes)."""
    rng = np.random.default_rng(6_000_000 + i)
    n_int = int(rng.integers(129, 257))
    n_rxn = int(rng.integers(2 * n_int, 3 * n_int))
    return synth.generate(n_int=n_int, n_targets=3, n_hubs=4, n_substrates=2, n_rxn=n_rxn, n_rev=n_rxn // 5,
                          size_range=(2, 6), coef_probs=synth.CORE_COEFS, gamma=2.2, hub_degree=(30, 80),
                          seed=6_000_000 + i, name=f"wide-{i}")


@pytest.mark.parametrize("budget", [2**10, 2**12])
def test_batch_mixed_row_widths(oracle_lib, efm, budget):
    """One launch over members of every row width it supports (1, 2, 4 and 8
    entries per lane, supports of 1 to 14 words), interleaved."""
    nets = []
    for i in range(24):
        nets += [wide_member(i), synth.batched_member(3000 + i)] + ([synth.tiny(100 + i)] if i % 3 == 0 else [])
    got = _batch(efm, nets, 30, 4, budget)
    widths = set()
    for net, (sup, ctr) in zip(nets, got):
        L = min(30, net.split_columns())
        osup, octr = oracle_lib.enumerate_pathways(net, net.targets[0], oracle_lib.Limits(L, 4, 0, budget))
        assert np.array_equal(sup, osup), net.name
        assert ctr == octr, (net.name, ctr, octr)
        need = max(1, -(-int((net.external == 0).sum()) // 32))
        widths.add(min(e for e in (1, 2, 4, 8) if e >= need))
    assert widths == {1, 2, 4, 8}


def test_batch_rejects_wider_rows(efm):
    """Members with more than 256 internal metabolites are refused
    (EFM_EUNSUPPORTED) before anything is launched."""
    wide = synth.generate(n_int=300, n_targets=3, n_hubs=4, n_substrates=2, n_rxn=700, n_rev=140,
                          size_range=(2, 6), coef_probs=synth.CORE_COEFS, gamma=2.2, hub_degree=(30, 80),
                          seed=6_100_000, name="too-wide")
    with pytest.raises(efm.EfmError) as e:
        _batch(efm, [synth.tiny(0), wide], 20, 2, 2**10)
    assert e.value.code == -6
