"""Element-wise parity at the benchmarked sizes.

tests/golden/fullsize.json holds the CPU oracle's answers (SHA-256 of the
sorted supports and every counter), written by tests/golden/make_fullsize.py
from the oracle alone.  Here the GPU path runs the same workloads through the
C-ABI and must give the same digest and counters:

* the core-shaped network, all 8 targets, max_len 30, 4 secondary steps,
  frontier budget 2^26 -- the benchmark's headline configuration;
* the genome-shaped network, its first 32 targets, max_len 40, at the largest
  budget the oracle's host holds (recorded in the file);
* all 4096 members of the batched workload in one persistent launch;
* first-K = 1000 on genome targets: where both the oracle (under its host's
  budget) and the GPU (under the 2^22 budget of the first-K workload) certify
  their answers, the two are the same K supports.
"""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_1804_02867_gb300 import synth

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "fullsize.json")


def _digest(sup):
    return hashlib.sha256(np.ascontiguousarray(sup, dtype=np.uint64).tobytes()).hexdigest()


@pytest.fixture(scope="module")
def golden():
    if not os.path.exists(GOLDEN):
        pytest.skip("tests/golden/fullsize.json not written")
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def efm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_02867_gb300 import build, efmgraph

    build.build()
    efmgraph.load_library()
    return efmgraph


def _check_rows(efm, nw, rows):
    by = {}
    for r in rows:
        by.setdefault((r["max_len"], r["max_secondary"], r["max_frontier"]), []).append(r)
    for (L, S, B), group in by.items():
        got = efm.enumerate_targets(nw, [r["target"] for r in group], L, S, 0, B)
        for r, (sup, ctr) in zip(group, got):
            assert len(sup) == r["n"] and _digest(sup) == r["sha256"], (r["target"], len(sup), r["n"])
            assert ctr == r["counters"], (r["target"], ctr, r["counters"])


def test_core_headline_configuration(golden, efm):
    if "core" not in golden:
        pytest.skip("no core records")
    net = synth.core()
    assert sorted(r["target"] for r in golden["core"]) == sorted(net.targets)
    with efm.Network(net) as nw:
        _check_rows(efm, nw, golden["core"])


def test_genome_targets(golden, efm):
    if "genome" not in golden:
        pytest.skip("no genome records")
    net = synth.genome()
    with efm.Network(net) as nw:
        _check_rows(efm, nw, golden["genome"])


def test_all_batched_members(golden, efm):
    if "batched" not in golden:
        pytest.skip("no batched records")
    rows = sorted(golden["batched"], key=lambda r: r["member"])
    assert [r["member"] for r in rows] == list(range(4096))
    nets = [synth.batched_member(r["member"]) for r in rows]
    handles = [efm.Network(n) for n in nets]
    try:
        # max_len 30 is capped at each member's column count, as in the records
        job, _ = efm.efm_find_pathways_batch([h.handle for h in handles], [r["target"] for r in rows], 30, 4, 0,
                                             rows[0]["max_frontier"])
        try:
            for i, r in enumerate(rows):
                sup, ctr, _ = efm.efm_fetch_results(job, i)
                assert len(sup) == r["n"] and _digest(sup) == r["sha256"], r["member"]
                assert ctr == r["counters"], (r["member"], ctr, r["counters"])
        finally:
            efm.efm_free_job(job)
    finally:
        for h in handles:
            h.close()


def test_first_k_on_genome_targets(golden, efm):
    if "firstk" not in golden:
        pytest.skip("no first-K records")
    rows = [r for r in golden["firstk"] if r.get("certified")]
    assert len(rows) >= 8, "fewer than 8 certified oracle records"
    net = synth.genome()
    compared = 0
    with efm.Network(net) as nw:
        for r in rows:
            (sup, ctr), = efm.enumerate_targets(nw, [r["target"]], r["max_len"], r["max_secondary"], 0, 1 << 22,
                                                first_k=r["k"])
            if ctr["status"] & efm.EFM_TRUNCATED:
                continue
            compared += 1
            assert len(sup) == r["n"] and _digest(sup) == r["sha256"], r["target"]
    # the GPU's budget is 4x the oracle's: it certifies every target the oracle does
    assert compared == len(rows)
