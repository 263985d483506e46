"""Write tests/golden/fullsize.json: the oracle's answers on the benchmarked
workloads, as a SHA-256 of the sorted result supports plus every counter.

Calls only the CPU oracle (oracle/) and the seeded generator (synth); the
GPU tests compare their own supports and counters with these records.

    python tests/golden/make_fullsize.py [core] [genome] [batched] [firstk]

core     the core-shaped network, 8 targets, max_len 30, max_secondary 4,
         frontier budget 2^26 (the benchmark's headline configuration);
         one target at a time (a level holds up to ~40 GB on the host)
genome   the genome-shaped network, its first 32 targets, max_len 40,
         max_secondary 4, frontier budget GENOME_BUDGET (the largest the
         host's memory holds for the oracle; the benchmark itself runs 2^22)
batched  all 4096 batched members, one target each, max_len min(30, N),
         max_secondary 4, frontier budget 2^12
firstk   first-K = 1000 on FIRSTK_TARGETS of the genome network, max_len 40,
         max_secondary 4, by the oracle's deepening under GENOME_BUDGET (the
         complete levels of a genome traversal do not fit the host); a record
         is the definition's answer only where "certified" is true
Records already present are kept unless their section is named again
(first-K records of targets already computed at the same budget are kept).
"""
from __future__ import annotations

import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "fullsize.json")
CORE_BUDGET = 2**26
GENOME_BUDGET = 2**20
GENOME_TARGETS = 32
BATCH_BUDGET = 2**12
FIRSTK = 1000
FIRSTK_TARGETS = tuple(range(80))  # positions in the genome network's target list


def digest(supports) -> str:
    import numpy as np

    return hashlib.sha256(np.ascontiguousarray(supports, dtype=np.uint64).tobytes()).hexdigest()


def _core_one(t):
    import oracle
    from paper_1804_02867_gb300 import synth

    net = synth.core()
    t0 = time.time()
    sup, ctr = oracle.enumerate_pathways(net, t, oracle.Limits(30, 4, 0, CORE_BUDGET))
    return {"target": int(t), "max_len": 30, "max_secondary": 4, "max_frontier": CORE_BUDGET, "n": int(len(sup)),
            "sha256": digest(sup), "counters": ctr, "oracle_s": round(time.time() - t0, 1)}


def _genome_one(t):
    import oracle
    from paper_1804_02867_gb300 import synth

    net = synth.genome()
    t0 = time.time()
    sup, ctr = oracle.enumerate_pathways(net, t, oracle.Limits(40, 4, 0, GENOME_BUDGET))
    return {"target": int(t), "max_len": 40, "max_secondary": 4, "max_frontier": GENOME_BUDGET, "n": int(len(sup)),
            "sha256": digest(sup), "counters": ctr, "oracle_s": round(time.time() - t0, 1)}


def _batched_chunk(rng):
    import oracle
    from paper_1804_02867_gb300 import synth

    out = []
    for i in rng:
        net = synth.batched_member(i)
        L = min(30, net.split_columns())
        sup, ctr = oracle.enumerate_pathways(net, net.targets[0], oracle.Limits(L, 4, 0, BATCH_BUDGET))
        out.append({"member": int(i), "target": int(net.targets[0]), "max_len": L, "max_secondary": 4,
                    "max_frontier": BATCH_BUDGET, "n": int(len(sup)), "sha256": digest(sup), "counters": ctr})
    return out


def _firstk_one(pos):
    import oracle
    from paper_1804_02867_gb300 import synth

    net = synth.genome()
    t = int(net.targets[pos])
    t0 = time.time()
    sup, P, ok = oracle.first_k_within(net, t, FIRSTK, 40, 4, GENOME_BUDGET)
    return {"target": t, "k": FIRSTK, "max_len": 40, "max_secondary": 4, "max_frontier": GENOME_BUDGET,
            "certified": bool(ok), "n": int(len(sup)), "depth_used": int(P), "sha256": digest(sup),
            "oracle_s": round(time.time() - t0, 1)}


def main(argv):
    import oracle
    from paper_1804_02867_gb300 import synth

    oracle.build()
    sections = [a for a in argv if a in ("core", "genome", "batched", "firstk")] or ["core", "genome", "batched",
                                                                                    "firstk"]
    rec = json.load(open(OUT)) if os.path.exists(OUT) else {}
    rec["_about"] = ("Oracle answers on the benchmarked workloads (SHA-256 of the sorted supports, uint64 rows, "
                     "little-endian; every counter), written by tests/golden/make_fullsize.py, which calls only "
                     "the CPU oracle and the seeded generator.")
    ctx = mp.get_context("spawn")
    threads = max(1, os.cpu_count() or 1)
    if "core" in sections:
        net = synth.core()
        rows = []
        for t in net.targets:  # sequential: one level of one target takes tens of GB
            rows.append(_core_one(t))
            print("core", rows[-1]["target"], rows[-1]["n"], rows[-1]["oracle_s"], "s", flush=True)
        rec["core"] = rows
        json.dump(rec, open(OUT, "w"), indent=1)
    if "genome" in sections:
        net = synth.genome()
        with ctx.Pool(min(threads, 2)) as pool:  # ~14 GB of host memory per traversal
            rec["genome"] = pool.map(_genome_one, list(net.targets[:GENOME_TARGETS]))
        json.dump(rec, open(OUT, "w"), indent=1)
        print("genome done", flush=True)
    if "batched" in sections:
        chunks = [range(i, min(4096, i + 128)) for i in range(0, 4096, 128)]
        with ctx.Pool(threads) as pool:
            rec["batched"] = [r for part in pool.map(_batched_chunk, chunks) for r in part]
        json.dump(rec, open(OUT, "w"), indent=1)
        print("batched done", flush=True)
    if "firstk" in sections:
        net = synth.genome()
        have = {r["target"]: r for r in rec.get("firstk", []) if r.get("max_frontier") == GENOME_BUDGET}
        todo = [p for p in FIRSTK_TARGETS if int(net.targets[p]) not in have]
        with ctx.Pool(min(threads, 2)) as pool:  # ~14 GB of host memory per traversal
            new = pool.map(_firstk_one, todo)
        order = {int(net.targets[p]): i for i, p in enumerate(FIRSTK_TARGETS)}
        rec["firstk"] = sorted(list(have.values()) + new, key=lambda r: order.get(r["target"], len(order)))
        json.dump(rec, open(OUT, "w"), indent=1)
        print("firstk done", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
