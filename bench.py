#!/usr/bin/env python3
"""Benchmark of the flux-balanced pathway traversal on one GB300.

Workload (the core-shaped network): 72 metabolites (58 internal), 95
reactions (19 reversible, 114 split columns, 128-bit supports), all pathways
to each of its 8 target externals, max_len 30, max_secondary 4, frontier
budget 2^26 states per level.  One step = efm_find_pathways over the 8
targets (seed, then per level: expand + dedup + prune, minimality test),
with the network already resident on the device.

Metric: materialised children (AND updates, before deduplication) per
second, whole job; balanced pathways per second alongside.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica on its own
GPU (the traversal of one target does not shard); rank 0 prints one JSON
line with the sum of work over the max of the ranks' times.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "partial-pathway expansions/sec and balanced pathways/sec at 1 GB300; first-K time vs plain"
UNIT = "expansions/s"
MAX_LEN, MAX_SEC = 30, 4
BUDGET = 2**26
CPU_SAMPLE_BUDGET = 2**20
REF_STEP_BUDGET = 2**17
L2_BYTES = 129 * 2**20


def workload_config(budget):
    return {
        "workload": "core-72x95 (58 internal, 114 split columns), 8 target externals",
        "max_len": MAX_LEN, "max_secondary": MAX_SEC, "max_frontier": budget,
        "support_bits": 128, "balance": "int32 x 58",
        "l2": "frontier arenas far exceed L2 (up to 2^26 states x 276 B); L2 also flushed between steps",
        "parallelism": "replicas",
    }


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--budget", type=int, default=BUDGET)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the batched, genome and first-K summaries of the default run")
    ap.add_argument("--workload", choices=["core", "batched", "genome", "firstk", "sample"], default="core",
                    help="core: the headline line; batched: 4096 uneven networks in one persistent launch; "
                         "genome: the genome-shaped network; firstk: first-K queries, learned vs plain order")
    ap.add_argument("--jobs", type=int, default=4096)
    ap.add_argument("--targets", type=str, default="",
                    help="comma-separated positions among the 8 targets (profiling a smaller case)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_over_ranks(times, work, device):
    """Replicas: the slowest rank's times (max) and all ranks' work (sum), over
    the initialised process group (NCCL with device "cuda", gloo with "cpu")."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x) for x in times], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([float(x) for x in work], device=device, dtype=torch.float64)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return [float(x) for x in t.tolist()], [int(x) for x in w.tolist()]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def profile_figure(name, key):
    """A figure from a committed ncu summary under profiles/, if that summary
    was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", name)
    src = os.path.join(ROOT, "paper_1804_02867_gb300", "csrc", "efm_kernels.cu")
    try:
        text = open(path).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    m_sha = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    m_val = re.search(re.escape(key) + r":\s*([0-9.eE+]+)", text)
    if not m_sha or not m_val or m_sha.group(1) != sha:
        return None
    return float(m_val.group(1))


def profile_traffic(alg_bytes_per_launch):
    """Per-launch DRAM traffic of the core network's level pass (generate,
    settle and dedup kernels of one expansion launch): the DRAM-to-algorithmic
    ratio ncu measured on a smaller case of the same kernels (traffic grows
    with the states read and written), applied to this run's algorithmic
    bytes per launch; None without a summary for the current source."""
    ratio = profile_figure("level_pass_core.md", "dram_to_algorithmic_ratio")
    return ratio * alg_bytes_per_launch if ratio else None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(net, budget, threads):
    """Run the CPU oracle over the 8 targets on `threads` host threads; with
    more threads than targets every target is run ceil(threads / 8) times,
    so that all of them have work (each run is one independent job)."""
    import oracle

    oracle.build()
    lim = oracle.Limits(MAX_LEN, MAX_SEC, 0, budget)
    reps = max(1, -(-threads // len(net.targets)))
    jobs = list(net.targets) * reps
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        outs = list(ex.map(lambda t: oracle.enumerate_pathways(net, t, lim), jobs))
    dt = time.perf_counter() - t0
    exp = sum(c["expansions"] for _, c in outs)
    res = sum(len(s) for s, _ in outs)
    return exp, res, dt


def host_threads():
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args):
    """Reference arm: the CPU oracle, as it stands, on the host cores."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_1804_02867_gb300 import synth

    net = synth.core()
    threads = host_threads()
    for _ in range(args.warmup):
        oracle_sample(net, REF_STEP_BUDGET, threads)
    tot_exp, tot_res, tot_t, times = 0, 0, 0.0, []
    for _ in range(args.steps):
        e, r, dt = oracle_sample(net, REF_STEP_BUDGET, threads)
        tot_exp += e
        tot_res += r
        tot_t += dt
        times.append(dt)
    value = tot_exp / tot_t
    sample = (f"core-72x95, the 8 targets x {max(1, -(-threads // 8))} jobs on {threads} threads, max_len {MAX_LEN}, "
              f"max_secondary {MAX_SEC}, frontier budget {REF_STEP_BUDGET} per step (the workload's own budget is "
              f"{args.budget})")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded core-shaped network)", "config": workload_config(args.budget),
        "balanced_pathways_per_s": tot_res / tot_t,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_1804_02867_gb300 import build as libbuild
    from paper_1804_02867_gb300 import efmgraph, synth

    libbuild.build()
    efmgraph.load_library()
    net = synth.core()
    targets = list(net.targets)
    if args.targets:
        targets = [targets[int(i)] for i in args.targets.split(",")]
    stream = torch.cuda.current_stream()
    budget = args.budget

    # CPU baseline first, before heavy GPU use (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        threads = host_threads()
        e, r, dt = oracle_sample(net, CPU_SAMPLE_BUDGET, threads)
        cpu = {"value": e / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"core-72x95, the 8 targets x {max(1, -(-threads // 8))} independent jobs on {threads} "
                         f"threads, max_len {MAX_LEN}, max_secondary {MAX_SEC}, frontier budget {CPU_SAMPLE_BUDGET} "
                         f"(GPU: {budget}); {e} expansions in {dt:.1f} s",
               "balanced_pathways_per_s": r / dt}

    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device="cuda")
    nw = efmgraph.Network(net, stream)

    def step():
        job, _ = efmgraph.efm_find_pathways(nw.handle, targets, MAX_LEN, MAX_SEC, 0, budget)
        exp = res = 0
        kl = 0
        tms = ems = eb = 0.0
        el = 0
        for i in range(len(targets)):
            _, ctr, _ = efmgraph.efm_fetch_results(job, i, copy=False)
            tm = efmgraph.efm_job_timing(job, i)
            exp += ctr["expansions"]
            res += ctr["results"]
            kl += tm["kernel_launches"]
            ems += tm["expand_ms"]
            eb += tm["expand_bytes"]
            el += tm["expand_launches"]
        efmgraph.efm_free_job(job)
        return exp, res, kl, ems, eb, el

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    tot_exp = tot_res = tot_kl = tot_el = 0
    tot_ms = tot_ems = tot_eb = 0.0
    for _ in range(args.steps):
        flush.fill_(1)  # evict L2 between timed steps (not timed)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        e, r, kl, ems, eb, el = step()
        ev1.record(stream)
        ev1.synchronize()
        tot_ms += ev0.elapsed_time(ev1)
        tot_exp += e
        tot_res += r
        tot_kl += kl
        tot_ems += ems
        tot_eb += eb
        tot_el += el
    torch.cuda.synchronize()
    clk = clocks.stop()
    if ws > 1:
        torch.distributed.barrier()

    # end to end through the C-ABI: host arrays in (pinned), results out (pinned)
    arrs = [net.row_ptr, net.col_idx, net.coef, net.reversible, net.external]
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in arrs]
    h2d = sum(p.numel() * p.element_size() for p in pinned) + 4 * len(targets)
    e2e_steps = max(1, min(args.steps, 3))
    e2e_t = 0.0
    e2e_exp = 0
    d2h = 0
    for _ in range(e2e_steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        views = [p.numpy() for p in pinned]
        h = efmgraph.efm_load_network(net.n_met, net.n_rxn, *views, stream)
        job, _ = efmgraph.efm_find_pathways(h, targets, MAX_LEN, MAX_SEC, 0, budget)
        step_d2h = 0
        for i in range(len(targets)):
            sup, ctr, _ = efmgraph.efm_fetch_results(job, i)
            e2e_exp += ctr["expansions"]
            step_d2h += sup.nbytes + 11 * 8
        efmgraph.efm_free_job(job)
        efmgraph.efm_free_net(h)
        torch.cuda.synchronize()
        e2e_t += time.perf_counter() - t0
        d2h = step_d2h

    # the other workloads, compact, after the headline's timed region (rank 0, N = 1)
    secondary = None
    if rank == 0 and ws == 1 and not args.no_secondary:
        secondary = run_secondary(args)

    # max over ranks of the device time; sum of work over ranks
    if ws > 1:
        (tot_ms, e2e_t), (tot_exp, tot_res, e2e_exp) = reduce_over_ranks([tot_ms, e2e_t], [tot_exp, tot_res, e2e_exp],
                                                                         "cuda")
    nw.close()
    if rank != 0:
        return
    peaks, peak_kind = measured_peaks()
    achieved = (tot_eb / (tot_ems * 1e-3)) / 1e9 if tot_ems > 0 else 0.0
    traffic = profile_traffic(tot_eb / max(tot_el, 1))
    line = {
        "metric": METRIC,
        "value": tot_exp / (tot_ms * 1e-3),
        "unit": UNIT,
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": tot_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32",
        "data": "synthetic (seeded core-shaped network, no dataset)",
        "config": workload_config(budget),
        "balanced_pathways_per_s": tot_res / (tot_ms * 1e-3),
        "expansions_per_step": tot_exp / args.steps / max(ws, 1),
        "results_per_step": tot_res / args.steps / max(ws, 1),
        "roofline": {
            "kernel": "level pass: generate_narrow_kernel<8> + prune_rows_kernel + write_rows_kernel<8,2> + settle_kernel<8> + dedup_kernel",
            "bound": "hbm",
            "achieved": achieved,
            "peak": float(peaks["hbm_gbs"]),
            "unit": "GB/s",
            "frac": achieved / float(peaks["hbm_gbs"]),
            "traffic": traffic,
            "peak_kind": f"{peak_kind} HBM copy bandwidth",
            "launches": tot_el,
            "avg_launch_ms": tot_ems / max(tot_el, 1),
            "alg_bytes_per_launch": tot_eb / max(tot_el, 1),
            "expand_share_of_step": tot_ems / tot_ms if tot_ms else None,
        },
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_exp / e2e_t, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": tot_kl,
        "clocks": clk,
        "secondary": secondary,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


BATCH_BUDGET = 2**12
GENOME_BUDGET = 2**22


def run_secondary(args):
    """Compact runs of the batched, genome and first-K workloads for the
    default line (each measured on its own, after the headline)."""
    from types import SimpleNamespace

    out = {}
    b = run_batched(SimpleNamespace(steps=2, warmup=1, jobs=4096))
    out["batched"] = {"jobs": 4096, "ms_per_launch": b["ms_per_step"], "expansions_per_s": b["value"],
                      "sequential_ms": b["sequential"]["ms"], "speedup_vs_sequential": b["speedup_vs_sequential"],
                      "untuned_ms": b["untuned_ms"], "tuned_speedup": b["tuned_speedup"], "autotuner": b["autotuner"]}
    g = run_genome(SimpleNamespace(steps=1, warmup=1, jobs=32, budget=BUDGET))
    out["genome"] = {"targets": 32, "max_frontier": GENOME_BUDGET, "expansions_per_s": g["value"],
                     "ms_per_step": g["ms_per_step"], "roofline_frac": g["roofline"]["frac"],
                     "status_counts": g["status_counts"]}
    f = run_firstk(SimpleNamespace(steps=1, warmup=1, jobs=192))
    out["firstk"] = {"k": FIRSTK_K, "held_out_targets": 192, "plain_over_learned_time": f["value"],
                     **{k: f["first_k"][k] for k in ("certified_both", "certified_plain_only",
                                                      "certified_learned_only", "identical_sets")}}
    return out


def run_genome(args):
    """Genome-scale shape: 1000 metabolites (850 internal), 2500 reactions
    (3125 split columns, 4096-bit supports), max_len 40, 4 secondary steps,
    frontier budget 2^22 per target, over the first --jobs of its 256
    targets (all 256 with --jobs 256)."""
    import torch

    torch.cuda.set_device(0)
    from paper_1804_02867_gb300 import build as libbuild
    from paper_1804_02867_gb300 import efmgraph, synth

    libbuild.build()
    efmgraph.load_library()
    stream = torch.cuda.current_stream()
    net = synth.genome()
    n_t = min(args.jobs, len(net.targets))
    targets = net.targets[:n_t]
    budget = args.budget if args.budget != BUDGET else GENOME_BUDGET
    nw = efmgraph.Network(net, stream)

    status_counts = {}

    def step():
        job, _ = efmgraph.efm_find_pathways(nw.handle, targets, 40, MAX_SEC, 0, budget)
        exp = res = el = 0
        eb = ems = 0.0
        for i in range(n_t):
            _, c, _ = efmgraph.efm_fetch_results(job, i, copy=False)
            key = "+".join(n for n, b in (("truncated", 1), ("capped", 2), ("overflow_dropped", 4))
                           if c["status"] & b) or "complete"
            status_counts[key] = status_counts.get(key, 0) + 1
            tm = efmgraph.efm_job_timing(job, i)
            exp += c["expansions"]
            res += c["results"]
            eb += tm["expand_bytes"]
            ems += tm["expand_ms"]
            el += tm["expand_launches"]
        efmgraph.efm_free_job(job)
        return exp, res, eb, ems, el

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    status_counts.clear()
    tot_ms = eb = ems = 0.0
    exp = res = el = 0
    for _ in range(args.steps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        e, r, b, m, n = step()
        ev1.record(stream)
        ev1.synchronize()
        tot_ms += ev0.elapsed_time(ev1)
        exp += e
        res += r
        eb += b
        ems += m
        el += n
    nw.close()
    peaks, kind = measured_peaks()
    achieved = eb / (ems * 1e-3) / 1e9 if ems else 0.0
    # DRAM traffic: the ratio ncu measured on one launch of this kernel,
    # applied to this run's algorithmic bytes per launch
    ratio = profile_figure("level_pass_genome.md", "dram_to_algorithmic_ratio")
    traffic = ratio * eb / el if ratio and el else None
    line = {
        "metric": METRIC, "value": exp / (tot_ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic (seeded genome-shaped network)",
        "config": {"workload": f"genome-1000x2500 (850 internal, 3125 split columns), {n_t} targets",
                   "max_len": 40, "max_secondary": MAX_SEC, "max_frontier": budget, "support_bits": 3136},
        "balanced_pathways_per_s": res / (tot_ms * 1e-3),
        "roofline": {"kernel": "level pass: generate_kernel<32,7> + dedup_kernel", "bound": "hbm", "achieved": achieved,
                     "peak": float(peaks["hbm_gbs"]), "unit": "GB/s", "frac": achieved / float(peaks["hbm_gbs"]),
                     "traffic": traffic, "peak_kind": f"{kind} HBM copy bandwidth", "launches": el,
                     "avg_launch_ms": ems / max(el, 1), "alg_bytes_per_launch": eb / max(el, 1)},
        "status_counts": status_counts,
    }
    return line


def run_batched(args):
    """4096 seeded networks of uneven size (10-120 metabolites, 15-200
    reactions), one target each, max_len min(30, columns), 4 secondary steps,
    frontier budget 2^12 per job: one persistent graph-captured launch
    (efm_find_pathways_batch) against the same jobs as sequential
    efm_find_pathways calls on the same GPU."""
    import torch

    torch.cuda.set_device(0)
    from paper_1804_02867_gb300 import build as libbuild
    from paper_1804_02867_gb300 import efmgraph, synth

    libbuild.build()
    efmgraph.load_library()
    stream = torch.cuda.current_stream()
    nets = [synth.batched_member(i) for i in range(args.jobs)]
    loaded = [efmgraph.Network(n, stream) for n in nets]
    handles = [h.handle for h in loaded]
    targets = [n.targets[0] for n in nets]

    def batch_once():
        job, _ = efmgraph.efm_find_pathways_batch(handles, targets, MAX_LEN, MAX_SEC, 0, BATCH_BUDGET)
        exp = res = 0
        for i in range(len(nets)):
            _, c, _ = efmgraph.efm_fetch_results(job, i, copy=False)
            exp += c["expansions"]
            res += c["results"]
        efmgraph.efm_free_job(job)
        return exp, res

    for _ in range(max(1, args.warmup)):
        batch_once()  # includes the autotuner's sample runs the first time
    torch.cuda.synchronize()
    tot_ms = 0.0
    exp = res = 0
    for _ in range(args.steps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        e, r = batch_once()
        ev1.record(stream)
        ev1.synchronize()
        tot_ms += ev0.elapsed_time(ev1)
        exp += e
        res += r
    tune = efmgraph.efm_batch_tuning()
    # the same batch in the untuned launch configuration (8 warps per job,
    # every CTA an SM holds, input order, tile 32, queue chunk 1)
    efmgraph.efm_batch_set_tuning(ctas_per_sm=0, largest_first=0, warps_per_job=8, tile=32, queue_chunk=1)
    try:
        batch_once()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            batch_once()
        ev1.record(stream)
        ev1.synchronize()
        default_ms = ev0.elapsed_time(ev1) / args.steps
    finally:
        efmgraph.efm_batch_set_tuning(None)
    # the same jobs as sequential single-job calls (one pass)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    seq_exp = 0
    for h, n in zip(loaded, nets):
        job, _ = efmgraph.efm_find_pathways(h.handle, [n.targets[0]], MAX_LEN, MAX_SEC, 0, BATCH_BUDGET)
        _, c, _ = efmgraph.efm_fetch_results(job, 0, copy=False)
        seq_exp += c["expansions"]
        efmgraph.efm_free_job(job)
    ev1.record(stream)
    ev1.synchronize()
    seq_ms = ev0.elapsed_time(ev1)
    for h in loaded:
        h.close()
    value = exp / (tot_ms * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic (seeded uneven networks)",
        "config": {"workload": f"batched: {args.jobs} networks (10-120 metabolites, 15-200 reactions), one target each",
                   "max_len": f"min({MAX_LEN}, columns)", "max_secondary": MAX_SEC, "max_frontier": BATCH_BUDGET,
                   "launch": "one persistent graph-captured kernel"},
        "balanced_pathways_per_s": res / (tot_ms * 1e-3),
        "expansions_per_step": exp / args.steps,
        "sequential": {"ms": seq_ms, "value": seq_exp / (seq_ms * 1e-3), "calls": len(nets)},
        "speedup_vs_sequential": (seq_ms / (tot_ms / args.steps)),
        "autotuner": tune,
        "untuned_ms": default_ms,
        "tuned_speedup": default_ms / (tot_ms / args.steps),
    }
    return line


FIRSTK_K = 1000
FIRSTK_TRAIN = 64         # genome target positions [0, 64) train the model
FIRSTK_BUDGET = 2**22


def run_firstk(args):
    """First-K queries (K = 1000 smallest results) on the genome-shaped
    network, learned order against plain order, same kernels, same GPU.

    Setup (untimed): a proposal model is trained on traces of plain first-K
    searches: genome targets at positions 0-63 (K = 1000), the core network's
    8 targets and 64 batched-workload networks (K = 100 each).  One step =
    the first-K query of every held-out genome target (positions 64 .. 63 +
    --jobs, at most 192), once in plain order and once in learned order.
    value = plain time / learned time over the targets both orders certify
    (the answer is exact only when no level overflows the frontier budget);
    both answers must be identical there."""
    import numpy as np
    import torch

    torch.cuda.set_device(0)
    from paper_1804_02867_gb300 import build as libbuild
    from paper_1804_02867_gb300 import efmgraph, synth

    libbuild.build()
    efmgraph.load_library()
    stream = torch.cuda.current_stream()
    net = synth.genome()
    n_eval = min(args.jobs, len(net.targets) - FIRSTK_TRAIN)
    train_t = [int(t) for t in net.targets[:FIRSTK_TRAIN]]
    eval_t = [int(t) for t in net.targets[FIRSTK_TRAIN:FIRSTK_TRAIN + n_eval]]
    nw = efmgraph.Network(net, stream)
    model = efmgraph.efm_model_create(1, stream)
    t0 = time.time()
    efmgraph.efm_model_trace(model, nw.handle, train_t, 40, MAX_SEC, FIRSTK_K, FIRSTK_BUDGET, rows_per_level=8192)
    core = synth.core()
    with efmgraph.Network(core, stream) as cw:
        efmgraph.efm_model_trace(model, cw.handle, list(core.targets), MAX_LEN, MAX_SEC, 100, FIRSTK_BUDGET, 8192)
    for i in range(64):
        bn = synth.batched_member(i)
        with efmgraph.Network(bn, stream) as bw:
            efmgraph.efm_model_trace(model, bw.handle, [bn.targets[0]], min(MAX_LEN, bw.n_columns), MAX_SEC, 100,
                                     2**16, 2048)
    n_rows, n_pos = efmgraph.efm_model_rows(model)
    trace_s = time.time() - t0
    pos_weight = float(min(50.0, max(1.0, (n_rows - n_pos) / max(n_pos, 1))))
    t0 = time.time()
    loss = efmgraph.efm_model_train(model, epochs=20, batch_tiles=16, lr=1e-3, pos_weight=pos_weight)
    train_s = time.time() - t0

    def query(t, learned):
        kw = dict(first_k=FIRSTK_K, proposal=efmgraph.EFM_LEARNED, model=model) if learned else dict(first_k=FIRSTK_K)
        (sup, ctr, tm), = efmgraph.enumerate_targets(nw, [t], 40, MAX_SEC, 0, FIRSTK_BUDGET, timing=True, **kw)
        return sup, ctr, tm

    for _ in range(args.warmup):
        for t in eval_t[:4]:
            query(t, False)
            query(t, True)
    torch.cuda.synchronize()
    rows = []
    for _ in range(args.steps):
        for t in eval_t:
            a, ca, ta = query(t, False)
            b, cb, tb = query(t, True)
            rows.append((t, a, ca, ta, b, cb, tb))
    nw.close()
    efmgraph.efm_model_free(model)
    both = [r for r in rows if not (r[2]["status"] & 1) and not (r[5]["status"] & 1)]
    plain_ms = sum(r[3]["total_ms"] for r in both)
    learned_ms = sum(r[6]["total_ms"] for r in both)
    identical = all(np.array_equal(r[1], r[4]) for r in both)
    line = {
        "metric": METRIC, "value": plain_ms / learned_ms if learned_ms else None,
        "unit": "x (time to certified first-K: plain order / learned order)", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum(r[3]["total_ms"] + r[6]["total_ms"] for r in rows) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32 (search), bf16 (model)",
        "data": "synthetic (seeded genome-shaped network; model trained on traces of other targets and networks)",
        "config": {"workload": f"first-K: genome-1000x2500, K={FIRSTK_K}, {n_eval} held-out targets",
                   "max_len": 40, "max_secondary": MAX_SEC, "max_frontier": FIRSTK_BUDGET,
                   "model": "MLP 128-256-1, BF16 weights, FP32 accumulate (tcgen05)"},
        "first_k": {"certified_both": len(both) // args.steps,
                    "certified_plain_only": sum(1 for r in rows if not (r[2]["status"] & 1) and r[5]["status"] & 1)
                    // args.steps,
                    "certified_learned_only": sum(1 for r in rows if r[2]["status"] & 1 and not (r[5]["status"] & 1))
                    // args.steps,
                    "identical_sets": identical,
                    "plain_ms": plain_ms / args.steps, "learned_ms": learned_ms / args.steps,
                    "plain_expansions": sum(r[2]["expansions"] for r in both) // args.steps,
                    "learned_expansions": sum(r[5]["expansions"] for r in both) // args.steps},
        "training": {"rows": n_rows, "positives": n_pos, "pos_weight": pos_weight, "epochs": 20,
                     "final_loss": loss, "trace_s": trace_s, "train_s": train_s},
    }
    return line


SAMPLE_WALKS = 2**20
COVERAGE_TARGET, COVERAGE_LEN = 63, 16


def run_sample(args):
    """Monte-Carlo mode (the paper's own random walks) on the core-shaped
    network: one step = 2^20 walks for each of the 8 targets (max_len 30,
    4 secondary steps).  value = AND updates per second; walks, balanced
    walks and distinct results per second alongside.  Coverage: for target
    63 at max_len 16, where the exhaustive traversal is complete, the share
    of its results the walks find as the walk count grows, next to the
    coupon-collector curve N (1 - (1 - 1/N)^C) of N equally likely results
    and its expected count N H_N to see them all (Theorem 1)."""
    import torch

    torch.cuda.set_device(0)
    from paper_1804_02867_gb300 import build as libbuild
    from paper_1804_02867_gb300 import efmgraph, synth

    libbuild.build()
    efmgraph.load_library()
    stream = torch.cuda.current_stream()
    net = synth.core()
    targets = [int(t) for t in net.targets]
    nw = efmgraph.Network(net, stream)

    def step(seed):
        tot = {"expansions": 0, "seeds": 0, "balanced": 0, "results": 0}
        for t in targets:
            _, c = efmgraph.sample_target(nw, t, MAX_LEN, MAX_SEC, seed, SAMPLE_WALKS)
            for k in tot:
                tot[k] += c[k]
        return tot

    for i in range(args.warmup):
        step(1000 + i)
    torch.cuda.synchronize()
    tot_ms = 0.0
    agg = {"expansions": 0, "seeds": 0, "balanced": 0, "results": 0}
    for i in range(args.steps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        r = step(i)
        ev1.record(stream)
        ev1.synchronize()
        tot_ms += ev0.elapsed_time(ev1)
        for k in agg:
            agg[k] += r[k]
    (full, _), = efmgraph.enumerate_targets(nw, [COVERAGE_TARGET], COVERAGE_LEN, MAX_SEC)
    n_all = len(full)
    full_set = set(map(bytes, full))
    coverage = []
    for lg in range(10, 23, 2):
        sup, c = efmgraph.sample_target(nw, COVERAGE_TARGET, COVERAGE_LEN, MAX_SEC, 7, 2**lg)
        found = set(map(bytes, sup))
        assert found <= full_set
        coverage.append({"walks": 2**lg, "found": len(found), "of": n_all,
                         "uniform_coupon_expectation": n_all * (1 - (1 - 1 / n_all) ** (2**lg))})
    nw.close()
    h_n = sum(1.0 / k for k in range(1, n_all + 1))
    sec = tot_ms * 1e-3
    line = {
        "metric": METRIC, "value": agg["expansions"] / sec, "unit": "expansions/s (AND updates of random walks)",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded core-shaped network)",
        "config": {"workload": f"Monte-Carlo walks: core-72x95, 8 targets x {SAMPLE_WALKS} walks",
                   "max_len": MAX_LEN, "max_secondary": MAX_SEC, "rng": "SplitMix64 counters"},
        "walks_per_s": agg["seeds"] / sec, "balanced_walks_per_s": agg["balanced"] / sec,
        "distinct_results_per_step": agg["results"] / args.steps,
        "coverage": {"target": COVERAGE_TARGET, "max_len": COVERAGE_LEN, "results_exhaustive": n_all,
                     "uniform_coupon_walks_to_all": n_all * h_n, "curve": coverage},
    }
    return line


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        print(json.dumps(run_batched(args)), flush=True)
    elif args.workload == "genome":
        print(json.dumps(run_genome(args)), flush=True)
    elif args.workload == "firstk":
        print(json.dumps(run_firstk(args)), flush=True)
    elif args.workload == "sample":
        print(json.dumps(run_sample(args)), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
