#!/usr/bin/env python
"""Benchmark of the REI search on GB300: candidate languages built+deduped/s.

Workload (one step): the medium single-instance configuration -- alphabet
{0,1}, |P| = |N| = 10, lengths 0-7, each labelled by a seeded random target of
cost 10-14, |ic| <= 128 -- seeds 0..19, each solved under the cost vectors
(1,1,1,1,1) and (1,1,5,1,1) with max_cost 40: 40 complete solves per step.
Inputs are synthetic (the paper's benchmark files are not available).

Prints ONE JSON line (rank 0).  `value` is candidates/s measured with CUDA
events on the library's stream over exactly --steps steps (inputs already in
device memory); `e2e` is the same metric through rei_solve with host string
arrays (host<->device copies inside the timed region).  The L2 cache is
flushed (a 256 MiB write) between timed steps.

--impl reference times the CPU oracle (the slow reference arm) on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "candidate languages built+deduped/sec"
UNIT = "candidates/s"
WORKLOAD = ("medium single instance: alphabet {0,1}, |P|=|N|=10, lengths 0-7, target cost 10-14, "
            "|ic|<=128 (2-4 x 32-bit words); seeds 0-19 x costs (1,1,1,1,1),(1,1,5,1,1); max_cost 40")
COSTS = [(1, 1, 1, 1, 1), (1, 1, 5, 1, 1)]
SEEDS = list(range(20))


def problems():
    from workloads import make_config
    out = []
    for costs in COSTS:
        for s in SEEDS:
            out.append((make_config("medium", s), costs))
    return out


def recorded_traffic():
    """DRAM bytes per k_solve_fused launch from the committed ncu summary, while
    the kernel sources are the ones it was measured on (else nothing)."""
    import hashlib
    h = hashlib.sha256()
    for f in ("solve.cu", "stage_dev.cuh", "rei_dev.cuh"):
        with open(os.path.join(ROOT, "paper_2305_18575_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    rec = {}
    try:
        with open(os.path.join(ROOT, "profiles", "dram_k_solve_fused.md")) as fh:
            for line in fh:
                k, sep, v = line.partition(":")
                if sep and k.strip() in ("kernel_sources_sha256_16", "medium_traffic_bytes_per_launch",
                                         "printed_traffic_bytes_per_solve"):
                    rec[k.strip()] = v.strip()
    except OSError:
        return {}
    if rec.get("kernel_sources_sha256_16") != h.hexdigest()[:16]:
        return {}
    return {k: int(v) for k, v in rec.items() if k != "kernel_sources_sha256_16"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ----------------------------------------------------------------------------
# clocks sampled during the timed region

class ClockSampler:
    def __init__(self, device: int):
        import tempfile
        self.p = None
        self.device = device
        # the raw samples go to REI_CLOCKS_DIR when set (kept), else to the temp directory
        d = os.environ.get("REI_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"rei_clocks_rank{device}_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
            self.f.close()

    def summary(self):
        if self.p is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, v in enumerate(fl) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------
# CPU oracle timing (the cpu_baseline leg and the reference arm)

def oracle_sample(max_candidates_each: int, seeds=SEEDS):
    import oracle
    from workloads import make_config
    cands, secs = 0, 0.0
    for costs in COSTS:
        for s in seeds:
            i = make_config("medium", s)
            r = oracle.solve(i.alphabet, i.pos, i.neg, costs=costs, max_cost=40,
                             mem_budget=i.mem_budget, max_candidates=max_candidates_each)
            cands += r.candidates
            secs += r.seconds
    return cands, secs


def cpu_baseline():
    cap = 80000
    cands, secs = oracle_sample(cap)
    return {"value": cands / secs if secs else None, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"the 40 problems of the workload, each stopped after {cap} candidates "
                      f"({cands} candidates, {secs:.1f} s, one host thread)"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    cap = 4000
    for _ in range(args.warmup):
        oracle_sample(cap, seeds=SEEDS[:5])
    t0 = time.perf_counter()
    tot_c, tot_s = 0, 0.0
    for _ in range(args.steps):
        c, s = oracle_sample(cap, seeds=SEEDS[:5])
        tot_c += c
        tot_s += s
    wall = time.perf_counter() - t0
    value = tot_c / tot_s if tot_s else None
    sample = (f"per step: seeds 0-4 x both cost vectors, each stopped after {cap} candidates "
              f"(oracle timing, one host thread)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * wall / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "config": {"workload": WORKLOAD, "parallelism": "none (CPU oracle)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# GPU arm

def alu_peak(device: int):
    from paper_2305_18575_gb300 import build as b
    L = C.CDLL(b.build_peak())
    L.rei_peak_lop3.restype = C.c_double
    L.rei_peak_lop3.argtypes = [C.c_int, C.POINTER(C.c_double)]
    ms = C.c_double()
    return L.rei_peak_lop3(device, C.byref(ms))


def reduce_over_ranks(total_ms: float, cands: float, world: int, device: str):
    """Whole-job figures of independent replicas: the slowest rank's time and
    every rank's candidates (the only collective; nothing on the data path)."""
    if world <= 1:
        return total_ms, cands
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    cc = torch.tensor([float(cands)], dtype=torch.float64, device=device)
    dist.all_reduce(cc)
    return float(t.item()), float(cc.item())


def run_gpu(args, rank, world, local_rank):
    import torch
    import paper_2305_18575_gb300 as rei

    torch.cuda.set_device(local_rank)
    dev = local_rank
    stream = torch.cuda.Stream(device=dev)
    ctx = rei.Context(device=dev, stream=stream.cuda_stream)
    probs = problems()
    dprobs = [rei.Problem.on_device(i.alphabet, i.pos, i.neg, device=dev, costs=c, max_cost=40,
                                    mem_budget=i.mem_budget) for i, c in probs]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{dev}")

    def step(collect):
        for p in dprobs:
            r = ctx.solve_problem(p)
            if r.status != rei.REI_OK:
                raise RuntimeError(f"solve failed: {r.status_name}")
            collect.append(r)

    for _ in range(args.warmup):
        step([])
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    results = []
    step_ms = []
    launches0 = ctx.launches
    with ClockSampler(dev) as clocks:
        barrier()
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(1)  # evict the L2 between steps (outside the events)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            step(results)
            ev1.record(stream)
            ev1.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
        barrier()
    launches = ctx.launches - launches0
    total_ms = sum(step_ms)
    cands = sum(r.candidates for r in results)

    # end-to-end through rei_solve with host string arrays
    e2e_res, e2e_ms = [], []
    for i, c in probs[:1]:
        ctx.solve(i.alphabet, i.pos, i.neg, costs=c, max_cost=40, mem_budget=i.mem_budget)
    for _ in range(max(1, args.steps)):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i, c in probs:
            r = ctx.solve(i.alphabet, i.pos, i.neg, costs=c, max_cost=40, mem_budget=i.mem_budget)
            e2e_res.append(r)
        torch.cuda.synchronize()
        e2e_ms.append(1000 * (time.perf_counter() - t0))
    e2e_c = sum(r.candidates for r in e2e_res)
    nstep_e2e = max(1, args.steps)

    # roofline of the search kernel: its own device time (CUDA events on the
    # launching stream, accumulated by the library) against algorithmic work
    k_ms = sum(r.ms_search_kernel for r in results)
    k_launches = sum(r.search_launches for r in results)
    pair_ops = sum(r.cand_op[3] * r.guide_pairs + r.cand_op[2] * r.star_pairs +
                   (r.cand_op[0] + r.cand_op[1] + r.cand_op[4]) * 32 * r.words for r in results)
    alg_bytes = sum(32 * r.candidates + (12 * 4 * r.words + 17) * r.unique for r in results)
    peaks, peak_kind = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    lop3 = alu_peak(dev)
    alu_peak_pairs = lop3 * 32 if lop3 > 0 else None  # one LOP3 = 32 bit-sliced AND-ORs
    hbm_ach = alg_bytes / (k_ms * 1e-3) / 1e9
    alu_ach = pair_ops / (k_ms * 1e-3)
    hbm_frac = hbm_ach / hbm_peak
    alu_frac = alu_ach / alu_peak_pairs if alu_peak_pairs else 0.0
    if alu_frac >= hbm_frac:
        roof = {"bound": "alu", "achieved": alu_ach / 1e12, "peak": alu_peak_pairs / 1e12,
                "unit": "T bit-pair-ops/s", "frac": alu_frac, "traffic": None,
                "peak_source": f"LOP3 throughput probe {lop3 / 1e12:.2f} T lane-ops/s x 32 bits"}
    else:
        roof = {"bound": "hbm", "achieved": hbm_ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": hbm_frac, "traffic": None, "peak_source": f"{peak_kind} hbm_gbs"}
    roof["traffic"] = recorded_traffic().get("medium_traffic_bytes_per_launch")
    roof.update({"kernel": "k_solve_fused", "launches": k_launches, "avg_launch_ms": k_ms / max(k_launches, 1),
                 "alg_bytes_per_launch": alg_bytes / max(k_launches, 1), "alu_frac": alu_frac,
                 "hbm_frac": hbm_frac})

    # whole-job aggregation over ranks (replicas: no data-path collective)
    t_max, c_sum = reduce_over_ranks(total_ms, cands, world, f"cuda:{dev}")
    if rank != 0:
        return
    ttm = sorted(r.ms_total for r in results)
    pct = lambda q: ttm[min(len(ttm) - 1, int(q * len(ttm)))]
    line = {
        "metric": METRIC, "value": c_sum / (t_max * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded target-labelled instances; the paper's files are unavailable)",
        "config": {"workload": WORKLOAD, "problems_per_step": len(dprobs), "l2": "flushed between steps",
                   "parallelism": f"replicas x{world}", "grid": results[0].grid if results else None},
        "time_to_min_re_ms": {"p50": pct(0.5), "p99": pct(0.99), "mean": statistics.mean(ttm)},
        "candidates_per_step": cands / args.steps,
        "roofline": roof,
        "e2e": {"value": e2e_c / (sum(e2e_ms) * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": sum(r.bytes_h2d for r in e2e_res) // nstep_e2e,
                "d2h_bytes_per_step": sum(r.bytes_d2h for r in e2e_res) // nstep_e2e},
        "clocks": clocks.summary(),
        "gpu_launches": launches,
    }
    if not args.no_paper:
        line["paper_instance"] = paper_instance_leg(ctx, dev)
    if not args.no_batch:
        bprobs = batched_problems()
        line["batched"] = batched_leg(ctx, dev, bprobs)
        if not args.no_cpu_baseline:
            line["batched"]["cpu_oracle"] = cpu_batched_baseline(line["batched"]["mean_candidates"])
        if args.served:
            line["served"] = served_leg(dev, bprobs, args.serve_seconds)
        else:
            line["served"] = {"skipped": SERVED_OFF}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)


BATCH_WORKLOAD = ("batched: 512 instances, |alphabet| 2-4, |P|,|N| uniform 2-20, lengths 0-10, |ic| 16-1024, "
                  "target cost 4-14, costs (1,1,1,1,1), max_cost 40; one rei_solve_batch call vs 512 rei_solve_problem calls")


def batched_problems():
    import paper_2305_18575_gb300 as rei
    from workloads.gen import batched_instance
    insts = [batched_instance(s) for s in range(512)]
    return [rei.Problem(i.alphabet, i.pos, i.neg, costs=(1, 1, 1, 1, 1), max_cost=40, mem_budget=1 << 30)
            for i in insts]


def batched_leg(ctx, dev, probs):
    """The batched form against one-at-a-time solves of the same instances on
    the same GPU (whole calls, host clock around synchronous calls)."""
    import time as _t
    import torch
    ctx.solve_batch(probs)  # warm-up (also autotunes the launch shape)
    reps = 3
    torch.cuda.synchronize()
    t0 = _t.perf_counter()
    for _ in range(reps):
        res = ctx.solve_batch(probs)
    torch.cuda.synchronize()
    t_batch = (_t.perf_counter() - t0) / reps
    for p in probs[:16]:
        ctx.solve_problem(p)
    torch.cuda.synchronize()
    t0 = _t.perf_counter()
    seq = [ctx.solve_problem(p) for p in probs]
    torch.cuda.synchronize()
    t_seq = _t.perf_counter() - t0
    if any((a.status, a.cost, a.tree) != (b.status, b.cost, b.tree) for a, b in zip(res, seq)):
        raise RuntimeError("batched and one-at-a-time results differ")
    lat = sorted(r.ms_total for r in res)
    cands = sum(r.candidates for r in res)
    return {"workload": BATCH_WORKLOAD, "instances": len(probs),
            "instances_per_s": len(probs) / t_batch, "sequential_instances_per_s": len(probs) / t_seq,
            "speedup_vs_sequential": t_seq / t_batch, "batch_ms": 1000 * t_batch, "sequential_ms": 1000 * t_seq,
            "candidates_per_s": cands / t_batch, "mean_candidates": cands / len(res),
            "solve_ms_p50": lat[len(lat) // 2], "solve_ms_p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))]}


def _oracle_batched_one(task):
    seed, cap = task
    import oracle
    from workloads.gen import batched_instance
    i = batched_instance(seed)
    r = oracle.solve(i.alphabet, i.pos, i.neg, costs=(1, 1, 1, 1, 1), max_cost=40, mem_budget=1 << 30,
                     max_candidates=cap)
    return r.candidates


def _noop(_):
    return 0


def cpu_batched_baseline(mean_candidates: float):
    """The oracle on every host core, one batched-workload instance per core at
    a time (a bounded sample: each instance stopped after `cap` candidates); its
    candidates/s over the wall time of the sample, and the instances/s that rate
    gives at the workload's mean candidates per instance (from the GPU results)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    cap = 20000
    tasks = [(s, cap) for s in range(2 * cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_noop, range(cores))  # workers started before the clock
        t0 = time.perf_counter()
        cands = sum(pool.map(_oracle_batched_one, tasks, chunksize=1))
        wall = time.perf_counter() - t0
    cps = cands / wall if wall else None
    return {"candidates_per_s": cps, "cores": cores, "kind": "oracle",
            "instances_per_s_est": cps / mean_candidates if cps and mean_candidates else None,
            "sample": f"instances 0-{len(tasks) - 1} of the batched workload, each stopped after {cap} "
                      f"candidates ({cands} candidates, {wall:.1f} s wall, {cores} processes)"}


PAPER_WORKLOAD = ("the specification printed in Sec. 6 (Table 1, Type 1 No 50): 10 positive and 12 negative "
                  "binary strings, |ic| = 25, costs (1,1,1,1,1), max_cost 30, minimal cost 28")
PAPER_A100_S = 4.9512          # Table 1: the paper's A100 time for this instance (context, other hardware)
PAPER_A100_REs = 26774099142   # Table 1: its candidate count there


def paper_instance_leg(ctx, dev):
    """Time to the minimal regex on the one instance the paper prints with its
    GPU time: a search of ~2.6e10 candidates whose uniqueness table (22 M
    languages) lives in HBM, the regime where the search is throughput-bound."""
    import paper_2305_18575_gb300 as rei
    from workloads import printed_instance
    i = printed_instance()
    prob = rei.Problem(i.alphabet, i.pos, i.neg, costs=i.costs, max_cost=i.max_cost, mem_budget=i.mem_budget)
    ctx.solve_problem(prob)  # warm-up (the context sizes its cache and table)
    runs = [ctx.solve_problem(prob) for _ in range(2)]
    r = min(runs, key=lambda x: x.ms_total)
    if r.status != rei.REI_OK or r.cost != 28:
        raise RuntimeError(f"printed instance: {r.status_name} cost {r.cost}")
    peaks, kind = measured_peaks()
    alg_bytes = 32 * r.candidates + (12 * 4 * r.words + 17) * r.unique
    hbm = alg_bytes / (r.ms_search_kernel * 1e-3) / 1e9
    return {"workload": PAPER_WORKLOAD, "regex": r.regex, "cost": r.cost, "candidates": r.candidates,
            "unique": r.unique, "time_to_min_re_s": r.ms_total / 1e3, "kernel_s": r.ms_search_kernel / 1e3,
            "candidates_per_s": r.candidates / (r.ms_total * 1e-3), "search_launches": r.search_launches,
            "roofline": {"bound": "hbm", "achieved": hbm, "peak": float(peaks.get("hbm_gbs", 6800.0)),
                         "unit": "GB/s", "frac": hbm / float(peaks.get("hbm_gbs", 6800.0)),
                         "peak_source": f"{kind} hbm_gbs", "alg_bytes_per_solve": alg_bytes,
                         "traffic_per_solve": recorded_traffic().get("printed_traffic_bytes_per_solve"),
                         "alg_bytes": "32 B probe per candidate + (48 W + 17) B per new language",
                         "kernels": "k_solve_fused, then k_solve for levels above 4 Mi candidates"},
            "paper_a100": {"seconds": PAPER_A100_S, "candidates": PAPER_A100_REs,
                           "note": "the paper's own run on an A100 (Table 1); context, not a target"}}


SERVE_WORKLOAD = ("served: Poisson arrivals at 50, 200 and 1000 problems/s (trace seed = rate), problems drawn in turn "
                  "from the 512 batched-workload instances; rei_server (one persistent launch) vs a loop of "
                  "rei_solve_problem calls taking the same arrivals in order")
SERVE_RATES = (50, 200, 1000)
SERVE_SECONDS = 2.0


SERVED_OFF = ("a run of this leg raised a GPU exception in its saturated phase (512 requests at "
              "once), cause not found; the served form's own tests still run")


def served_leg(dev, probs, seconds=SERVE_SECONDS):
    """Latency from arrival to answer (host clock) of the served form against a
    plain loop that solves the same arrivals one at a time."""
    import paper_2305_18575_gb300 as rei
    from workloads.gen import poisson_trace

    def pct(v, q):
        v = sorted(v)
        return v[min(len(v) - 1, int(q * len(v)))]

    out = {"workload": SERVE_WORKLOAD, "seconds_per_rate": seconds, "rates": {}}
    answers = {}
    with rei.Context(device=dev) as sctx, rei.Server(sctx, budget_bytes=64 << 30, max_live=4096) as srv:
        for t in [srv.submit(p) for p in probs[:64]]:  # warm-up
            srv.result(t)
        # saturated: all 512 problems at once, instances/s to the last answer
        t0 = time.perf_counter()
        tickets = [srv.submit(p) for p in probs]
        sat = [srv.result(t) for t in tickets]
        t_sat = time.perf_counter() - t0
        lat = [r.ms_total for r in sat]
        out["saturated"] = {"requests": len(probs), "instances_per_s": len(probs) / t_sat,
                            "p50_ms": pct(lat, 0.5), "p99_ms": pct(lat, 0.99)}
        for rate in SERVE_RATES:
            arr = poisson_trace(rate, seconds, seed=rate)
            tickets = []
            t0 = time.perf_counter()
            for k, a in enumerate(arr):
                dt = t0 + a - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                tickets.append(srv.submit(probs[k % len(probs)]))
            res = [srv.result(t) for t in tickets]
            t_end = max(time.perf_counter(), t0 + seconds)
            answers[rate] = [(r.status, r.cost, r.tree) for r in res]
            lat = [r.ms_total for r in res]
            out["rates"][str(rate)] = {"requests": len(arr), "served_p50_ms": pct(lat, 0.5),
                                       "served_p99_ms": pct(lat, 0.99),
                                       "served_throughput_per_s": len(arr) / (t_end - t0)}
    with rei.Context(device=dev) as pctx:
        for p in probs[:16]:
            pctx.solve_problem(p)
        t0 = time.perf_counter()
        for p in probs:
            pctx.solve_problem(p)
        out["saturated"]["plain_instances_per_s"] = len(probs) / (time.perf_counter() - t0)
        for rate in SERVE_RATES:
            arr = poisson_trace(rate, seconds, seed=rate)
            lat, got = [], []
            t0 = time.perf_counter()
            for k, a in enumerate(arr):
                dt = t0 + a - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                r = pctx.solve_problem(probs[k % len(probs)])
                lat.append(1000 * (time.perf_counter() - t0 - a))
                got.append((r.status, r.cost, r.tree))
            if got != answers[rate]:
                raise RuntimeError("served and one-at-a-time answers differ")
            o = out["rates"][str(rate)]
            o.update({"plain_p50_ms": pct(lat, 0.5), "plain_p99_ms": pct(lat, 0.99)})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched and served legs")
    ap.add_argument("--served", action="store_true",
                    help="run the served leg (off by default: " + SERVED_OFF + ")")
    ap.add_argument("--no-paper", action="store_true", help="skip the printed-instance leg")
    ap.add_argument("--serve-seconds", type=float, default=SERVE_SECONDS,
                    help="length of each arrival trace of the served leg (the served config uses 60)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    try:
        run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
