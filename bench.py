#!/usr/bin/env python
"""Benchmark of the REI search on GB300: candidate languages built+deduped/s.

Workload (one step, the headline `value`): the medium single-instance
configuration -- alphabet {0,1}, |P| = |N| = 10, lengths 0-7, each labelled by a
seeded random target of cost 10-14, |ic| <= 128 -- seeds 0..19, each solved
under the cost vectors (1,1,1,1,1) and (1,1,5,1,1) with max_cost 40: 40
complete solves per step.  Inputs are synthetic (the paper's benchmark files
are not available).

Prints ONE JSON line (rank 0).  `value` is candidates/s measured with CUDA
events on the library's stream over exactly --steps steps (inputs already in
device memory); `e2e` is the same metric through rei_solve with host string
arrays (host<->device copies inside the timed region).  The L2 cache is
flushed (a 256 MiB write) between timed steps.  Further legs on the same line:
the wide configuration (multiword languages), the paper's printed instance
(the throughput regime) and the batched form.

--impl reference times the CPU oracle (the slow reference arm) on the same 40
problems, each stopped after a stated number of candidates.
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


def kernel_sources_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("solve.cu", "stage_dev.cuh", "rei_dev.cuh"):
        with open(os.path.join(ROOT, "paper_2305_18575_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes of the search kernels from the committed one-pass ncu capture
    (profiles/dram_traffic.json), while the kernel sources are the ones it was
    measured on (else nothing)."""
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return {}
    if rec.get("kernel_sources_sha256_16") != kernel_sources_hash():
        return {}
    return {k: v for k, v in rec.items() if isinstance(v, int)}


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
# CPU oracle timing (the cpu_baseline legs and the reference arm)

def oracle_sample(probs, max_candidates_each: int, max_cost: int = 40):
    """The oracle on (instance, costs) pairs, each stopped after
    max_candidates_each candidates: (candidates, seconds of oracle time)."""
    import oracle
    cands, secs = 0, 0.0
    for i, costs in probs:
        r = oracle.solve(i.alphabet, i.pos, i.neg, costs=costs, max_cost=max_cost,
                         mem_budget=i.mem_budget, max_candidates=max_candidates_each)
        cands += r.candidates
        secs += r.seconds
    return cands, secs


def cpu_baseline():
    cap = 80000
    cands, secs = oracle_sample(problems(), cap)
    return {"value": cands / secs if secs else None, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"the 40 problems of the workload, each stopped after {cap} candidates "
                      f"({cands} candidates, {secs:.1f} s, one host thread)"}


REF_CAP = 20000  # candidates per problem and step of the reference arm


def config_of(world: int) -> dict:
    """The workload as both arms name it (the same problems in both)."""
    return {"workload": WORKLOAD, "problems_per_step": len(SEEDS) * len(COSTS), "parallelism": f"replicas x{world}"}


def run_reference(args, rank, world):
    """The CPU oracle on the GPU arm's 40 problems, each stopped after REF_CAP
    candidates per step (rank 0 only)."""
    if rank != 0:
        return
    probs = problems()
    for _ in range(args.warmup):
        oracle_sample(probs, REF_CAP)
    t0 = time.perf_counter()
    tot_c, tot_s = 0, 0.0
    for _ in range(args.steps):
        c, s = oracle_sample(probs, REF_CAP)
        tot_c += c
        tot_s += s
    wall = time.perf_counter() - t0
    value = tot_c / tot_s if tot_s else None
    sample = (f"per step: the 40 problems of the workload (seeds 0-19 x both cost vectors), each stopped "
              f"after {REF_CAP} candidates ({tot_c // max(args.steps, 1)} candidates per step; oracle timing, "
              f"one host thread)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * wall / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "config": config_of(world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# GPU arm

def _peak_lib():
    from paper_2305_18575_gb300 import build as b
    L = C.CDLL(b.build_peak())
    L.rei_peak_lop3.restype = C.c_double
    L.rei_peak_lop3.argtypes = [C.c_int, C.POINTER(C.c_double)]
    L.rei_peak_l2_random.restype = C.c_double
    L.rei_peak_l2_random.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_double)]
    return L


def alu_peak(device: int):
    """LOP3 lane-operations per second of the GPU (the integer-throughput probe)."""
    ms = C.c_double()
    return _peak_lib().rei_peak_lop3(device, C.byref(ms))


def l2_peak(device: int):
    """Bytes per second of random 32-byte sectors the L2 serves (the probe's
    best of three runs over a 32 MiB buffer that stays resident)."""
    ms = C.c_double()
    return max(_peak_lib().rei_peak_l2_random(device, 32, C.byref(ms)) for _ in range(3))


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


def alg_work(results):
    """Algorithmic work of a set of solves (per-candidate figures of the
    method): bytes = a 32-byte uniqueness probe per candidate + (48 W + 17)
    bytes per new language; bit-pair operations = G per concatenation, G* per
    star, 32 W per symbol, ? and + candidate."""
    bytes_ = sum(32 * r.candidates + (12 * 4 * r.words + 17) * r.unique for r in results)
    pairs = sum(r.cand_op[3] * r.guide_pairs + r.cand_op[2] * r.star_pairs +
                (r.cand_op[0] + r.cand_op[1] + r.cand_op[4]) * 32 * r.words for r in results)
    return bytes_, pairs


def l2_resident(results) -> bool:
    """Whether the uniqueness probes of these solves hit a structure that fits
    the L2: the bitmap of cached languages of 1-word languages (2^|ic| bits,
    at most 64 MiB for |ic| <= 29)."""
    return bool(results) and all(r.words == 1 and r.n_ic <= 29 for r in results)


def roofline(results, k_ms: float, launches: int, lop3: float, kernel: str, traffic=None, l2=None):
    """The roofs of a kernel from its algorithmic work and its CUDA-event time.
    `bound`: the L2 (random 32-byte sectors, measured) when the uniqueness
    probes hit an L2-resident bitmap and `l2` (its peak, bytes/s) is given,
    else the better-fitting of HBM and the integer pipes (the larger
    fraction).  Every fraction is reported."""
    peaks, peak_kind = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    alg_bytes, pair_ops = alg_work(results)
    alu_peak_pairs = lop3 * 32 if lop3 > 0 else None  # one LOP3 = 32 bit-sliced AND-ORs
    hbm_ach = alg_bytes / (k_ms * 1e-3) / 1e9 if k_ms > 0 else 0.0
    alu_ach = pair_ops / (k_ms * 1e-3) if k_ms > 0 else 0.0
    hbm_frac = hbm_ach / hbm_peak
    alu_frac = alu_ach / alu_peak_pairs if alu_peak_pairs else 0.0
    l2_gbs = l2 / 1e9 if l2 else None
    l2_frac = hbm_ach / l2_gbs if l2_gbs else None
    if l2_gbs and l2_resident(results):
        roof = {"bound": "l2", "achieved": hbm_ach, "peak": l2_gbs, "unit": "GB/s", "frac": l2_frac}
    elif alu_frac > hbm_frac:
        roof = {"bound": "alu", "achieved": alu_ach / 1e12, "peak": alu_peak_pairs / 1e12,
                "unit": "T bit-pair-ops/s", "frac": alu_frac}
    else:
        roof = {"bound": "hbm", "achieved": hbm_ach, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_frac}
    roof.update({"traffic": traffic, "kernel": kernel, "launches": launches,
                 "avg_launch_ms": k_ms / max(launches, 1), "alg_bytes_per_launch": alg_bytes / max(launches, 1),
                 "hbm_frac": hbm_frac, "hbm_peak_gbs": hbm_peak, "hbm_peak_source": f"{peak_kind} hbm_gbs",
                 "alu_frac": alu_frac, "lop3_lane_ops_per_s": lop3,
                 "alu_peak_source": "LOP3 throughput probe (peak.cu) x 32 bit-slices"})
    if l2_gbs:
        roof.update({"l2_frac": l2_frac, "l2_random_sector_peak_gbs": l2_gbs,
                     "l2_peak_source": "L2 random 32-byte-sector probe (peak.cu), best of 3"})
    return roof


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
    lop3 = alu_peak(dev)
    roof = roofline(results, sum(r.ms_search_kernel for r in results), sum(r.search_launches for r in results),
                    lop3, "k_solve_fused", recorded_traffic().get("medium_traffic_bytes_per_launch"))

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
        "config": config_of(world),
        "launch": {"grid": results[0].grid if results else None, "l2": "flushed between steps (256 MiB write)"},
        "time_to_min_re_ms": {"p50": pct(0.5), "p99": pct(0.99), "mean": statistics.mean(ttm)},
        "candidates_per_step": cands / args.steps,
        "roofline": roof,
        "e2e": {"value": e2e_c / (sum(e2e_ms) * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": sum(r.bytes_h2d for r in e2e_res) // nstep_e2e,
                "d2h_bytes_per_step": sum(r.bytes_d2h for r in e2e_res) // nstep_e2e},
        "clocks": clocks.summary(),
        "gpu_launches": launches,
    }
    if not args.no_wide:
        line["wide"] = wide_leg(ctx, lop3, cpu=not args.no_cpu_baseline)
    if not args.no_paper:
        line["paper_instance"] = paper_instance_leg(ctx, lop3, l2_peak(dev))
    if not args.no_batch:
        bprobs = batched_problems()
        line["batched"] = batched_leg(ctx, dev, bprobs)
        if not args.no_cpu_baseline:
            line["batched"]["cpu_oracle"] = cpu_batched_baseline(line["batched"]["mean_candidates"])
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# the wide configuration: multiword languages

WIDE_WORKLOAD = ("wide single instance: alphabet {a,b,c,d}, |P|=|N|=20, lengths 1-10, target cost 12-18, "
                 "|ic| 400-1500 (16-48 x 32-bit words); seeds 0-9, costs (1,1,1,1,1), max_cost 40, "
                 "memory budget 64 GB")
WIDE_SEEDS = list(range(10))


def wide_problems():
    from workloads import make_config
    return [(make_config("wide", s), (1, 1, 1, 1, 1)) for s in WIDE_SEEDS]


def wide_leg(ctx, lop3: float, cpu: bool = True, reps: int = 3):
    """Time to the minimal regex of each wide problem (whole rei_solve_problem
    calls, host clock, inputs in host memory), candidates/s over the search
    kernels' CUDA-event time, and their roofline."""
    import paper_2305_18575_gb300 as rei
    wp = wide_problems()
    probs = [rei.Problem(i.alphabet, i.pos, i.neg, costs=c, max_cost=40, mem_budget=i.mem_budget) for i, c in wp]
    for p in probs:  # warm-up (the context sizes its buffers)
        ctx.solve_problem(p)
    res = []
    for _ in range(reps):
        for p in probs:
            r = ctx.solve_problem(p)
            if r.status != rei.REI_OK:
                raise RuntimeError(f"wide solve failed: {r.status_name}")
            res.append(r)
    ttm = sorted(r.ms_total for r in res)
    pct = lambda q: ttm[min(len(ttm) - 1, int(q * len(ttm)))]
    k_ms = sum(r.ms_search_kernel for r in res)
    cands = sum(r.candidates for r in res)
    out = {"workload": WIDE_WORKLOAD, "solves": len(res), "n_ic": sorted({r.n_ic for r in res}),
           "words": sorted({r.words for r in res}),
           "candidates_per_s": cands / (k_ms * 1e-3) if k_ms else None,
           "candidates_per_s_wall": cands / (sum(ttm) * 1e-3),
           "time_to_min_re_ms": {"p50": pct(0.5), "p99": pct(0.99), "mean": statistics.mean(ttm)},
           "roofline": roofline(res, k_ms, sum(r.search_launches for r in res), lop3, "k_solve_fused / k_solve")}
    if cpu:
        cap = 20000
        c, s = oracle_sample(wp, cap)
        out["cpu_baseline"] = {"value": c / s if s else None, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"the 10 wide problems, each stopped after {cap} candidates "
                                         f"({c} candidates, {s:.1f} s, one host thread)"}
    return out


# ----------------------------------------------------------------------------
# the batched form

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


# ----------------------------------------------------------------------------
# the paper's printed instance: the throughput regime

PAPER_WORKLOAD = ("the specification printed in Sec. 6 (Table 1, Type 1 No 50): 10 positive and 12 negative "
                  "binary strings, |ic| = 25, costs (1,1,1,1,1), max_cost 30, minimal cost 28")
PAPER_A100_S = 4.9512          # Table 1: the paper's A100 time for this instance (context, other hardware)
PAPER_A100_REs = 26774099142   # Table 1: its candidate count there


def paper_instance_leg(ctx, lop3: float, l2: float):
    """Time to the minimal regex on the one instance the paper prints with its
    GPU time: a search of ~2.6e10 candidates whose uniqueness structures live
    in HBM, the regime where the search is throughput-bound."""
    import paper_2305_18575_gb300 as rei
    from workloads import printed_instance
    i = printed_instance()
    prob = rei.Problem(i.alphabet, i.pos, i.neg, costs=i.costs, max_cost=i.max_cost, mem_budget=i.mem_budget)
    ctx.solve_problem(prob)  # warm-up (the context sizes its cache and table)
    runs = [ctx.solve_problem(prob) for _ in range(2)]
    r = min(runs, key=lambda x: x.ms_total)
    if r.status != rei.REI_OK or r.cost != 28:
        raise RuntimeError(f"printed instance: {r.status_name} cost {r.cost}")
    roof = roofline([r], r.ms_search_kernel, r.search_launches, lop3, "k_solve_fused, then k_solve", l2=l2)
    alg_bytes, _ = alg_work([r])
    roof.update({"alg_bytes_per_solve": alg_bytes, "traffic": None,
                 "traffic_per_solve": recorded_traffic().get("printed_traffic_bytes_per_solve"),
                 "alg_bytes": "32 B probe per candidate + (48 W + 17) B per new language"})
    return {"workload": PAPER_WORKLOAD, "regex": r.regex, "cost": r.cost, "candidates": r.candidates,
            "unique": r.unique, "time_to_min_re_s": r.ms_total / 1e3, "kernel_s": r.ms_search_kernel / 1e3,
            "candidates_per_s": r.candidates / (r.ms_total * 1e-3), "search_launches": r.search_launches,
            "roofline": roof,
            "paper_a100": {"seconds": PAPER_A100_S, "candidates": PAPER_A100_REs,
                           "note": "the paper's own run on an A100 (Table 1); context, not a target"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched leg")
    ap.add_argument("--no-wide", action="store_true", help="skip the wide-configuration leg")
    ap.add_argument("--no-paper", action="store_true", help="skip the printed-instance leg")
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
