"""Solve workload instances from the command line (also the profiling driver).

    python -m paper_2305_18575_gb300.cli medium 16 --costs 1,1,5,1,1 [--repeat 3]

Prints one line per solve: status, cost, expression, candidates, unique, times.
"""
from __future__ import annotations

import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main(argv=None):
    import paper_2305_18575_gb300 as rei
    from workloads import make_config, printed_instance

    ap = argparse.ArgumentParser()
    ap.add_argument("config", choices=["small", "medium", "wide", "batched", "served", "printed"])
    ap.add_argument("seed", type=int)
    ap.add_argument("--costs", default="1,1,1,1,1")
    ap.add_argument("--max-cost", type=int, default=None, help="default: 30 for the printed instance, else 40")
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--cache-init", type=int, default=0, help="initial cache rows (0 = library default)")
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--device-input", action="store_true")
    ap.add_argument("--solo-tiles", type=int, default=None, help="chunks of at most this many tiles run on one CTA")
    ap.add_argument("--grid", type=int, default=0)
    a = ap.parse_args(argv)
    costs = tuple(int(x) for x in a.costs.split(","))
    inst = printed_instance() if a.config == "printed" else make_config(a.config, a.seed)
    with rei.Context(device=0) as ctx:
        if a.cache_init:
            ctx.set_option(rei.REI_OPT_CACHE_INIT, a.cache_init)
        if a.chunk:
            ctx.set_option(rei.REI_OPT_CHUNK, a.chunk)
        if a.solo_tiles is not None:
            ctx.set_option(rei.REI_OPT_SOLO_TILES, a.solo_tiles)
        if a.grid:
            ctx.set_option(rei.REI_OPT_GRID, a.grid)
        mk = rei.Problem.on_device if a.device_input else rei.Problem
        max_cost = a.max_cost if a.max_cost is not None else inst.max_cost if a.config == "printed" else 40
        prob = mk(inst.alphabet, inst.pos, inst.neg, costs=costs, max_cost=max_cost,
                  mem_budget=inst.mem_budget)
        for _ in range(a.repeat):
            r = ctx.solve_problem(prob)
            print(f"{a.config}:{a.seed} costs={costs} n_ic={r.n_ic} W={r.words} status={r.status_name} "
                  f"cost={r.cost} regex={r.regex} candidates={r.candidates} unique={r.unique} "
                  f"ms_total={r.ms_total:.3f} ms_search_kernel={r.ms_search_kernel:.3f} "
                  f"launches={r.launches} grid={r.grid}", flush=True)
            if r.status not in (rei.REI_OK, rei.REI_NOT_FOUND, rei.REI_OOM):
                return 1
    return 0


if __name__ == "__main__":
    sys.exit(main())
