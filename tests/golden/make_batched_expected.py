"""Writes batched_expected.txt and served_expected.txt: the oracle's results on
every instance of the batched configuration (512 instances, |ic| 16-1024) and
on the served pool (instances 0-63 of the served configuration, |ic| 16-2048),
costs (1,1,1,1,1), max_cost 40, for the GPU parity tests of the batched and
served forms.  Calls only the oracle and the seeded generator.

    python tests/golden/make_batched_expected.py [processes]
"""
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

BATCHED = 512
SERVED = 64
BUDGET = 1 << 30  # the memory budget both forms' tests give every problem


def solve(task):
    kind, seed = task
    import oracle
    from workloads import make_config
    i = make_config(kind, seed)
    t = time.time()
    r = oracle.solve(i.alphabet, i.pos, i.neg, costs=(1, 1, 1, 1, 1), max_cost=40, mem_budget=BUDGET)
    return kind, seed, r.status, r.cost, r.candidates, r.unique, r.n_ic, (r.tree or b"").hex(), time.time() - t


def main():
    procs = int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count() or 1
    tasks = [("batched", s) for s in range(BATCHED)] + [("served", s) for s in range(SERVED)]
    rows = {"batched": [], "served": []}
    with mp.get_context("spawn").Pool(procs) as pool:
        for kind, seed, st, cost, cand, uniq, n_ic, tree, secs in pool.imap_unordered(solve, tasks):
            rows[kind].append((seed, st, cost, cand, uniq, n_ic, tree))
            print(kind, seed, st, cost, cand, n_ic, f"{secs:.1f}s", flush=True)
    for kind, n in (("batched", BATCHED), ("served", SERVED)):
        lines = [f"# {kind} configuration, instances 0-{n - 1}, costs (1,1,1,1,1), max_cost 40, "
                 f"memory budget {BUDGET}: the oracle's results",
                 "# seed status cost candidates unique n_ic tree(hex)"]
        for seed, st, cost, cand, uniq, n_ic, tree in sorted(rows[kind]):
            lines.append(f"{seed} {st} {cost} {cand} {uniq} {n_ic} {tree}")
        with open(os.path.join(HERE, f"{kind}_expected.txt"), "w") as f:
            f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
