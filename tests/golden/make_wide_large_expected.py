"""Writes wide_large_expected.txt: the oracle's results on wide instances whose
|ic| is 1000-1500 words (32-bit words per language: 36 and 48), costs
(1,1,1,1,1), max_cost 40, for the GPU parity test at those widths.  Calls only
the oracle and the seeded generator (workloads.wide_large_instance).

    python tests/golden/make_wide_large_expected.py [processes]
"""
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

# (variant, seed): seeds whose search the oracle finishes in minutes
CASES = [("len10", 0), ("len10", 9), ("len10", 20), ("len10", 21), ("len10", 7),
         ("30x30", 0), ("30x30", 10), ("30x30", 7)]


def solve(case):
    import oracle
    from workloads import wide_large_instance
    variant, seed = case
    i = wide_large_instance(variant, seed)
    r = oracle.solve(i.alphabet, i.pos, i.neg, max_cost=40, mem_budget=i.mem_budget)
    return variant, seed, r.status, r.cost, r.candidates, r.unique, r.n_ic, (r.tree or b"").hex()


def main():
    procs = int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count() or 1
    with mp.get_context("spawn").Pool(procs) as pool:
        rows = pool.map(solve, CASES, chunksize=1)
    lines = ["# wide instances with |ic| 1000-1500, costs (1,1,1,1,1), max_cost 40: the oracle's results",
             "# variant seed status cost candidates unique n_ic tree(hex)"]
    lines += [" ".join(str(x) for x in r) for r in rows]
    with open(os.path.join(HERE, "wide_large_expected.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
