"""Writes wide_expected.txt: the oracle's results on the wide configuration
(seeds 0-9, costs (1,1,1,1,1), max_cost 40), for the GPU parity test at full
size.  Calls only the oracle and the seeded generator.

    python tests/golden/make_wide_expected.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from workloads import make_config  # noqa: E402


def main():
    lines = ["# wide configuration, costs (1,1,1,1,1), max_cost 40: the oracle's results",
             "# seed status cost candidates unique n_ic tree(hex)"]
    for s in range(10):
        i = make_config("wide", s)
        r = oracle.solve(i.alphabet, i.pos, i.neg, max_cost=40, mem_budget=i.mem_budget)
        lines.append(f"{s} {r.status} {r.cost} {r.candidates} {r.unique} {r.n_ic} {(r.tree or b'').hex()}")
        print(lines[-1], flush=True)
    with open(os.path.join(HERE, "wide_expected.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
