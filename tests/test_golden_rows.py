"""The stored oracle results used by the GPU parity tests of the batched and
served forms still equal what the oracle computes now (a sample of rows;
CPU only).  A stale file after a change to the generator or the oracle fails
here instead of in a GPU run."""
import pytest

import oracle
from workloads import make_config

from conftest import load_expected


@pytest.mark.parametrize("name,kind,seeds", [("batched_expected.txt", "batched", (0, 7, 100, 255, 446, 511)),
                                             ("served_expected.txt", "served", (0, 23, 63))])
def test_stored_rows_equal_the_oracle(name, kind, seeds):
    rows = load_expected(name)
    for s in seeds:
        i = make_config(kind, s)
        r = oracle.solve(i.alphabet, i.pos, i.neg, costs=(1, 1, 1, 1, 1), max_cost=40, mem_budget=1 << 30)
        assert rows[s] == (r.status, r.cost, r.candidates, r.unique, r.n_ic, r.tree or b""), (kind, s)
        # the stored answer is precise and no costlier than the instance's target
        assert all(oracle.match(r.tree, i.alphabet, p) for p in i.pos)
        assert not any(oracle.match(r.tree, i.alphabet, q) for q in i.neg)
        assert r.cost <= i.target_cost


def test_stored_wide_large_rows_equal_the_oracle():
    """Two of the stored |ic| 1000-1500 rows (the quick ones) against the oracle now."""
    import os
    from workloads import wide_large_instance
    path = os.path.join(os.path.dirname(__file__), "golden", "wide_large_expected.txt")
    rows = {(l.split()[0], int(l.split()[1])): l.split()[2:] for l in open(path) if not l.startswith("#")}
    for var, seed in (("len10", 0), ("30x30", 0)):
        i = wide_large_instance(var, seed)
        r = oracle.solve(i.alphabet, i.pos, i.neg, max_cost=40, mem_budget=i.mem_budget)
        st, cost, cand, uniq, n_ic, tree = rows[(var, seed)]
        assert (r.status, r.cost, r.candidates, r.unique, r.n_ic, r.tree.hex()) == \
            (int(st), int(cost), int(cand), int(uniq), int(n_ic), tree)
        assert 1000 <= r.n_ic <= 1500
