"""The served form (rei_server_*): problems that arrive at any time are solved by
one persistent launch as its CTAs free up.  Every result must be exactly the one
the plain entry point gives for the problem alone, whatever else is in flight."""
import random
import threading
import time

import pytest

import oracle
import paper_2305_18575_gb300 as rei
from workloads import make_config, type1_instance
from workloads.gen import batched_instance

from conftest import load_expected
from test_batch_gpu import ST, key, mixed_problems

pytestmark = pytest.mark.gpu


def test_serve_matches_plain_solves():
    probs = mixed_problems()
    with rei.Context(device=0) as ctx:
        plain = [ctx.solve_problem(p) for p in probs]
        with rei.Server(ctx, budget_bytes=64 << 30, max_live=4096) as srv:
            tickets = [srv.submit(p) for p in probs]
            got = [srv.result(t) for t in tickets]
    for k, (a, b) in enumerate(zip(plain, got)):
        assert key(a) == key(b), (k, a, b)
    assert got[5].status == rei.REI_EINVAL and got[9].status == rei.REI_EINVAL


def test_serve_small_budget_and_staggered_arrivals():
    """A budget that admits one or two problems at a time, arrivals spread over
    time (some after the launch has gone idle and returned), two submitting
    threads."""
    insts = [batched_instance(s) for s in range(40)] + [make_config("small", s) for s in range(20)]
    probs = [rei.Problem(i.alphabet, i.pos, i.neg, costs=(1, 1, 1, 1, 1), max_cost=40, mem_budget=48 << 20)
             for i in insts]
    with rei.Context(device=0) as ctx:
        plain = [ctx.solve_problem(p) for p in probs]
        with rei.Server(ctx, budget_bytes=80 << 20, max_live=3) as srv:
            tickets = [None] * len(probs)
            rng = random.Random(7)
            gaps = [rng.choice([0.0, 0.0, 0.001, 0.01, 0.3]) for _ in probs]

            def submit(ids):
                for k in ids:
                    time.sleep(gaps[k])
                    tickets[k] = srv.submit(probs[k])

            th = [threading.Thread(target=submit, args=(list(range(j, len(probs), 2)),)) for j in range(2)]
            for t in th:
                t.start()
            for t in th:
                t.join()
            got = [srv.result(t) for t in tickets]
    for k, (a, b) in enumerate(zip(plain, got)):
        assert key(a) == key(b), (k, a, b)


def test_serve_matches_oracle_on_small_problems():
    insts = [make_config("small", s) for s in range(24)] + [type1_instance(s, 3, 3, 3) for s in range(6)]
    costs = (2, 1, 1, 1, 3)
    probs = [rei.Problem(i.alphabet, i.pos, i.neg, costs=costs, max_cost=24) for i in insts]
    with rei.Context(device=0) as ctx, rei.Server(ctx) as srv:
        tickets = [srv.submit(p) for p in probs]
        got = [srv.result(t) for t in tickets]
    for i, g in zip(insts, got):
        ref = oracle.solve(i.alphabet, i.pos, i.neg, costs=costs, max_cost=24)
        assert (g.status, g.cost, g.tree, g.candidates, g.unique) == \
            (rei.REI_OK, ref.cost, ref.tree, ref.candidates, ref.unique)


def test_serve_requests_larger_than_a_ring_entry():
    """More strings than a ring entry holds: solved alone on the plain path."""
    tails = [b""] + [format(v, f"0{n}b").encode() for n in range(1, 8) for v in range(1 << n)]
    pos = [b"1" + t for t in tails]
    neg = [b"0" + t for t in tails]
    assert len(pos) + len(neg) > 255
    big = rei.Problem(b"01", pos, neg, max_cost=12, mem_budget=1 << 30)
    small = [rei.Problem(i.alphabet, i.pos, i.neg, max_cost=20) for i in (make_config("small", s) for s in range(4))]
    with rei.Context(device=0) as ctx:
        plain = [ctx.solve_problem(p) for p in [big] + small]
        with rei.Server(ctx) as srv:
            tickets = [srv.submit(p) for p in small[:2] + [big] + small[2:]]
            got = [srv.result(t) for t in tickets]
    got = [got[2]] + got[:2] + got[3:]
    for a, b in zip(plain, got):
        assert key(a) == key(b)
    # 1(0+1)* costs 6: the answer costs at most that and separates the sides
    assert got[0].status == rei.REI_OK and got[0].cost <= 6
    assert all(oracle.match(got[0].tree, b"01", w) for w in pos[::7])
    assert not any(oracle.match(got[0].tree, b"01", w) for w in neg[::7])


def test_serve_poll_without_blocking_and_not_found():
    i = make_config("small", 5)
    with rei.Context(device=0) as ctx, rei.Server(ctx) as srv:
        t = srv.submit(rei.Problem(i.alphabet, i.pos, i.neg, max_cost=1))
        r = None
        for _ in range(2000):
            r = srv.result(t, block_ms=0)
            if r is not None:
                break
            time.sleep(0.005)
        assert r is not None and r.status == rei.REI_NOT_FOUND
        with pytest.raises(RuntimeError):
            srv.result(t, block_ms=0)  # released once read


def test_serve_with_per_symbol_costs():
    insts = [make_config("small", s) for s in range(10)] + [batched_instance(s) for s in range(10)]
    probs = []
    for k, i in enumerate(insts):
        sc = [1 + (a * 5 + k) % 3 for a in range(len(i.alphabet))]
        probs.append(rei.Problem(i.alphabet, i.pos, i.neg, max_cost=40, mem_budget=1 << 30, sym_costs=sc))
    with rei.Context(device=0) as ctx:
        plain = [ctx.solve_problem(p) for p in probs]
        with rei.Server(ctx) as srv:
            got = [srv.result(t) for t in [srv.submit(p) for p in probs]]
    for k, (a, b) in enumerate(zip(plain, got)):
        assert key(a) == key(b), k



@pytest.mark.parametrize("yield_us", [0, 1, 300])
def test_serve_time_allowance_does_not_change_results(yield_us):
    probs = mixed_problems()
    with rei.Context(device=0) as ctx:
        plain = [ctx.solve_problem(p) for p in probs]
        ctx.set_option(rei.REI_OPT_YIELD_US, yield_us)
        with rei.Server(ctx) as srv:
            got = [srv.result(t) for t in [srv.submit(p) for p in probs]]
    for k, (a, b) in enumerate(zip(plain, got)):
        assert key(a) == key(b), (k, yield_us)


def test_served_pool_matches_stored_oracle_results():
    """The served configuration's pool (instances 0-63, |ic| up to 2048 by
    the recipe): every served result equals the oracle's stored result
    (tests/golden/make_batched_expected.py, which calls only the oracle).  At
    most eight problems are live at once."""
    from workloads import make_config
    want = load_expected("served_expected.txt")
    insts = [make_config("served", s) for s in sorted(want)]
    probs = [rei.Problem(i.alphabet, i.pos, i.neg, costs=(1, 1, 1, 1, 1), max_cost=40, mem_budget=1 << 30)
             for i in insts]
    with rei.Context(device=0) as ctx, rei.Server(ctx, budget_bytes=8 << 30, max_live=8) as srv:
        got = [srv.result(t) for t in [srv.submit(p) for p in probs]]
    for s, r in zip(sorted(want), got):
        st, cost, cand, uniq, n_ic, tree = want[s]
        assert r.status == ST[st], s
        assert (r.cost, r.tree, r.candidates, r.unique, r.n_ic) == (cost, tree, cand, uniq, n_ic), s


def test_serve_sessions_on_one_context_match_plain():
    """Servers created one after another on one context reuse memory the
    earlier ones (and the plain solves) freed; every session's first searches
    must still start from empty slot tables.  Three sessions, with and without
    a time allowance, each result against the problem solved alone."""
    probs = mixed_problems()
    with rei.Context(device=0) as ctx:
        plain = [ctx.solve_problem(p) for p in probs]
        for rep in range(3):
            for yield_us in (0, 300):
                ctx.set_option(rei.REI_OPT_YIELD_US, yield_us)
                with rei.Server(ctx) as srv:
                    got = [srv.result(t) for t in [srv.submit(p) for p in probs]]
                for k, (a, b) in enumerate(zip(plain, got)):
                    assert key(a) == key(b), (rep, yield_us, k)
