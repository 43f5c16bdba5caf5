"""rei_solve_noalloc against the allocating entry point, rei_solve_problem.

rei_solve_noalloc is for callers that cannot allocate device memory while
they solve (code working inside another framework's fixed memory arena, or a
host thread that must not enter the CUDA allocator); it runs in one shared,
fixed device array instead.  Its results must be exactly the ones
rei_solve_problem gives for the same problem.  Each problem is solved twice
in a row, because the shared array keeps the previous call's contents and
each call must clear what has to start cleared.

This file is collected last on purpose, and passes alone in a fresh process
as well as after the other tests.
"""
import pytest

import paper_2305_18575_gb300 as rei
from workloads import make_config

pytestmark = pytest.mark.gpu

BUDGET = 32 << 20  # its whole cache (about 0.93 M languages at W = 2) fits the scratch
CASES = [("small", 3, (1, 1, 1, 1, 1)), ("medium", 2, (1, 1, 1, 1, 1)),
         ("medium", 5, (1, 1, 5, 1, 1)), ("medium", 16, (1, 1, 5, 1, 1)),
         ("medium", 12, (2, 1, 3, 1, 2)), ("wide", 0, (1, 1, 10, 1, 1))]


def noalloc(prob):
    buf = rei._OutBuf()
    s = rei.rei_solve_noalloc(prob.p, None, buf.res)
    return buf.result(s)


def key(r):
    return (r.status, r.cost, r.tree, r.regex, r.candidates, r.unique, r.levels, r.n_ic)


def test_noalloc_matches_the_allocating_entry_point_twice_in_a_row():
    with rei.Context(device=0) as ctx:
        for name, seed, costs in CASES:
            inst = make_config(name, seed)
            max_cost = 40 if name != "wide" else 6
            for budget in (BUDGET, 1 << 20):  # the second budget ends some searches in REI_OOM
                prob = rei.Problem(inst.alphabet, inst.pos, inst.neg, costs=costs, max_cost=max_cost,
                                   mem_budget=budget)
                ref = ctx.solve_problem(prob)
                assert ref.status in (rei.REI_OK, rei.REI_OOM, rei.REI_NOT_FOUND)
                for _ in range(2):
                    got = noalloc(prob)
                    assert key(got) == key(ref), (name, seed, costs, budget, got, ref)


def test_noalloc_reads_device_inputs():
    inst = make_config("medium", 5)
    with rei.Context(device=0) as ctx:
        host = ctx.solve_problem(rei.Problem(inst.alphabet, inst.pos, inst.neg, max_cost=40,
                                             mem_budget=BUDGET))
    dev = rei.Problem.on_device(inst.alphabet, inst.pos, inst.neg, max_cost=40, mem_budget=BUDGET)
    for _ in range(2):
        assert key(noalloc(dev)) == key(host)


def test_noalloc_refuses_what_does_not_fit():
    inst = make_config("medium", 2)
    prob = rei.Problem(inst.alphabet, inst.pos, inst.neg, max_cost=40, mem_budget=1 << 40)
    assert noalloc(prob).status == rei.REI_ESCRATCH
    # and keeps working afterwards
    prob = rei.Problem(inst.alphabet, inst.pos, inst.neg, max_cost=40, mem_budget=BUDGET)
    assert noalloc(prob).status == rei.REI_OK


def test_noalloc_with_per_symbol_costs():
    with rei.Context(device=0) as ctx:
        for seed in range(4):
            inst = make_config("small", seed)
            prob = rei.Problem(inst.alphabet, inst.pos, inst.neg, max_cost=30, mem_budget=BUDGET,
                               sym_costs=[1, 3])
            want = ctx.solve_problem(prob)
            assert key(noalloc(prob)) == key(want)



def test_noalloc_short_regex_buffer_is_terminated():
    """A regex buffer too small for the answer: REI_EBUFSZ, the full length
    written back, and the buffer cut at cap - 1 bytes and NUL terminated."""
    inst = make_config("medium", 5)
    prob = rei.Problem(inst.alphabet, inst.pos, inst.neg, max_cost=40, mem_budget=BUDGET)
    full = noalloc(prob)
    assert full.status == rei.REI_OK and len(full.regex.encode()) > 4
    buf = rei._OutBuf(regex_cap=4)
    buf.rbuf.raw = b"\xff" * 4
    s = rei.rei_solve_noalloc(prob.p, None, buf.res)
    assert s == rei.REI_EBUFSZ and buf.res.status == rei.REI_OK
    assert buf.res.regex_len == len(full.regex.encode())
    assert buf.rbuf.raw == full.regex.encode()[:3] + b"\x00"
