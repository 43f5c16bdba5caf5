"""The batched form (rei_solve_batch): one staging launch and one persistent
search launch for many problems, each result exactly the one the plain entry
point (and, where it is fast enough, the oracle) gives."""
import pytest

import oracle
import paper_2305_18575_gb300 as rei
from workloads import make_config, type1_instance, type2_instance
from workloads.gen import batched_instance

from conftest import load_expected

pytestmark = pytest.mark.gpu

ST = {oracle.OK: rei.REI_OK, oracle.NOT_FOUND: rei.REI_NOT_FOUND, oracle.OOM: rei.REI_OOM}


def key(r):
    return (r.status, r.cost, r.tree, r.regex, r.candidates, r.unique)


def mixed_problems():
    probs = []
    for s in range(12):
        i = make_config("small", s)
        probs.append(rei.Problem(i.alphabet, i.pos, i.neg, costs=(1, 1, 1, 1, 1), max_cost=20))
    for s in range(10):
        i = make_config("medium", s)
        probs.append(rei.Problem(i.alphabet, i.pos, i.neg, costs=(1, 1, 5, 1, 1), max_cost=40,
                                 mem_budget=i.mem_budget))
    # the largest medium search caches ~844 K languages: more than a batch slot holds
    i = make_config("medium", 16)
    probs.append(rei.Problem(i.alphabet, i.pos, i.neg, costs=(1, 1, 5, 1, 1), max_cost=40, mem_budget=8 << 30))
    for s in range(6):
        i = batched_instance(s)
        probs.append(rei.Problem(i.alphabet, i.pos, i.neg, costs=(1, 1, 1, 1, 1), max_cost=40, mem_budget=1 << 30))
    for s in range(4):
        i = type2_instance(s, 4, 4, 5)
        probs.append(rei.Problem(i.alphabet, i.pos, i.neg, costs=(2, 1, 3, 1, 2), max_cost=30))
    # invalid ones in the middle: a foreign byte, P and N overlapping
    probs.insert(5, rei.Problem(b"01", [b"2"], [b""]))
    probs.insert(9, rei.Problem(b"01", [b"0"], [b"0"]))
    return probs


@pytest.mark.parametrize("warps", [8, 4])
def test_batch_matches_plain_solves(warps):
    probs = mixed_problems()
    with rei.Context(device=0) as ctx:
        plain = [ctx.solve_problem(p) for p in probs]
        batch = ctx.solve_batch(probs, warps_per_cta=warps)
        again = ctx.solve_batch(probs, warps_per_cta=warps)  # slots reused after a batch
    for k, (a, b, c) in enumerate(zip(plain, batch, again)):
        assert key(a) == key(b) == key(c), (k, a, b)
    assert batch[5].status == rei.REI_EINVAL and batch[9].status == rei.REI_EINVAL


def test_batch_matches_oracle_on_small_problems():
    insts = [make_config("small", s) for s in range(30)] + [type1_instance(s, 3, 3, 3) for s in range(6)]
    probs = [rei.Problem(i.alphabet, i.pos, i.neg, costs=(1, 2, 1, 2, 1), max_cost=20) for i in insts]
    with rei.Context(device=0) as ctx:
        got = ctx.solve_batch(probs)
    for i, g in zip(insts, got):
        ref = oracle.solve(i.alphabet, i.pos, i.neg, costs=(1, 2, 1, 2, 1), max_cost=20)
        assert (g.status, g.cost, g.tree, g.candidates, g.unique) == \
            (rei.REI_OK, ref.cost, ref.tree, ref.candidates, ref.unique)


def test_batch_config_matches_stored_oracle_results():
    """Every one of the 512 instances of the batched configuration, solved in
    one rei_solve_batch call with the autotuned launch shape: status, cost,
    tree, candidate and unique counts and |ic| equal the oracle's (stored by
    tests/golden/make_batched_expected.py, which calls only the oracle)."""
    want = load_expected("batched_expected.txt")
    assert sorted(want) == list(range(512))
    insts = [batched_instance(s) for s in range(512)]
    probs = [rei.Problem(i.alphabet, i.pos, i.neg, costs=(1, 1, 1, 1, 1), max_cost=40, mem_budget=1 << 30)
             for i in insts]
    with rei.Context(device=0) as ctx:
        batch = ctx.solve_batch(probs)
        for k in range(0, 512, 17):  # a sample against the plain path too
            assert key(ctx.solve_problem(probs[k])) == key(batch[k]), k
    for s, r in enumerate(batch):
        st, cost, cand, uniq, n_ic, tree = want[s]
        assert r.status == ST[st], s
        assert (r.cost, r.tree, r.candidates, r.unique, r.n_ic) == (cost, tree, cand, uniq, n_ic), s
    for i, r in zip(insts, batch):
        assert r.cost <= i.target_cost


@pytest.mark.parametrize("yield_us,chunk", [(1, 0), (50, 4096)])
def test_batch_config_parked_everywhere_matches_stored_oracle_results(yield_us, chunk):
    """The 512 batched instances with a time allowance so short that nearly
    every search parks on its CTA: more parked searches than the GPU has CTA
    pairs, so some continue in slot groups and the rest on helper contexts
    from their slots; every result still equals the oracle's."""
    want = load_expected("batched_expected.txt")
    insts = [batched_instance(s) for s in range(512)]
    probs = [rei.Problem(i.alphabet, i.pos, i.neg, costs=(1, 1, 1, 1, 1), max_cost=40, mem_budget=1 << 30)
             for i in insts]
    with rei.Context(device=0) as ctx:
        batch = ctx.solve_batch(probs, warps_per_cta=8, chunk=chunk, yield_us=yield_us)
    for s, r in enumerate(batch):
        st, cost, cand, uniq, n_ic, tree = want[s]
        assert r.status == ST[st], s
        assert (r.cost, r.tree, r.candidates, r.unique, r.n_ic) == (cost, tree, cand, uniq, n_ic), s


def test_batch_with_per_symbol_costs():
    insts = [make_config("small", s) for s in range(12)] + [batched_instance(s) for s in range(12)]
    probs = []
    for k, i in enumerate(insts):
        sc = [1 + (a * 3 + k) % 4 for a in range(len(i.alphabet))]
        probs.append(rei.Problem(i.alphabet, i.pos, i.neg, max_cost=40, mem_budget=1 << 30, sym_costs=sc))
    with rei.Context(device=0) as ctx:
        plain = [ctx.solve_problem(p) for p in probs]
        batch = ctx.solve_batch(probs)
    for k, (a, b) in enumerate(zip(plain, batch)):
        assert key(a) == key(b), k



@pytest.mark.parametrize("yield_us", [0, 1, 300])
def test_batch_time_allowance_does_not_change_results(yield_us):
    """A problem still searching on its CTA after yield_us gives up there and
    is solved again on the whole GPU (1 us: nearly all do; 0: none does)."""
    probs = mixed_problems()
    with rei.Context(device=0) as ctx:
        plain = [ctx.solve_problem(p) for p in probs]
        ctx.set_option(rei.REI_OPT_YIELD_US, yield_us)
        batch = ctx.solve_batch(probs)
    for k, (a, b) in enumerate(zip(plain, batch)):
        assert key(a) == key(b), (k, yield_us)


@pytest.mark.parametrize("warps,chunk,yield_us", [(8, 256, 0xFFFFFFFF), (4, 65536, 1), (2, 1000, 300),
                                                  (1, 4096, 0)])
def test_batch_tune_fields_do_not_change_results(warps, chunk, yield_us):
    """Every rei_tune field (warps per CTA, chunk in a slot, time allowance;
    0 = chosen by the library) leaves every result as the plain path gives it."""
    probs = mixed_problems()
    with rei.Context(device=0) as ctx:
        plain = [ctx.solve_problem(p) for p in probs]
        batch = ctx.solve_batch(probs, warps_per_cta=warps, chunk=chunk, yield_us=yield_us)
    for k, (a, b) in enumerate(zip(plain, batch)):
        assert key(a) == key(b), (k, warps, chunk, yield_us)


@pytest.mark.parametrize("bad", [dict(warps_per_cta=3), dict(warps_per_cta=16), dict(chunk=100),
                                 dict(chunk=1 << 17)])
def test_batch_tune_out_of_range(bad):
    probs = mixed_problems()[:3]
    with rei.Context(device=0) as ctx:
        with pytest.raises(RuntimeError):
            ctx.solve_batch(probs, **bad)
