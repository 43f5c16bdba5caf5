"""Pins for the CPU oracle, against facts the paper and mathematics fix.

Nothing here compares the oracle with itself: every expected value is printed
in the paper (tests/golden), a closed form or invariant, an independent
implementation (brute force over syntax trees; the generator's Thompson NFA;
Python set comprehensions for substrings), or a special case with a known
answer.  A final test plants mistakes in the oracle and shows each one fails a
pin.
"""
import random

import pytest

import oracle
from workloads import make_config, type1_instance, type2_instance
from workloads.gen import _Nfa, random_tree, _buildable

A01 = b"01"


def substrings(strings):
    return {s[i:j] for s in strings for i in range(len(s) + 1) for j in range(i, len(s) + 1)}


def shortlex_key(alphabet):
    rank = {c: i for i, c in enumerate(alphabet)}
    return lambda w: (len(w), [rank[c] for c in w])


def tree_tokens(t, out=None):
    """generator tree -> postfix tokens (2 bytes each)."""
    out = bytearray() if out is None else out
    op = t[0]
    if op == "a":
        out += bytes([ord("a"), t[1]])
    else:
        for sub in t[1:]:
            tree_tokens(sub, out)
        out += bytes([ord(op), 0])
    return bytes(out)


# ---------------------------------------------------------------------------
# infix closure and order (Sec. 2 definitions, Example 1, figure walkthrough)

def test_example1_ic_matches_paper(golden):
    g = golden("example1_ic.txt")
    P = [b"1", b"011", b"1011", b"11011"]
    N = [b"", b"10", b"101", b"0011"]
    ic = oracle.ic(A01, P + N)
    assert set(ic) == set(g["words"]) and len(ic) == 15
    for row in g["rows"]:
        if row[0] == "index":
            assert ic.index(row[1].encode()) == int(row[2])
        if row[0] == "pair":
            w, u, v = (x.encode() for x in row[1:])
            assert u + v == w and u in ic and v in ic


@pytest.mark.parametrize("seed", range(12))
def test_ic_is_sorted_infix_closure(seed):
    rng = random.Random(seed)
    alpha = [b"01", b"abc", b"xyzw"][seed % 3]
    strings = [bytes(rng.choice(alpha) for _ in range(rng.randint(0, 7))) for _ in range(rng.randint(1, 9))]
    ic = oracle.ic(alpha, strings)
    assert set(ic) == substrings(strings)          # smallest infix-closed superset
    assert len(ic) == len(set(ic))
    assert ic == sorted(ic, key=shortlex_key(alpha))
    assert ic[0] == b""
    for w in ic:                                     # infix-closed
        for i in range(len(w) + 1):
            for j in range(i, len(w) + 1):
                assert w[i:j] in ic


# ---------------------------------------------------------------------------
# languages on ic: Example 1, the derivative matcher, semiring laws

def test_example1_language_of_0q1star1(golden):
    g = golden("example1_ic.txt")
    P = [b"1", b"011", b"1011", b"11011"]
    N = [b"", b"10", b"101", b"0011"]
    ic = oracle.ic(A01, P + N)
    t = oracle.parse("(0?1)*1", A01)
    lang = oracle.tree_lang(t, A01, P + N)
    got = {ic[i] for i in range(len(ic)) if lang[i]}
    assert got == set(g["lang"]["(0?1)*1"])
    for w in ic:                                     # same set via derivatives
        assert oracle.match(t, A01, w) == (w in got)


@pytest.mark.parametrize("seed", range(40))
def test_matcher_agrees_with_thompson_nfa(seed):
    """Derivative matcher vs the generator's independent NFA simulation."""
    rng = random.Random(1000 + seed)
    k = rng.randint(2, 3)
    alpha = b"abc"[:k]
    costs = (1, 1, 1, 1, 1)
    t = random_tree(rng, rng.randint(1, 9), costs, k, _buildable(costs, 9))
    nfa = _Nfa(t, alpha)
    tok = tree_tokens(t)
    for _ in range(60):
        s = bytes(rng.choice(alpha) for _ in range(rng.randint(0, 7)))
        assert oracle.match(tok, alpha, s) == nfa.fullmatch(s)


@pytest.mark.parametrize("seed", range(40))
def test_ips_language_equals_matching_on_ic(seed):
    """On an infix-closed domain, the set operations of Sec. 3 compute exactly
    L(r) restricted to ic (the paper's reason for using ic)."""
    rng = random.Random(2000 + seed)
    alpha = b"01" if seed % 2 else b"abc"
    costs = (1, 1, 1, 1, 1)
    t = random_tree(rng, rng.randint(1, 11), costs, len(alpha), _buildable(costs, 11))
    tok = tree_tokens(t)
    strings = [bytes(rng.choice(alpha) for _ in range(rng.randint(0, 6))) for _ in range(6)]
    ic = oracle.ic(alpha, strings)
    lang = oracle.tree_lang(tok, alpha, strings)
    nfa = _Nfa(t, alpha)
    for i, w in enumerate(ic):
        assert bool(lang[i]) == nfa.fullmatch(w) == oracle.match(tok, alpha, w)


@pytest.mark.parametrize("seed", range(10))
def test_semiring_laws_on_ic(seed):
    rng = random.Random(3000 + seed)
    costs = (1, 1, 1, 1, 1)
    ok = _buildable(costs, 7)
    r, s, u = (tree_tokens(random_tree(rng, rng.randint(1, 6), costs, 2, ok)) for _ in range(3))
    strings = [bytes(rng.choice(A01) for _ in range(rng.randint(0, 6))) for _ in range(5)]
    L = lambda tok: oracle.tree_lang(tok, A01, strings)
    cat = lambda x, y: x + y + b".\x00"
    alt = lambda x, y: x + y + b"+\x00"
    star = lambda x: x + b"*\x00"
    eps = b"e\x00"
    assert L(cat(cat(r, s), u)) == L(cat(r, cat(s, u)))            # associativity
    assert L(cat(alt(r, s), u)) == L(alt(cat(r, u), cat(s, u)))    # distributivity
    assert L(cat(u, alt(r, s))) == L(alt(cat(u, r), cat(u, s)))
    assert L(alt(r, s)) == L(alt(s, r))
    assert L(star(r)) == L(alt(eps, cat(r, star(r))))              # r* = 1 + r r*
    assert L(star(r)) == L(star(star(r)))
    assert L(r + b"?\x00") == L(alt(eps, r))                        # r? = eps + r
    assert L(star(r))[0] == 1                                        # eps in r*


# ---------------------------------------------------------------------------
# cost homomorphism and the printed table (Sec. 3 definition; Sec. 6 table)

def test_printed_table_costs_and_precision(golden):
    g = golden("allowed_error_table.txt")
    P, N = g["P"], g["N"]
    for row in g["rows"]:
        pct, text, cost = int(row[1]), row[2], int(row[3])
        tok = oracle.parse(text, A01)
        assert oracle.tree_cost(tok, (1, 1, 1, 1, 1)) == cost
        errs = sum(not oracle.match(tok, A01, p) for p in P) + sum(oracle.match(tok, A01, q) for q in N)
        assert errs <= pct * (len(P) + len(N)) // 100


def test_cost_homomorphism_weights():
    tok = oracle.parse("10?+0?(00+10*10?(0+1))1?", A01)
    # 12 symbols, 4 "?", 1 "*", 8 concatenations, 3 unions: 12+4+1+8+3 = 28
    assert oracle.tree_cost(tok, (1, 0, 0, 0, 0)) == 12
    assert oracle.tree_cost(tok, (0, 1, 0, 0, 0)) == 4
    assert oracle.tree_cost(tok, (0, 0, 1, 0, 0)) == 1
    assert oracle.tree_cost(tok, (0, 0, 0, 1, 0)) == 8
    assert oracle.tree_cost(tok, (0, 0, 0, 0, 1)) == 3


# ---------------------------------------------------------------------------
# the search: worked examples, brute force, special cases

def test_example1_minimal_regex():
    P = [b"1", b"011", b"1011", b"11011"]
    N = [b"", b"10", b"101", b"0011"]
    r = oracle.solve(A01, P, N, max_cost=12, flags=oracle.F_SELFCHECK)
    bc, _ = oracle.brute_min_cost(A01, P, N, max_cost=8)
    assert r.status == oracle.OK and r.cost == bc == 7
    assert r.text == "(0?1)*1"


def test_intro_example_minimal_regex(golden):
    g = golden("intro_example.txt")
    r = oracle.solve(A01, g["P"], g["N"], max_cost=12, flags=oracle.F_SELFCHECK)
    bc, _ = oracle.brute_min_cost(A01, g["P"], g["N"], max_cost=9)
    assert r.status == oracle.OK and r.cost == bc == 8
    assert r.text == "10(0+1)*"


@pytest.mark.parametrize("pct", [50, 45, 40, 35, 30, 25, 20, 15])
def test_allowed_error_rows(golden, pct):
    """Sec. 6 table: minimal cost per allowed error on the printed spec.  The
    regular expressions printed there also coincide with this oracle's fixed
    enumeration order on every row it can reach in seconds."""
    g = golden("allowed_error_table.txt")
    P, N = g["P"], g["N"]
    row = next(r for r in g["rows"] if int(r[1]) == pct)
    r = oracle.solve(A01, P, N, max_cost=30, max_errors=pct * (len(P) + len(N)) // 100)
    assert r.status == oracle.OK and r.cost == int(row[3])
    printed = row[2].replace("#", "∅")
    assert r.text == printed


COST_VECTORS = [(1, 1, 1, 1, 1), (1, 10, 1, 1, 1), (1, 1, 10, 1, 1), (1, 1, 1, 10, 1),
                (1, 1, 1, 1, 10), (2, 1, 3, 1, 2), (3, 2, 1, 2, 1)]


def _tiny_instances():
    out = []
    for s in range(8):
        out.append(make_config("small", s))
    for s in range(4):
        out.append(type1_instance(s, 3, 3, 3))
        out.append(type2_instance(s, 3, 3, 4))
    return out


@pytest.mark.parametrize("costs", COST_VECTORS)
def test_search_minimal_cost_equals_brute_force(costs):
    for inst in _tiny_instances():
        r = oracle.solve(inst.alphabet, inst.pos, inst.neg, costs=costs, max_cost=30,
                         flags=oracle.F_SELFCHECK)
        assert r.status == oracle.OK
        limit = r.cost if r.cost <= 9 * min(costs) else 0
        if not limit:
            continue
        bc, _ = oracle.brute_min_cost(inst.alphabet, inst.pos, inst.neg, costs=costs,
                                      max_cost=limit, node_limit=4_000_000)
        if bc < 0:
            continue
        assert bc == r.cost, (inst.seed, costs, r.text)
        # the answer is precise and its recomputed cost is the level
        assert oracle.tree_cost(r.tree, costs) == r.cost
        assert all(oracle.match(r.tree, inst.alphabet, p) for p in inst.pos)
        assert not any(oracle.match(r.tree, inst.alphabet, q) for q in inst.neg)


SYM_COSTS = [((1, 1, 1, 1, 1), [1, 3]), ((1, 1, 1, 1, 1), [4, 1]), ((2, 1, 3, 1, 2), [2, 5]),
             ((3, 2, 1, 2, 1), [1, 2]), ((5, 1, 1, 1, 1), [2, 2])]


@pytest.mark.parametrize("costs,sym", SYM_COSTS)
def test_per_symbol_costs_minimal_cost_equals_brute_force(costs, sym):
    """Different costs for different symbols (the remark after the cost
    function's definition, Sec. 3): the search's cost is the brute force's."""
    insts = _tiny_instances() + [type1_instance(s, 3, 3, 3, alphabet=b"abc") for s in range(3)]
    for inst in insts:
        sc = (sym + [3])[:len(inst.alphabet)]
        r = oracle.solve(inst.alphabet, inst.pos, inst.neg, costs=costs, max_cost=40, sym_costs=sc,
                         flags=oracle.F_SELFCHECK)
        assert r.status == oracle.OK
        assert oracle.tree_cost(r.tree, costs, sc) == r.cost
        assert all(oracle.match(r.tree, inst.alphabet, p) for p in inst.pos)
        assert not any(oracle.match(r.tree, inst.alphabet, q) for q in inst.neg)
        if r.cost > 12:
            continue
        bc, _ = oracle.brute_min_cost(inst.alphabet, inst.pos, inst.neg, costs=costs, max_cost=r.cost,
                                      node_limit=4_000_000, sym_costs=sc)
        if bc < 0:
            continue
        assert bc == r.cost, (inst.seed, costs, sc, r.text)


def test_uniform_symbol_costs_are_the_plain_homomorphism():
    for inst in _tiny_instances():
        for costs in [(1, 1, 1, 1, 1), (2, 1, 3, 1, 2)]:
            a = oracle.solve(inst.alphabet, inst.pos, inst.neg, costs=costs, max_cost=30)
            b = oracle.solve(inst.alphabet, inst.pos, inst.neg, costs=costs, max_cost=30,
                             sym_costs=[costs[0]] * len(inst.alphabet))
            assert (a.status, a.cost, a.tree, a.candidates, a.unique) == \
                (b.status, b.cost, b.tree, b.candidates, b.unique)


def test_symbol_costs_change_the_answer():
    # only the symbol 1 separates the sides; it costs 7, so no answer up to 6
    r = oracle.solve(A01, [b"1"], [b"", b"0"], max_cost=20, sym_costs=[1, 7])
    assert (r.cost, r.text) == (7, "1")
    r = oracle.solve(A01, [b"1"], [b"", b"0"], max_cost=6, sym_costs=[1, 7])
    assert r.status == oracle.NOT_FOUND
    # eps and the empty set keep c_sym
    r = oracle.solve(A01, [b""], [b"0"], costs=(5, 1, 1, 1, 1), max_cost=20, sym_costs=[1, 1])
    assert (r.cost, r.text) == (5, "ε")
    # an invalid symbol cost
    r = oracle.solve(A01, [b"1"], [b"0"], max_cost=20, sym_costs=[1, 0])
    assert r.status == oracle.EINVAL


def test_upper_bound_by_target_cost():
    for s in range(6):
        inst = make_config("medium", s)
        r = oracle.solve(inst.alphabet, inst.pos, inst.neg, max_cost=40, max_candidates=3_000_000)
        if r.status == oracle.OK:
            assert r.cost <= inst.target_cost


def test_questions_come_before_stars():
    r = oracle.solve(A01, [b"", b"0"], [b"1"], max_cost=6)
    assert r.status == oracle.OK and r.cost == 2 and r.text == "0?"


def test_trivial_and_special_cases():
    # P empty -> empty set; P = {eps} -> eps (Alg. 1), both at cost c1
    r = oracle.solve(A01, [], [b"0"], costs=(3, 1, 1, 1, 1))
    assert r.status == oracle.OK and r.cost == 3 and r.text == "∅"
    r = oracle.solve(A01, [b""], [b"0", b"1"], costs=(3, 1, 1, 1, 1))
    assert r.status == oracle.OK and r.cost == 3 and r.text == "ε"
    # one symbol separates P from N -> that symbol at cost c1
    r = oracle.solve(b"abc", [b"b"], [b"a", b"c", b""])
    assert r.status == oracle.OK and r.cost == 1 and r.text == "b"
    # max cost too small -> not found; tiny budget -> out of memory
    r = oracle.solve(A01, [b"0110", b"1"], [b"", b"01", b"11"], max_cost=3)
    assert r.status == oracle.NOT_FOUND
    r = oracle.solve(A01, [b"0110", b"1"], [b"", b"01", b"11"], max_cost=30, mem_budget=64)
    assert r.status == oracle.OOM
    # invalid inputs
    assert oracle.solve(b"00", [b"0"], [b""]).status == oracle.EINVAL     # repeated symbol
    assert oracle.solve(A01, [b"2"], [b""]).status == oracle.EINVAL       # foreign symbol
    assert oracle.solve(A01, [b"0"], [b"0"]).status == oracle.EINVAL      # P and N overlap
    assert oracle.solve(A01, [b"0"], [b""], costs=(1, 0, 1, 1, 1)).status == oracle.EINVAL


def test_star_free_fragment_with_expensive_star():
    for s in range(6):
        inst = make_config("small", s)
        r = oracle.solve(inst.alphabet, inst.pos, inst.neg, costs=(1, 1, 200, 1, 1), max_cost=60)
        assert r.status == oracle.OK and "*" not in r.text


def test_onthefly_keeps_the_answer():
    """OnTheFly (Sec. 3) continues from cached levels without caching; with a
    budget that fills the cache early it must still return the same answer
    whenever it returns one."""
    agree = 0
    for s in range(8):
        inst = make_config("small", s)
        for costs in [(1, 1, 1, 1, 1), (1, 2, 3, 3, 3), (1, 3, 3, 4, 4)]:
            ref = oracle.solve(inst.alphabet, inst.pos, inst.neg, costs=costs, max_cost=30)
            n = ref.n_ic
            per = 4 * (1 if n <= 32 else 2 if n <= 64 else 4 * ((n + 127) // 128)) + 28
            for cap in (3, 6, 12):
                r = oracle.solve(inst.alphabet, inst.pos, inst.neg, costs=costs, max_cost=30,
                                 mem_budget=cap * per, flags=oracle.F_ONTHEFLY)
                if r.status == oracle.OK:
                    agree += 1
                    assert (r.cost, r.tree) == (ref.cost, ref.tree)
                else:
                    assert r.status == oracle.OOM
    assert agree > 0


def test_level_order_and_uniqueness_of_cache():
    inst = make_config("medium", 2)
    run = oracle.Run()
    r = run.solve(inst.alphabet, inst.pos, inst.neg, max_cost=40, flags=oracle.F_SELFCHECK)
    assert r.status == oracle.OK
    n = r.n_ic
    seen = set()
    for k in range(run.cache_size()):
        lang, op, l, rr = run.cache_entry(k, n)
        assert lang not in seen                       # every cached language is new
        seen.add(lang)
    # levels are contiguous, ordered by cost, operands come from lower levels
    prev_end = 0
    for c in range(1, r.cost):
        st, cnt = run.level(c)
        assert st == prev_end
        prev_end = st + cnt
        for k in range(st, st + cnt):
            _, op, l, rr = run.cache_entry(k, n)
            if op in (1, 2, 3, 4):
                assert l < st and (rr < st if op in (3, 4) else rr == -1)
    assert r.unique == prev_end


# ---------------------------------------------------------------------------
# the pins have teeth: each planted mistake fails at least one of them

def _pins_pass():
    checks = []
    try:
        test_example1_language_of_0q1star1(__import__("conftest").load_golden)
        checks.append(True)
    except AssertionError:
        checks.append(False)
    P = [b"1", b"011", b"1011", b"11011"]
    N = [b"", b"10", b"101", b"0011"]
    r = oracle.solve(A01, P, N, max_cost=12)
    checks.append(r.status == oracle.OK and r.cost == 7 and r.text == "(0?1)*1")
    checks.append(oracle.ic(A01, [b"01", b"10"]) == [b"", b"0", b"1", b"01", b"10"])
    # Alg. 1 builds questions before stars: 0? and 0* both denote {eps, 0} on
    # ic = {eps, 0, 1}, so the question must be returned
    r = oracle.solve(A01, [b"", b"0"], [b"1"], max_cost=6)
    checks.append(r.text == "0?")
    g = __import__("conftest").load_golden("allowed_error_table.txt")
    for pct, cost, text in [(20, 12, "(0+11)*(1+00)"), (35, 7, "1+(0+1)0")]:
        r = oracle.solve(A01, g["P"], g["N"], max_cost=30, max_errors=pct * 22 // 100)
        checks.append(r.cost == cost and r.text == text)
    # per-symbol costs: the only precise symbol costs 7; with symbols at cost 1
    # and c_sym = 3, the answer must use them as operands (brute force: cost 4)
    r = oracle.solve(A01, [b"1"], [b"", b"0"], max_cost=20, sym_costs=[1, 7])
    checks.append(r.cost == 7 and r.text == "1")
    r = oracle.solve(A01, [b"1", b"11"], [b"", b"0"], costs=(3, 1, 1, 1, 1), max_cost=20, sym_costs=[1, 1])
    checks.append(r.cost == oracle.brute_min_cost(A01, [b"1", b"11"], [b"", b"0"], costs=(3, 1, 1, 1, 1),
                                                  max_cost=8, sym_costs=[1, 1])[0] == 4)
    return all(checks)


@pytest.mark.parametrize("mutation", range(1, 10))
def test_planted_mistakes_are_caught(mutation):
    assert _pins_pass()
    oracle.set_mutation(mutation)
    try:
        assert not _pins_pass(), f"mutation {mutation} escaped the pins"
    finally:
        oracle.set_mutation(0)
    assert _pins_pass()
