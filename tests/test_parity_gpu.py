"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer work, so the bar is bit-exactness: the same status, minimal cost,
expression tree (postfix tokens), candidate and unique counts, and, where the
cache is dumped, the same languages in the same order with the same
back-pointers.
"""
import random

import pytest

import oracle
import paper_2305_18575_gb300 as rei
from workloads import make_config, type1_instance, type2_instance

pytestmark = pytest.mark.gpu

A01 = b"01"
EX1 = ([b"1", b"011", b"1011", b"11011"], [b"", b"10", b"101", b"0011"])
PIN_P = [b"00", b"1101", b"0001", b"0111", b"001", b"1", b"10", b"1100", b"111", b"1010"]
PIN_N = [b"", b"0", b"0000", b"0011", b"01", b"010", b"011", b"100", b"1000", b"1001", b"11", b"1110"]
COSTS = [(1, 1, 1, 1, 1), (1, 1, 5, 1, 1), (1, 10, 1, 1, 1), (1, 1, 1, 10, 1), (1, 1, 1, 1, 10),
         (2, 1, 3, 1, 2), (3, 2, 1, 2, 1), (10, 10, 10, 1, 10)]
ST = {oracle.OK: rei.REI_OK, oracle.NOT_FOUND: rei.REI_NOT_FOUND, oracle.OOM: rei.REI_OOM,
      oracle.EINVAL: rei.REI_EINVAL}


@pytest.fixture(scope="module")
def ctx():
    c = rei.Context(device=0)
    yield c
    c.close()


def check_same(got, ref, what=""):
    assert got.status == ST[ref.status], (what, got, ref)
    if ref.status == oracle.OK:
        assert got.cost == ref.cost, (what, got.regex, ref.text)
        assert got.tree == ref.tree, (what, got.regex, ref.text)
        assert got.regex == ref.text, what
    assert got.candidates == ref.candidates, (what, got.candidates, ref.candidates)
    assert got.unique == ref.unique, (what, got.unique, ref.unique)


def solve_both(ctx, inst_or_abc, pos=None, neg=None, **kw):
    if pos is None:
        alpha, pos, neg = inst_or_abc.alphabet, inst_or_abc.pos, inst_or_abc.neg
    else:
        alpha = inst_or_abc
    flags = kw.pop("flags", 0)
    ref = oracle.solve(alpha, pos, neg, flags=(oracle.F_ONTHEFLY if flags & rei.REI_F_ONTHEFLY else 0), **kw)
    prob = rei.Problem(alpha, pos, neg, flags=flags, **kw)
    got = ctx.solve_problem(prob)
    return got, ref


# ---------------------------------------------------------------------------
# staging (ic, guide table, masks, leaves)

def _stage_cases():
    cases = [("ex1", A01, *EX1), ("pin", A01, PIN_P, PIN_N)]
    for s in range(3):
        i = make_config("small", s)
        cases.append((f"small{s}", i.alphabet, i.pos, i.neg))
        i = make_config("medium", s)
        cases.append((f"medium{s}", i.alphabet, i.pos, i.neg))
    i = make_config("wide", 0)
    cases.append(("wide0", i.alphabet, i.pos, i.neg))
    rng = random.Random(5)
    cases.append(("rand", b"xyz", [bytes(rng.choice(b"xyz") for _ in range(rng.randint(0, 30))) for _ in range(6)],
                  [bytes(rng.choice(b"xyz") for _ in range(rng.randint(0, 30))) for _ in range(6)]))
    return cases


@pytest.mark.parametrize("case", _stage_cases(), ids=lambda c: c[0])
def test_stage_matches_oracle(ctx, case):
    _, alpha, pos, neg = case
    neg = [s for s in neg if s not in set(pos)]
    prob = rei.Problem(alpha, pos, neg)
    s, g = ctx.stage(prob)
    assert s == rei.REI_OK
    buf = b"".join(pos + neg)
    words = [buf[g["word_start"][w]: g["word_start"][w] + g["word_len"][w]] for w in range(g["n"])]
    ic = oracle.ic(alpha, pos + neg)
    assert words == ic                                  # same words, same shortlex order
    index = {w: i for i, w in enumerate(ic)}
    assert g["G"] == sum(len(w) + 1 for w in ic)        # |gt[w]| = |w| + 1
    for w, word in enumerate(ic):
        lo, hi = g["gt_off"][w], g["gt_off"][w + 1]
        assert hi - lo == len(word) + 1
        for k in range(len(word) + 1):
            pr = g["gt_pair"][lo + k]
            assert (pr & 0xFFFF, pr >> 16) == (index[word[:k]], index[word[k:]])
    W = g["W"]
    bits = lambda ws: {32 * b + t for b in range(W) for t in range(32) if ws[b] >> t & 1}
    assert bits(g["pos"]) == {index[p] for p in pos}
    assert bits(g["neg"]) == {index[q] for q in neg}
    for a, sym in enumerate(alpha):
        want = {index[bytes([sym])]} if bytes([sym]) in index else set()
        assert bits(g["leaf"][a]) == want


# ---------------------------------------------------------------------------
# whole solves

@pytest.mark.parametrize("costs", COSTS)
def test_small_config_matches_oracle(ctx, costs):
    for s in range(30):
        inst = make_config("small", s)
        got, ref = solve_both(ctx, inst, costs=costs, max_cost=20)
        check_same(got, ref, f"small{s} {costs}")


def test_paper_examples(ctx, golden):
    got, ref = solve_both(ctx, A01, *EX1, max_cost=12)
    check_same(got, ref)
    assert got.regex == "(0?1)*1" and got.cost == 7
    g = golden("intro_example.txt")
    got, ref = solve_both(ctx, A01, g["P"], g["N"], max_cost=12)
    check_same(got, ref)
    assert got.regex == "10(0+1)*"


@pytest.mark.parametrize("pct", [50, 45, 40, 35, 30, 25, 20, 15])
def test_allowed_error_rows_match_oracle_and_paper(ctx, golden, pct):
    g = golden("allowed_error_table.txt")
    row = next(r for r in g["rows"] if int(r[1]) == pct)
    e = pct * 22 // 100
    got, ref = solve_both(ctx, A01, PIN_P, PIN_N, max_cost=30, max_errors=e)
    check_same(got, ref, pct)
    assert got.cost == int(row[3])


@pytest.mark.parametrize("seed", range(20))
@pytest.mark.parametrize("costs", [(1, 1, 1, 1, 1), (1, 1, 5, 1, 1)])
def test_medium_config_matches_oracle(ctx, seed, costs):
    inst = make_config("medium", seed)
    ref = oracle.solve(inst.alphabet, inst.pos, inst.neg, costs=costs, max_cost=40,
                       max_candidates=2_000_000)
    got = ctx.solve_problem(rei.Problem(inst.alphabet, inst.pos, inst.neg, costs=costs, max_cost=40,
                                        mem_budget=inst.mem_budget))
    if ref.status == oracle.LIMIT:
        # beyond the oracle's budget here: check what holds at any size
        assert got.status == rei.REI_OK and got.cost <= inst.target_cost + 4 * (costs[2] - 1)
        assert oracle.tree_cost(got.tree, costs) == got.cost
        assert all(oracle.match(got.tree, inst.alphabet, p) for p in inst.pos)
        assert not any(oracle.match(got.tree, inst.alphabet, q) for q in inst.neg)
        assert got.candidates > ref.candidates
        return
    check_same(got, ref, f"medium{seed} {costs}")


def _wide_expected():
    import os
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "wide_expected.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            sd, st, cost, cand, uniq, n_ic, tree = line.split()
            rows.append((int(sd), int(st), int(cost), int(cand), int(uniq), int(n_ic), bytes.fromhex(tree)))
    return rows


@pytest.mark.parametrize("fused", [1, 0])
def test_wide_config_matches_stored_oracle_results(fused):
    """The wide configuration at full size (|ic| 400-480, 16-word languages):
    every seed's answer, tree and counts equal the oracle's (stored by
    tests/golden/make_wide_expected.py, which calls only the oracle)."""
    with rei.Context(device=0) as c:
        c.set_option(rei.REI_OPT_FUSED_STAGE, fused)
        for sd, st, cost, cand, uniq, n_ic, tree in _wide_expected():
            inst = make_config("wide", sd)
            got = c.solve_problem(rei.Problem(inst.alphabet, inst.pos, inst.neg, max_cost=40,
                                              mem_budget=inst.mem_budget))
            assert got.status == ST[st], sd
            assert (got.cost, got.tree, got.candidates, got.unique, got.n_ic) == (cost, tree, cand, uniq, n_ic), sd


def _wide_large_expected():
    import os
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "wide_large_expected.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            var, sd, st, cost, cand, uniq, n_ic, tree = line.split()
            rows.append((var, int(sd), int(st), int(cost), int(cand), int(uniq), int(n_ic), bytes.fromhex(tree)))
    return rows


@pytest.mark.parametrize("fused", [1, 0])
def test_wide_large_ic_matches_stored_oracle_results(fused):
    """Wide instances with |ic| 1000-1500 (36- and 48-word languages) at their
    full minimal cost: answer, tree and counts equal the oracle's (stored by
    tests/golden/make_wide_large_expected.py, which calls only the oracle)."""
    from workloads import wide_large_instance
    rows = _wide_large_expected()
    assert {r[6] for r in rows} and max(r[6] for r in rows) > 1408
    with rei.Context(device=0) as c:
        c.set_option(rei.REI_OPT_FUSED_STAGE, fused)
        for var, sd, st, cost, cand, uniq, n_ic, tree in rows:
            inst = wide_large_instance(var, sd)
            got = c.solve_problem(rei.Problem(inst.alphabet, inst.pos, inst.neg, max_cost=40,
                                              mem_budget=inst.mem_budget))
            assert got.status == ST[st], (var, sd)
            assert (got.cost, got.tree, got.candidates, got.unique, got.n_ic) == (cost, tree, cand, uniq, n_ic), \
                (var, sd)
            assert got.words == 4 * ((n_ic + 127) // 128)  # 36 or 48 words


@pytest.mark.parametrize("chunk", [1, 7, 100, 4099])
@pytest.mark.parametrize("grid", [1, 3, 0])
@pytest.mark.parametrize("solo", [-1, 0, 1 << 30])
def test_chunking_and_grid_do_not_change_results(chunk, grid, solo):
    """Small chunks split every level into many chunks with ragged tails; a
    small grid makes every CTA process many tiles; `solo` forces every chunk
    onto the whole grid (0) or onto CTA 0 alone (2^30)."""
    with rei.Context(device=0) as c:
        c.set_option(rei.REI_OPT_CHUNK, chunk)
        c.set_option(rei.REI_OPT_GRID, grid)
        c.set_option(rei.REI_OPT_SOLO_TILES, solo)
        for s in (0, 2, 5):
            inst = make_config("medium", s)
            got, ref = solve_both(c, inst, max_cost=40, mem_budget=1 << 30)
            check_same(got, ref, (s, chunk, grid))
        got, ref = solve_both(c, A01, PIN_P, PIN_N, max_cost=30, max_errors=4)
        check_same(got, ref, ("pin20", chunk, grid))


_ORACLE = {}


def oracle_medium(seed, costs):
    key = (seed, costs)
    if key not in _ORACLE:
        inst = make_config("medium", seed)
        _ORACLE[key] = (inst, oracle.solve(inst.alphabet, inst.pos, inst.neg, costs=costs, max_cost=40))
    return _ORACLE[key]


@pytest.mark.parametrize("small", [0, 256, 1024, -1])
@pytest.mark.parametrize("chunk,solo", [(0, -1), (7, -1), (100, 1 << 30)])
def test_shared_memory_start_does_not_change_results(small, chunk, solo):
    """The search's start with its languages and uniqueness table in CTA 0's
    shared memory (`small` rows: 0 = never, 256 = leaves it after a few
    levels, -1 = as many as fit) gives the oracle's results, through the move
    to the global table in the middle of a search, with chunks split small
    and with every chunk on CTA 0 alone."""
    with rei.Context(device=0) as c:
        c.set_option(rei.REI_OPT_SMALL_ROWS, small)
        c.set_option(rei.REI_OPT_CHUNK, chunk)
        c.set_option(rei.REI_OPT_SOLO_TILES, solo)
        for s in (0, 2, 5, 12):
            for costs in [(1, 1, 1, 1, 1), (1, 1, 5, 1, 1)]:
                inst, ref = oracle_medium(s, costs)
                got = c.solve_problem(rei.Problem(inst.alphabet, inst.pos, inst.neg, costs=costs, max_cost=40,
                                                  mem_budget=inst.mem_budget))
                check_same(got, ref, (s, costs, small, chunk))
        got, ref = solve_both(c, A01, PIN_P, PIN_N, max_cost=30, max_errors=4)
        check_same(got, ref, ("pin20", small, chunk))
        # budgets that fill the cache while it is still in shared memory
        P, N = [b"0110", b"1"], [b"", b"01", b"11"]
        for budget in (64, 400, 2000, 9000):
            got, ref = solve_both(c, A01, P, N, max_cost=30, mem_budget=budget)
            check_same(got, ref, (budget, small))
        for rows in (3, 6, 12):
            inst = make_config("small", rows)
            got, ref = solve_both(c, inst, costs=(1, 2, 3, 3, 3), max_cost=30, mem_budget=rows * 32,
                                  flags=rei.REI_F_ONTHEFLY)
            check_same(got, ref, ("otf", rows, small))


def test_shared_memory_start_with_cache_growth():
    """A tiny first cache makes the search ask for more memory while its
    languages are still in shared memory: they move to the global table
    before the relaunch."""
    with rei.Context(device=0) as c:
        c.set_option(rei.REI_OPT_CACHE_INIT, 8)
        c.set_option(rei.REI_OPT_SMALL_ROWS, 4096)
        for s in (2, 5, 16):
            inst = make_config("medium", s)
            got, ref = solve_both(c, inst, max_cost=40, costs=(1, 1, 1, 1, 1))
            check_same(got, ref, s)
            assert got.launches > 2


def test_small_rows_option_checked():
    with rei.Context(device=0) as c:
        for bad in (1, 100, 255, 300, 32768):
            with pytest.raises(ValueError):
                c.set_option(rei.REI_OPT_SMALL_ROWS, bad)


@pytest.mark.parametrize("fused", [0, 1])
def test_fused_and_separate_staging_agree(fused):
    """Staging inside the search launch (1) or in its own launch (0): the same
    results, including a problem too large for the fused launch's staging
    (|ic| = 3538 > 2048), which goes through the separate staging launch."""
    with rei.Context(device=0) as c:
        c.set_option(rei.REI_OPT_FUSED_STAGE, fused)
        for s in (0, 3, 12):
            for costs in [(1, 1, 1, 1, 1), (1, 1, 5, 1, 1)]:
                inst, ref = oracle_medium(s, costs)
                got = c.solve_problem(rei.Problem(inst.alphabet, inst.pos, inst.neg, costs=costs, max_cost=40,
                                                  mem_budget=inst.mem_budget))
                check_same(got, ref, (s, costs, fused))
        for s in range(6):
            got, ref = solve_both(c, make_config("small", s), max_cost=20)
            check_same(got, ref, ("small", s))
        got, ref = solve_both(c, A01, *EX1, max_cost=12)
        check_same(got, ref, "ex1")
        rng = random.Random(0)
        pos = list({bytes(rng.choice(b"abcd") for _ in range(rng.randint(20, 34))) for _ in range(6)})
        neg = list({bytes(rng.choice(b"abcd") for _ in range(rng.randint(20, 34))) for _ in range(6)} - set(pos))
        got, ref = solve_both(c, b"abcd", pos, neg, max_cost=3)
        assert got.n_ic == 3538
        check_same(got, ref, "ic3538")
        assert c.solve(A01, [b"2"], [b""]).status == rei.REI_EINVAL
        assert c.solve(A01, [b"0"], [b"0"]).status == rei.REI_EINVAL


@pytest.mark.parametrize("exact", [0, 1])
@pytest.mark.parametrize("chunk,solo,small", [(0, -1, -1), (7, -1, 0), (0, 0, 0), (0, 1 << 30, 0)])
def test_exact_keys_do_not_change_results(exact, chunk, solo, small):
    """Uniqueness keyed by the languages themselves (|ic| <= 62) or by
    fingerprints and rows: the same results, on chunks split small, on the
    whole grid (solo 0), on one CTA (solo 2^30), with and without the
    shared-memory start, through cache growth and out-of-memory ends."""
    with rei.Context(device=0) as c:
        c.set_option(rei.REI_OPT_EXACT_KEYS, exact)
        c.set_option(rei.REI_OPT_CHUNK, chunk)
        c.set_option(rei.REI_OPT_SOLO_TILES, solo)
        c.set_option(rei.REI_OPT_SMALL_ROWS, small)
        for s in (0, 3, 5, 12):
            for costs in [(1, 1, 1, 1, 1), (1, 1, 5, 1, 1)]:
                inst, ref = oracle_medium(s, costs)
                got = c.solve_problem(rei.Problem(inst.alphabet, inst.pos, inst.neg, costs=costs, max_cost=40,
                                                  mem_budget=inst.mem_budget))
                check_same(got, ref, (s, costs, exact, chunk, solo))
        got, ref = solve_both(c, A01, PIN_P, PIN_N, max_cost=30, max_errors=4)
        check_same(got, ref, ("pin20", exact))
        P, N = [b"0110", b"1"], [b"", b"01", b"11"]
        for budget in (64, 400, 2000, 9000):
            got, ref = solve_both(c, A01, P, N, max_cost=30, mem_budget=budget)
            check_same(got, ref, (budget, exact))
    with rei.Context(device=0) as c:
        c.set_option(rei.REI_OPT_EXACT_KEYS, exact)
        c.set_option(rei.REI_OPT_CACHE_INIT, 8)
        for s in (2, 5):
            inst = make_config("medium", s)
            got, ref = solve_both(c, inst, max_cost=40, costs=(1, 1, 1, 1, 1))
            check_same(got, ref, ("growth", s, exact))


SYM = [((1, 1, 1, 1, 1), [1, 3]), ((1, 1, 1, 1, 1), [4, 1]), ((2, 1, 3, 1, 2), [2, 5]), ((5, 1, 1, 1, 1), [2, 2])]


@pytest.mark.parametrize("costs,sym", SYM)
def test_per_symbol_costs_match_oracle(ctx, costs, sym):
    """Different costs for different symbols (Sec. 3): the same answers, counts
    and trees as the oracle, on both staging paths and on the whole grid."""
    insts = [make_config("small", s) for s in range(10)] + [make_config("medium", s) for s in (0, 2, 7)]
    insts += [type1_instance(s, 3, 3, 3, alphabet=b"abc") for s in range(3)]
    for fused, solo in [(1, -1), (0, -1), (1, 0)]:
        with rei.Context(device=0) as c:
            c.set_option(rei.REI_OPT_FUSED_STAGE, fused)
            c.set_option(rei.REI_OPT_SOLO_TILES, solo)
            for inst in insts:
                sc = (sym + [3])[:len(inst.alphabet)]
                ref = oracle.solve(inst.alphabet, inst.pos, inst.neg, costs=costs, max_cost=40, sym_costs=sc,
                                   max_candidates=3_000_000)
                if ref.status == oracle.LIMIT:
                    continue
                got = c.solve_problem(rei.Problem(inst.alphabet, inst.pos, inst.neg, costs=costs, max_cost=40,
                                                  sym_costs=sc, mem_budget=1 << 30))
                check_same(got, ref, (inst.name, inst.seed, costs, sc, fused, solo))
    bad = rei.Problem(A01, [b"1"], [b"0"], sym_costs=[1, 0])
    assert ctx.solve_problem(bad).status == rei.REI_EINVAL


@pytest.mark.parametrize("handover", [1, 500, 20000])
def test_handover_to_the_relaunch_does_not_change_results(handover):
    """Levels above `handover` candidates leave the fused launch for the
    relaunch; with small thresholds every search crosses over mid-way."""
    with rei.Context(device=0) as c:
        c.set_option(rei.REI_OPT_HANDOVER, handover)
        for s in (0, 3, 5, 12):
            for costs in [(1, 1, 1, 1, 1), (1, 1, 5, 1, 1)]:
                inst, ref = oracle_medium(s, costs)
                got = c.solve_problem(rei.Problem(inst.alphabet, inst.pos, inst.neg, costs=costs, max_cost=40,
                                                  mem_budget=inst.mem_budget))
                check_same(got, ref, (s, costs, handover))
        got, ref = solve_both(c, A01, PIN_P, PIN_N, max_cost=30, max_errors=4)
        check_same(got, ref, ("pin20", handover))
        for s in range(4):
            got, ref = solve_both(c, make_config("small", s), max_cost=20, sym_costs=[1, 2])
            check_same(got, ref, ("small sym", s, handover))


def test_fused_launch_growth_keeps_rows_of_wide_languages():
    """A fused launch sizes its cache from what the context holds (here rows of
    2 words) and asks for more memory on a 12-word problem; the relaunch must
    keep the rows it cached."""
    from workloads.gen import batched_instance
    i = batched_instance(0)
    sc = [1, 4, 3, 2][:len(i.alphabet)]
    ref = oracle.solve(i.alphabet, i.pos, i.neg, max_cost=40, sym_costs=sc)
    for sym in (sc, None):
        with rei.Context(device=0) as c:
            got = c.solve_problem(rei.Problem(i.alphabet, i.pos, i.neg, max_cost=40, mem_budget=1 << 30,
                                              sym_costs=sym))
            if sym is not None:
                check_same(got, ref, "sym")
                assert got.launches > 1


@pytest.mark.parametrize("fused", [0, 1])
def test_cache_growth_relaunch_matches(ctx, fused):
    with rei.Context(device=0) as c:
        c.set_option(rei.REI_OPT_FUSED_STAGE, fused)
        c.set_option(rei.REI_OPT_CACHE_INIT, 8)
        c.set_option(rei.REI_OPT_CHUNK, 64)
        for s in (2, 5, 16):
            inst = make_config("medium", s)
            got, ref = solve_both(c, inst, max_cost=40, costs=(1, 1, 1, 1, 1))
            check_same(got, ref, s)
            assert got.launches > 2   # at least one regrow relaunch


def test_cache_contents_match_oracle(ctx):
    """Every cached language, in order, with its back-pointer, per level."""
    for inst, costs in [(make_config("medium", 2), (1, 1, 1, 1, 1)), (make_config("medium", 11), (2, 1, 3, 1, 2)),
                        (make_config("wide", 0), (1, 1, 1, 1, 1))]:
        max_cost = 40 if inst.name != "wide" else 5
        run = oracle.Run()
        ref = run.solve(inst.alphabet, inst.pos, inst.neg, costs=costs, max_cost=max_cost)
        prob = rei.Problem(inst.alphabet, inst.pos, inst.neg, costs=costs, max_cost=max_cost)
        got = ctx.solve_keep(prob)
        check_same(got, ref, inst.name)
        rows, op, left, right, ls, lc = ctx.cache_dump(max_cost + 1)
        n = ref.n_ic
        assert len(rows) >= ref.unique
        for k in range(ref.unique):
            lang, oop, ol, orr = run.cache_entry(k, n)
            bits = bytes((rows[k][w >> 5] >> (w & 31)) & 1 for w in range(n))
            assert bits == lang, (inst.name, k)
            assert (op[k], left[k]) == (oop, ol), k
            assert right[k] == (orr if orr >= 0 else 0xFFFFFFFF), k
            # padding bits beyond n stay zero
            for w in range(n, 32 * len(rows[k])):
                assert not (rows[k][w >> 5] >> (w & 31)) & 1
        for c in range(1, got.cost):
            assert (ls[c], lc[c]) == run.level(c), c


@pytest.mark.parametrize("chunk,solo,exact,handover", [(0, 0, 1, 0), (777, 0, 1, 0), (0, 1 << 30, 1, 0),
                                                         (0, 0, 0, 0), (0, 0, 1, 1000), (777, 64, 1, 1000)])
def test_one_word_cache_matches_oracle(chunk, solo, exact, handover):
    """The 1-word path (|ic| = 25: candidates built in registers through nibble
    tables, the bitmap of cached languages, a table slot per language) row by
    row against the oracle: the printed specification searched to cost 14
    (796 K candidates, 88.8 K languages), every chunk on the whole grid (solo 0)
    or on one CTA, chunks split small and ragged (777), with fingerprint keys
    instead of exact ones, and with levels above 1000 candidates handed from
    the fused launch to the relaunched search kernel."""
    run = oracle.Run()
    ref = run.solve(A01, PIN_P, PIN_N, max_cost=14)
    assert ref.status == oracle.NOT_FOUND
    with rei.Context(device=0) as c:
        c.set_option(rei.REI_OPT_CHUNK, chunk)
        c.set_option(rei.REI_OPT_SOLO_TILES, solo)
        c.set_option(rei.REI_OPT_EXACT_KEYS, exact)
        if handover:
            c.set_option(rei.REI_OPT_HANDOVER, handover)
        got = c.solve_keep(rei.Problem(A01, PIN_P, PIN_N, max_cost=14, mem_budget=1 << 30))
        check_same(got, ref, (chunk, solo, exact, handover))
        assert got.words == 1 and got.n_ic == 25
        rows, op, left, right, ls, lc = c.cache_dump(15)
    assert len(rows) == ref.unique
    for k in range(ref.unique):
        lang, oop, ol, orr = run.cache_entry(k, 25)
        assert bytes((rows[k][0] >> w) & 1 for w in range(25)) == lang, k
        assert rows[k][0] >> 25 == 0, k  # padding bits stay zero
        assert (op[k], left[k], right[k]) == (oop, ol, orr if orr >= 0 else 0xFFFFFFFF), k
    for cst in range(1, 15):
        assert (ls[cst], lc[cst]) == run.level(cst), cst


def test_dynamic_tile_handout_keeps_results_and_cache():
    """A chunk of at least 32 tiles per warp of the grid hands its tiles out
    from a counter, in an order that varies from run to run; the order must not
    change anything.  The printed specification searched to cost 22 (levels of
    tens of millions of candidates, chunks of up to 32 Mi) gives the same result
    and the same cache, row for row, as with chunks of 1 Mi candidates (32 Ki
    tiles, below 32 per warp: the fixed round robin)."""
    out = []
    for chunk in (0, 1 << 20):
        with rei.Context(device=0) as c:
            if chunk:
                c.set_option(rei.REI_OPT_CHUNK, chunk)
            got = c.solve_keep(rei.Problem(A01, PIN_P, PIN_N, max_cost=22, mem_budget=64 << 30))
            out.append((got, c.cache_dump(23, raw=True)))
    (a, ca), (b, cb) = out
    assert a.status == b.status == rei.REI_NOT_FOUND
    assert (a.candidates, a.unique, a.levels) == (b.candidates, b.unique, b.levels)
    assert a.candidates > 5e7   # levels large enough for the counter
    assert ca == cb


def test_device_input_matches_host_input(ctx):
    inst = make_config("medium", 5)
    host = ctx.solve_problem(rei.Problem(inst.alphabet, inst.pos, inst.neg, max_cost=40))
    dev = ctx.solve_problem(rei.Problem.on_device(inst.alphabet, inst.pos, inst.neg, max_cost=40))
    assert (host.status, host.cost, host.tree, host.candidates) == (dev.status, dev.cost, dev.tree, dev.candidates)
    assert dev.bytes_h2d < host.bytes_h2d


def test_type1_type2_instances(ctx):
    for s in range(6):
        for inst in (type1_instance(s, 4, 4, 4), type2_instance(s, 5, 5, 5)):
            for costs in [(1, 1, 1, 1, 1), (1, 1, 10, 1, 1)]:
                got, ref = solve_both(ctx, inst, costs=costs, max_cost=30)
                check_same(got, ref, (inst.name, s, costs))


# ---------------------------------------------------------------------------
# edge cases

def test_trivial_answers(ctx):
    got = ctx.solve(A01, [], [b"0"], costs=(3, 1, 1, 1, 1))
    assert got.status == rei.REI_OK and got.regex == "∅" and got.cost == 3
    got = ctx.solve(A01, [b""], [b"0", b"1"], costs=(3, 1, 1, 1, 1))
    assert got.status == rei.REI_OK and got.regex == "ε" and got.cost == 3
    got = ctx.solve(b"abc", [b"b"], [b"a", b"c", b""])
    assert got.status == rei.REI_OK and got.regex == "b" and got.cost == 1


def test_not_found_and_oom_match_oracle(ctx):
    P, N = [b"0110", b"1"], [b"", b"01", b"11"]
    got, ref = solve_both(ctx, A01, P, N, max_cost=3)
    check_same(got, ref)
    assert got.status == rei.REI_NOT_FOUND
    for budget in (64, 400, 2000, 9000):
        got, ref = solve_both(ctx, A01, P, N, max_cost=30, mem_budget=budget)
        check_same(got, ref, budget)


def test_onthefly_matches_oracle(ctx):
    for s in range(8):
        inst = make_config("small", s)
        for costs in [(1, 2, 3, 3, 3), (1, 3, 3, 4, 4)]:
            for rows in (3, 6, 12):
                budget = rows * 32
                got, ref = solve_both(ctx, inst, costs=costs, max_cost=30, mem_budget=budget,
                                      flags=rei.REI_F_ONTHEFLY)
                check_same(got, ref, (s, costs, rows))


def test_invalid_inputs(ctx):
    assert ctx.solve(b"00", [b"0"], [b""]).status == rei.REI_EINVAL       # repeated symbol
    assert ctx.solve(A01, [b"2"], [b""]).status == rei.REI_EINVAL         # foreign byte
    assert ctx.solve(A01, [b"0"], [b"0"]).status == rei.REI_EINVAL        # P and N overlap
    assert ctx.solve(A01, [b"0"], [b""], costs=(1, 0, 1, 1, 1)).status == rei.REI_EINVAL
    assert ctx.solve(A01, [b"0"], [b""], max_cost=256).status == rei.REI_EINVAL
    # the context stays usable after errors
    assert ctx.solve(A01, *EX1, max_cost=12).cost == 7


@pytest.mark.parametrize("pct", [5, 10])
def test_allowed_error_rows_5_and_10_percent(ctx, golden, pct):
    """Sec. 6's allowed-error table on the printed specification at 5 % and
    10 % (1 and 2 of its 22 examples misclassified): minimal costs 22 and 18,
    beyond the oracle's reach, pinned like the 0 % row's cost 28."""
    g = golden("allowed_error_table.txt")
    row = next(r for r in g["rows"] if int(r[1]) == pct)
    e = pct * 22 // 100
    got = ctx.solve_problem(rei.Problem(A01, PIN_P, PIN_N, max_cost=30, mem_budget=64 << 30, max_errors=e))
    assert got.status == rei.REI_OK and got.cost == int(row[3]), (pct, got.regex, got.cost)
    assert oracle.tree_cost(got.tree, (1, 1, 1, 1, 1)) == got.cost
    wrong = sum(not oracle.match(got.tree, A01, p) for p in PIN_P) + sum(oracle.match(got.tree, A01, q) for q in PIN_N)
    assert wrong <= e
    # the paper's printed expression for the row has that cost and error too
    printed = oracle.parse(row[2], A01)
    assert oracle.tree_cost(printed, (1, 1, 1, 1, 1)) == got.cost
    assert sum(not oracle.match(printed, A01, p) for p in PIN_P) + sum(oracle.match(printed, A01, q) for q in PIN_N) <= e


def test_printed_instance_cost_28(ctx):
    """Sec. 6 / Table 1: the printed specification has minimal cost 28 under
    (1,1,1,1,1); the paper's A100 checked 26,774,099,142 candidates."""
    got = ctx.solve_problem(rei.Problem(A01, PIN_P, PIN_N, max_cost=30, mem_budget=64 << 30))
    assert got.status == rei.REI_OK and got.cost == 28
    assert oracle.tree_cost(got.tree, (1, 1, 1, 1, 1)) == 28
    assert all(oracle.match(got.tree, A01, p) for p in PIN_P)
    assert not any(oracle.match(got.tree, A01, q) for q in PIN_N)
    assert 1e9 < got.candidates < 1e11
