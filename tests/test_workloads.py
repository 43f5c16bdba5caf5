"""The synthetic generator: deterministic, and every instance obeys its recipe."""
from workloads import make_config, poisson_trace
from workloads.gen import _Nfa, batched_instance


def _subs(strings):
    return {s[i:j] for s in strings for i in range(len(s) + 1) for j in range(i, len(s) + 1)}


def test_deterministic_and_labelled():
    for name, seeds in (("small", range(6)), ("medium", range(4))):
        for s in seeds:
            a, b = make_config(name, s), make_config(name, s)
            assert (a.pos, a.neg, a.target) == (b.pos, b.neg, b.target)
            assert not set(a.pos) & set(a.neg)
            nfa = _Nfa(a.target, a.alphabet)
            assert all(nfa.fullmatch(p) for p in a.pos)
            assert not any(nfa.fullmatch(q) for q in a.neg)
            assert len(_subs(a.pos + a.neg)) == a.n_ic


def test_recipe_windows():
    i = make_config("medium", 3)
    assert len(i.pos) == len(i.neg) == 10 and i.n_ic <= 128
    assert all(len(s) <= 7 for s in i.pos + i.neg) and 10 <= i.target_cost <= 14
    b = batched_instance(5)
    assert 2 <= len(b.pos) <= 20 and 16 <= b.n_ic <= 1024 and 2 <= len(b.alphabet) <= 4


def test_poisson_trace():
    t = poisson_trace(200.0, 5.0)
    assert t == poisson_trace(200.0, 5.0)
    assert all(x < y for x, y in zip(t, t[1:])) and 700 < len(t) < 1300


def test_printed_instance_is_the_papers():
    """The benchmark's copy of the specification printed in Sec. 6 (Table 1,
    Type 1 No 50) equals the golden fixture transcribed from the paper."""
    import os
    from workloads import printed_instance
    inst = printed_instance()
    path = os.path.join(os.path.dirname(__file__), "golden", "allowed_error_table.txt")
    P = N = None
    for line in open(path):
        if line.startswith("P:"):
            P = [w.encode() for w in line.split()[1:]]
        if line.startswith("N:"):
            N = [b"" if w == "_" else w.encode() for w in line.split()[1:]]
    assert inst.pos == P and inst.neg == N
    assert inst.alphabet == b"01" and inst.costs == (1, 1, 1, 1, 1) and inst.target_cost == 28
