"""Seeded synthetic REI instances.

The paper's benchmark files (Type 1 / Type 2 suites, Sec. 5 "Benchmark
Construction") are not available, so every workload here is synthetic:

* target-labelled instances: draw a random target regular expression of a
  given cost, draw random strings, and label each string as positive or
  negative by matching it against the target.  Matching simulates a
  Thompson NFA of the target (a textbook construction), so this module
  shares no code with either the oracle or the CUDA path, and holds none of
  the inference method's arithmetic;
* Type 1 / Type 2 random specifications, written from the description in
  Sec. 5 (Benchmark Construction): uniform strings of length <= le, or a
  uniform length first and then a uniform string of that length.

All randomness comes from ``random.Random(<string seed>)``, whose seeding
(SHA-512 of the string) and Mersenne Twister stream are identical on every
platform, so an instance is a pure function of (config, seed).
"""
from __future__ import annotations

import math
import random
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

Tree = tuple  # ('a', k) | ('?', t) | ('*', t) | ('.', t, u) | ('+', t, u)


@dataclass
class Instance:
    name: str
    seed: int
    alphabet: bytes
    pos: List[bytes]
    neg: List[bytes]
    costs: Tuple[int, int, int, int, int] = (1, 1, 1, 1, 1)
    max_cost: int = 20
    mem_budget: int = 8 << 30
    target: Optional[Tree] = None
    target_cost: Optional[int] = None
    n_ic: int = 0  # distinct substrings of P u N (window filter only)
    extra: dict = field(default_factory=dict)

    def with_costs(self, costs, max_cost=None) -> "Instance":
        return Instance(self.name, self.seed, self.alphabet, list(self.pos), list(self.neg),
                        tuple(costs), self.max_cost if max_cost is None else max_cost,
                        self.mem_budget, self.target, None, self.n_ic, dict(self.extra))


def pack_strings(pos: Sequence[bytes], neg: Sequence[bytes]):
    """Concatenate P then N into one byte string with n+1 uint32 offsets."""
    buf = bytearray()
    offs = [0]
    for s in list(pos) + list(neg):
        buf += s
        offs.append(len(buf))
    return bytes(buf), offs


# ----------------------------------------------------------------------------
# random target trees

def _buildable(costs, top):
    """exact[c] is True when some tree over the five constructors has cost c."""
    c1, c2, c3, c4, c5 = costs
    ok = [False] * (top + 1)
    for c in range(1, top + 1):
        if c == c1:
            ok[c] = True
            continue
        for d in (c2, c3):
            if c - d >= 1 and ok[c - d]:
                ok[c] = True
        for d in (c4, c5):
            r = c - d
            for a in range(1, r):
                if ok[a] and ok[r - a]:
                    ok[c] = True
                    break
    return ok


def random_tree(rng: random.Random, cost: int, costs, n_sym: int, ok=None) -> Tree:
    """Top-down random tree of exactly `cost`: a uniform choice among the
    constructors that still fit the remaining budget, uniform symbols, and a
    uniform split of the budget of a binary constructor."""
    c1, c2, c3, c4, c5 = costs
    if ok is None:
        ok = _buildable(costs, cost)
    choices = []
    if cost == c1:
        choices.append(("a",))
    if cost - c2 >= 1 and ok[cost - c2]:
        choices.append(("?",))
    if cost - c3 >= 1 and ok[cost - c3]:
        choices.append(("*",))
    for op, d in ((".", c4), ("+", c5)):
        r = cost - d
        splits = [a for a in range(1, r) if ok[a] and ok[r - a]]
        if splits:
            choices.append((op, splits))
    if not choices:
        raise ValueError(f"no tree of cost {cost}")
    ch = rng.choice(choices)
    op = ch[0]
    if op == "a":
        return ("a", rng.randrange(n_sym))
    if op == "?":
        return ("?", random_tree(rng, cost - c2, costs, n_sym, ok))
    if op == "*":
        return ("*", random_tree(rng, cost - c3, costs, n_sym, ok))
    a = rng.choice(ch[1])
    d = c4 if op == "." else c5
    return (op, random_tree(rng, a, costs, n_sym, ok),
            random_tree(rng, cost - d - a, costs, n_sym, ok))


class _Nfa:
    """Thompson NFA of a target tree, simulated over state sets (labelling
    only; linear in the string length, no backtracking)."""

    def __init__(self, t: Tree, alphabet: bytes):
        self.sym = []    # state -> byte consumed, or None
        self.nxt = []    # state -> successor on that byte
        self.eps = []    # state -> list of epsilon successors
        self.alphabet = alphabet
        self.start, self.accept = self._build(t)

    def _new(self):
        self.sym.append(None)
        self.nxt.append(None)
        self.eps.append([])
        return len(self.sym) - 1

    def _build(self, t):
        op = t[0]
        if op == "a":
            s, f = self._new(), self._new()
            self.sym[s] = self.alphabet[t[1]]
            self.nxt[s] = f
            return s, f
        if op == ".":
            s1, f1 = self._build(t[1])
            s2, f2 = self._build(t[2])
            self.eps[f1].append(s2)
            return s1, f2
        s, f = self._new(), self._new()
        if op == "+":
            for sub in (t[1], t[2]):
                a, b = self._build(sub)
                self.eps[s].append(a)
                self.eps[b].append(f)
            return s, f
        a, b = self._build(t[1])
        self.eps[s] += [a, f]
        self.eps[b].append(f)
        if op == "*":
            self.eps[b].append(a)
        elif op != "?":
            raise ValueError(op)
        return s, f

    def _closure(self, states):
        stack, seen = list(states), set(states)
        while stack:
            q = stack.pop()
            for r in self.eps[q]:
                if r not in seen:
                    seen.add(r)
                    stack.append(r)
        return frozenset(seen)

    def _compile(self):
        # epsilon-closure of every state, then the closed successor set of
        # every closed state set per byte, memoised (a lazy subset construction)
        self._cl = [self._closure([q]) for q in range(len(self.sym))]
        self._start = self._cl[self.start]
        self._step = {}

    def fullmatch(self, s: bytes) -> bool:
        if not hasattr(self, "_cl"):
            self._compile()
        cur = self._start
        for ch in s:
            key = (cur, ch)
            nxt = self._step.get(key)
            if nxt is None:
                acc = set()
                for q in cur:
                    if self.sym[q] == ch:
                        acc |= self._cl[self.nxt[q]]
                nxt = frozenset(acc)
                self._step[key] = nxt
            cur = nxt
            if not cur:
                return False
        return self.accept in cur


def tree_to_text(t: Tree, alphabet: bytes) -> str:
    op = t[0]
    if op == "a":
        return chr(alphabet[t[1]])
    if op in "?*":
        return "(" + tree_to_text(t[1], alphabet) + ")" + op
    if op == ".":
        return "(" + tree_to_text(t[1], alphabet) + tree_to_text(t[2], alphabet) + ")"
    return "(" + tree_to_text(t[1], alphabet) + "+" + tree_to_text(t[2], alphabet) + ")"


def _n_distinct_substrings(strings) -> int:
    subs = set()
    for s in strings:
        for i in range(len(s) + 1):
            for j in range(i, len(s) + 1):
                subs.add(s[i:j])
    return len(subs)


def _rand_string(rng, alphabet: bytes, lo: int, hi: int) -> bytes:
    n = rng.randint(lo, hi)
    return bytes(rng.choices(alphabet, k=n))


def make_instance(name: str, seed: int, alphabet: bytes, n_pos: int, n_neg: int,
                  len_lo: int, len_hi: int, tcost_lo: int, tcost_hi: int,
                  ic_lo: int, ic_hi: int, costs=(1, 1, 1, 1, 1), max_cost: int = 40,
                  mem_budget: int = 8 << 30, max_tries: int = 2000) -> Instance:
    """A target-labelled instance: P and N are filled with distinct random
    strings that the target accepts / rejects.  The target is redrawn when a
    side cannot be filled within 10^4 string draws, and the whole instance is
    redrawn when the number of distinct substrings leaves [ic_lo, ic_hi]."""
    rng = random.Random(f"{name}:{seed}")
    ok = _buildable(costs, tcost_hi)
    tcosts = [c for c in range(tcost_lo, tcost_hi + 1) if ok[c]]
    for _ in range(max_tries):
        tc = rng.choice(tcosts)
        tree = random_tree(rng, tc, costs, len(alphabet), ok)
        pat = _Nfa(tree, alphabet)
        pos, neg, seen = [], [], set()
        for _draw in range(10_000):
            if len(pos) >= n_pos and len(neg) >= n_neg:
                break
            # a target that has labelled almost nothing on one side after
            # 2000 draws cannot fill it: give it up early
            if _draw == 2000 and (2 * len(pos) < n_pos or 2 * len(neg) < n_neg):
                break
            s = _rand_string(rng, alphabet, len_lo, len_hi)
            if s in seen:
                continue
            m = pat.fullmatch(s)
            if m and len(pos) < n_pos:
                pos.append(s)
                seen.add(s)
            elif not m and len(neg) < n_neg:
                neg.append(s)
                seen.add(s)
        if len(pos) < n_pos or len(neg) < n_neg:
            continue
        nic = _n_distinct_substrings(pos + neg)
        if not (ic_lo <= nic <= ic_hi):
            continue
        return Instance(name, seed, alphabet, pos, neg, tuple(costs), max_cost,
                        mem_budget, tree, tc, nic)
    raise RuntimeError(f"could not draw instance {name}:{seed}")


# ----------------------------------------------------------------------------
# the five workload recipes (sizes follow the paper's workloads: binary or
# small alphabets, lengths 0-10, a few to twenty examples per side)

GiB = 1 << 30

CONFIGS = {
    # Plain single instance, CPU-seconds size.
    "small": dict(alphabet=b"01", n_pos=5, n_neg=5, len_lo=0, len_hi=4,
                  tcost_lo=1, tcost_hi=6, ic_lo=1, ic_hi=32, max_cost=20,
                  mem_budget=1 * GiB),
    # Plain single instance, medium (the bench workload).
    "medium": dict(alphabet=b"01", n_pos=10, n_neg=10, len_lo=0, len_hi=7,
                   tcost_lo=10, tcost_hi=14, ic_lo=1, ic_hi=128, max_cost=40,
                   mem_budget=64 * GiB),
    # Plain single instance, wide (multiword characteristic sequences).
    "wide": dict(alphabet=b"abcd", n_pos=20, n_neg=20, len_lo=1, len_hi=10,
                 tcost_lo=12, tcost_hi=18, ic_lo=400, ic_hi=1500, max_cost=40,
                 mem_budget=64 * GiB),
}


# wide instances with |ic| of 1000-1500 words (32-48 words of 32 bits): the
# wide recipe with every string of the longest length, and with 30 examples a
# side for |ic| above 1408
WIDE_LARGE = {
    "len10": dict(len_lo=10, ic_lo=1000),
    "30x30": dict(n_pos=30, n_neg=30, len_lo=10, ic_lo=1409),
}


def wide_large_instance(variant: str, seed: int) -> Instance:
    return make_config("wide", seed, **WIDE_LARGE[variant])


def printed_instance() -> Instance:
    """The one specification the paper prints in full (Sec. 6, the top row of
    Table 1: Type 1, No 50, cost function (1,1,1,1,1)); its minimal cost is 28
    and the paper's A100 took 4.9512 s over 26,774,099,142 candidates."""
    pos = [b"00", b"1101", b"0001", b"0111", b"001", b"1", b"10", b"1100", b"111", b"1010"]
    neg = [b"", b"0", b"0000", b"0011", b"01", b"010", b"011", b"100", b"1000", b"1001", b"11", b"1110"]
    return Instance("printed", 0, b"01", pos, neg, (1, 1, 1, 1, 1), 30, 64 << 30, None, 28)


def make_config(name: str, seed: int, costs=(1, 1, 1, 1, 1), **over) -> Instance:
    if name in CONFIGS:
        kw = dict(CONFIGS[name])
        kw.update(over)
        return make_instance(name, seed, costs=costs, **kw)
    if name in ("batched", "served"):
        return batched_instance(seed, ic_hi=1024 if name == "batched" else 2048,
                                costs=costs, name=name, **over)
    raise KeyError(name)


def batched_instance(seed: int, ic_hi: int = 1024, costs=(1, 1, 1, 1, 1),
                     name: str = "batched", **over) -> Instance:
    """Uneven instances: |alphabet| 2-4, |P| and |N| each uniform in 2-20,
    lengths 0-10, 16 <= distinct substrings <= ic_hi, target cost 4-14."""
    rng = random.Random(f"{name}-shape:{seed}")
    k = rng.randint(2, 4)
    kw = dict(alphabet=b"0123"[:k], n_pos=rng.randint(2, 20), n_neg=rng.randint(2, 20),
              len_lo=0, len_hi=10, tcost_lo=4, tcost_hi=14, ic_lo=16, ic_hi=ic_hi,
              max_cost=40, mem_budget=4 * GiB)
    kw.update(over)
    return make_instance(name, seed, costs=costs, **kw)


# ----------------------------------------------------------------------------
# Type 1 / Type 2 random specifications (Sec. 5, Benchmark Construction)

def _uniform_upto(rng, alphabet: bytes, le: int) -> bytes:
    k = len(alphabet)
    total = sum(k ** i for i in range(le + 1))
    x = rng.randrange(total)
    n = 0
    while x >= k ** n:
        x -= k ** n
        n += 1
    out = bytearray()
    for _ in range(n):
        x, d = divmod(x, k)
        out.append(alphabet[d])
    return bytes(out)


def _fill(rng, draw, p: int, n: int):
    pos, neg, seen = [], [], set()
    space_guard = 0
    while (len(pos) < p or len(neg) < n) and space_guard < 1_000_000:
        space_guard += 1
        s = draw()
        if s in seen:
            continue
        seen.add(s)
        if len(pos) < p:
            pos.append(s)
        else:
            neg.append(s)
    if len(pos) < p or len(neg) < n:
        raise ValueError("string space too small for p + n distinct strings")
    return pos, neg


def type1_instance(seed: int, p: int, n: int, le: int, alphabet: bytes = b"01",
                   costs=(1, 1, 1, 1, 1), max_cost: int = 40) -> Instance:
    """Type 1: P and N drawn uniformly from all strings of length <= le, disjoint."""
    rng = random.Random(f"type1:{seed}:{p}:{n}:{le}")
    pos, neg = _fill(rng, lambda: _uniform_upto(rng, alphabet, le), p, n)
    return Instance("type1", seed, alphabet, pos, neg, tuple(costs), max_cost,
                    n_ic=_n_distinct_substrings(pos + neg))


def type2_instance(seed: int, p: int, n: int, le: int, alphabet: bytes = b"01",
                   costs=(1, 1, 1, 1, 1), max_cost: int = 40) -> Instance:
    """Type 2: every length 0..le equally likely, then a uniform string of it."""
    rng = random.Random(f"type2:{seed}:{p}:{n}:{le}")

    def draw():
        m = rng.randint(0, le)
        return bytes(rng.choice(alphabet) for _ in range(m))

    pos, neg = _fill(rng, draw, p, n)
    return Instance("type2", seed, alphabet, pos, neg, tuple(costs), max_cost,
                    n_ic=_n_distinct_substrings(pos + neg))


def poisson_trace(rate: float, duration_s: float, seed: Optional[int] = None):
    """Arrival times (seconds) of a Poisson stream of the given rate."""
    rng = random.Random(f"poisson:{rate}:{duration_s}:{seed if seed is not None else rate}")
    t, out = 0.0, []
    while True:
        t += -math.log(1.0 - rng.random()) / rate
        if t >= duration_s:
            return out
        out.append(t)
