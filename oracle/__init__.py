"""Python access to the plain CPU oracle (``rei_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline legs of ``bench.py`` are the only users.  Nothing in the library
package imports this module.

The oracle is compiled with gcc into ``oracle/_lib/librei_oracle.so`` by
:func:`build` (also called from ``__graft_entry__.build()``).

Parity unpinned by the paper: the choice among equal-cost precise expressions
(the fixed enumeration order) and the exact candidate counts; see the header of
``rei_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rei_oracle.c")
_LIB = os.path.join(_HERE, "_lib", "librei_oracle.so")

OK, NOT_FOUND, OOM, EINVAL, LIMIT, SELFCHECK = 0, 1, 2, 3, 4, 5
STATUS_NAMES = {OK: "ok", NOT_FOUND: "not_found", OOM: "oom", EINVAL: "einval",
                LIMIT: "limit", SELFCHECK: "selfcheck"}
F_SELFCHECK = 1
F_ONTHEFLY = 2


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-D_POSIX_C_SOURCE=199309L", "-fPIC",
                               "-shared", "-o", _LIB, _SRC])
    return _LIB


class _Stats(C.Structure):
    _fields_ = [("status", C.c_int), ("cost", C.c_int), ("candidates", C.c_uint64),
                ("unique", C.c_uint64), ("levels", C.c_int), ("n_ic", C.c_int),
                ("seconds", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        vp, u8p, u32p, i32p = C.c_void_p, C.POINTER(C.c_uint8), C.POINTER(C.c_uint32), C.POINTER(C.c_int)
        L.oracle_new.restype = vp
        L.oracle_free.argtypes = [vp]
        L.oracle_solve.argtypes = [vp, C.c_char_p, C.c_int, C.c_char_p, u32p, C.c_int, C.c_int,
                                   i32p, C.c_int, C.c_uint64, C.c_uint, C.c_uint32, C.c_uint64]
        L.oracle_solve.restype = C.c_int
        L.oracle_solve_sc.argtypes = [vp, C.c_char_p, C.c_int, C.c_char_p, u32p, C.c_int, C.c_int,
                                      i32p, i32p, C.c_int, C.c_uint64, C.c_uint, C.c_uint32, C.c_uint64]
        L.oracle_solve_sc.restype = C.c_int
        L.oracle_tree_cost_sc.argtypes = [C.c_char_p, C.c_int, i32p, i32p]
        L.oracle_brute_min_cost_sc.argtypes = [C.c_char_p, C.c_int, C.c_char_p, u32p, C.c_int, C.c_int,
                                               i32p, i32p, C.c_int, C.c_long, C.c_char_p, C.c_int, i32p]
        L.oracle_stats_of.argtypes = [vp]
        L.oracle_stats_of.restype = C.POINTER(_Stats)
        L.oracle_answer_tree.argtypes = [vp, C.c_char_p, C.c_int]
        L.oracle_answer_text.argtypes = [vp, C.c_char_p, C.c_int]
        L.oracle_ic_words.argtypes = [vp, C.c_char_p, C.c_int, u32p, C.c_int]
        L.oracle_cache_size.argtypes = [vp]
        L.oracle_cache_size.restype = C.c_uint64
        L.oracle_cache_entry.argtypes = [vp, C.c_uint64, C.c_char_p, i32p,
                                         C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.oracle_level.argtypes = [vp, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.oracle_match.argtypes = [C.c_char_p, C.c_int, C.c_char_p, C.c_int, C.c_char_p, C.c_int]
        L.oracle_tree_cost.argtypes = [C.c_char_p, C.c_int, i32p]
        L.oracle_tree_text.argtypes = [C.c_char_p, C.c_int, C.c_char_p, C.c_int, C.c_char_p, C.c_int]
        L.oracle_tree_lang.argtypes = [C.c_char_p, C.c_int, C.c_char_p, C.c_int, C.c_char_p, u32p,
                                       C.c_int, C.c_char_p, C.c_int]
        L.oracle_ic.argtypes = [C.c_char_p, C.c_int, C.c_char_p, u32p, C.c_int, C.c_char_p, C.c_int,
                                u32p, C.c_int]
        L.oracle_brute_min_cost.argtypes = [C.c_char_p, C.c_int, C.c_char_p, u32p, C.c_int, C.c_int,
                                            i32p, C.c_int, C.c_long, C.c_char_p, C.c_int, i32p]
        L.oracle_parse.argtypes = [C.c_char_p, C.c_char_p, C.c_int, C.c_char_p, C.c_int]
        L.oracle_set_mutation.argtypes = [C.c_int]
        L.oracle_budget_cap.argtypes = [C.c_uint64, C.c_int]
        L.oracle_budget_cap.restype = C.c_uint64
        _lib = L
    return _lib


def _pack(strings: Sequence[bytes]):
    buf = b"".join(strings)
    offs = [0]
    for s in strings:
        offs.append(offs[-1] + len(s))
    arr = (C.c_uint32 * len(offs))(*offs)
    return buf, arr


def _costs(costs):
    return (C.c_int * 5)(*costs)


def _sym(sym_costs, n_sym):
    """Per-symbol costs (one per alphabet symbol), or None for c_sym each."""
    if sym_costs is None:
        return None
    if len(sym_costs) != n_sym:
        raise ValueError("one cost per alphabet symbol")
    return (C.c_int * max(n_sym, 1))(*sym_costs)


@dataclass
class Result:
    status: int
    cost: int
    tree: Optional[bytes]     # postfix tokens, 2 bytes each
    text: Optional[str]
    candidates: int
    unique: int
    levels: int
    n_ic: int
    seconds: float

    @property
    def status_name(self) -> str:
        return STATUS_NAMES.get(self.status, str(self.status))


class Run:
    """One oracle search; keeps its cache for inspection after solve()."""

    def __init__(self):
        self._h = lib().oracle_new()

    def __del__(self):
        if getattr(self, "_h", None):
            lib().oracle_free(self._h)
            self._h = None

    def solve(self, alphabet: bytes, pos: Sequence[bytes], neg: Sequence[bytes],
              costs=(1, 1, 1, 1, 1), max_cost: int = 20, mem_budget: int = 1 << 30,
              flags: int = 0, max_errors: int = 0, max_candidates: int = 0, sym_costs=None) -> Result:
        buf, offs = _pack(list(pos) + list(neg))
        L = lib()
        L.oracle_solve_sc(self._h, alphabet, len(alphabet), buf, offs, len(pos), len(neg),
                          _costs(costs), _sym(sym_costs, len(alphabet)), max_cost, mem_budget, flags,
                          max_errors, max_candidates)
        st = L.oracle_stats_of(self._h).contents
        tree = text = None
        if st.status == OK:
            n = L.oracle_answer_tree(self._h, None, 0)
            tb = C.create_string_buffer(2 * n)
            L.oracle_answer_tree(self._h, tb, 2 * n)
            tree = tb.raw[: 2 * n]
            m = L.oracle_answer_text(self._h, None, 0)
            sb = C.create_string_buffer(m + 1)
            L.oracle_answer_text(self._h, sb, m + 1)
            text = sb.raw[:m].decode("utf-8")
        self.alphabet = alphabet
        return Result(st.status, st.cost, tree, text, st.candidates, st.unique, st.levels,
                      st.n_ic, st.seconds)

    def ic_words(self) -> List[bytes]:
        L = lib()
        n = L.oracle_ic_words(self._h, None, 0, None, 0)
        offs = (C.c_uint32 * (n + 1))()
        L.oracle_ic_words(self._h, None, 0, offs, n + 1)
        total = offs[n]
        b = C.create_string_buffer(max(total, 1))
        L.oracle_ic_words(self._h, b, total, offs, n + 1)
        raw = b.raw
        return [raw[offs[i]:offs[i + 1]] for i in range(n)]

    def cache_size(self) -> int:
        return lib().oracle_cache_size(self._h)

    def cache_entry(self, k: int, n_ic: int):
        lang = C.create_string_buffer(max(n_ic, 1))
        op, l, r = C.c_int(), C.c_int64(), C.c_int64()
        if lib().oracle_cache_entry(self._h, k, lang, C.byref(op), C.byref(l), C.byref(r)):
            raise IndexError(k)
        return lang.raw[:n_ic], op.value, l.value, r.value

    def level(self, c: int) -> Tuple[int, int]:
        st, cnt = C.c_int64(), C.c_int64()
        if lib().oracle_level(self._h, c, C.byref(st), C.byref(cnt)):
            return 0, 0
        return st.value, cnt.value


def solve(alphabet, pos, neg, **kw) -> Result:
    return Run().solve(alphabet, pos, neg, **kw)


def match(tree: bytes, alphabet: bytes, s: bytes) -> bool:
    r = lib().oracle_match(tree, len(tree) // 2, alphabet, len(alphabet), s, len(s))
    if r < 0:
        raise ValueError("bad tree")
    return bool(r)


def tree_cost(tree: bytes, costs, sym_costs=None) -> int:
    sc = None if sym_costs is None else (C.c_int * max(len(sym_costs), 1))(*sym_costs)
    return lib().oracle_tree_cost_sc(tree, len(tree) // 2, _costs(costs), sc)


def tree_text(tree: bytes, alphabet: bytes) -> str:
    L = lib()
    m = L.oracle_tree_text(tree, len(tree) // 2, alphabet, len(alphabet), None, 0)
    b = C.create_string_buffer(m + 1)
    L.oracle_tree_text(tree, len(tree) // 2, alphabet, len(alphabet), b, m + 1)
    return b.raw[:m].decode("utf-8")


def parse(text: str, alphabet: bytes) -> bytes:
    L = lib()
    raw = text.encode("utf-8")
    n = L.oracle_parse(raw, alphabet, len(alphabet), None, 0)
    if n < 0:
        raise ValueError(f"cannot parse {text!r}")
    b = C.create_string_buffer(2 * n)
    L.oracle_parse(raw, alphabet, len(alphabet), b, 2 * n)
    return b.raw[: 2 * n]


def ic(alphabet: bytes, strings: Sequence[bytes]) -> List[bytes]:
    L = lib()
    buf, offs = _pack(list(strings))
    n = L.oracle_ic(alphabet, len(alphabet), buf, offs, len(strings), None, 0, None, 0)
    wo = (C.c_uint32 * (n + 1))()
    L.oracle_ic(alphabet, len(alphabet), buf, offs, len(strings), None, 0, wo, n + 1)
    wb = C.create_string_buffer(max(wo[n], 1))
    L.oracle_ic(alphabet, len(alphabet), buf, offs, len(strings), wb, wo[n], wo, n + 1)
    raw = wb.raw
    return [raw[wo[i]:wo[i + 1]] for i in range(n)]


def tree_lang(tree: bytes, alphabet: bytes, strings: Sequence[bytes]) -> bytes:
    """Language of `tree` on ic(strings), one byte per ic word (IPS set ops)."""
    L = lib()
    buf, offs = _pack(list(strings))
    n = L.oracle_tree_lang(tree, len(tree) // 2, alphabet, len(alphabet), buf, offs,
                           len(strings), None, 0)
    out = C.create_string_buffer(max(n, 1))
    L.oracle_tree_lang(tree, len(tree) // 2, alphabet, len(alphabet), buf, offs,
                       len(strings), out, n)
    return out.raw[:n]


def brute_min_cost(alphabet, pos, neg, costs=(1, 1, 1, 1, 1), max_cost=8,
                   node_limit=30_000_000, sym_costs=None):
    """(minimal cost or 0 if none <= max_cost, postfix tree) by brute force."""
    buf, offs = _pack(list(pos) + list(neg))
    tok = C.create_string_buffer(4096)
    tl = C.c_int()
    c = lib().oracle_brute_min_cost_sc(alphabet, len(alphabet), buf, offs, len(pos), len(neg),
                                       _costs(costs), _sym(sym_costs, len(alphabet)), max_cost,
                                       node_limit, tok, 4096, C.byref(tl))
    return c, tok.raw[: 2 * tl.value]


def set_mutation(m: int) -> None:
    """Plant mistake number m in the oracle (0 restores it); tests only."""
    lib().oracle_set_mutation(m)


def budget_cap(budget: int, n_ic: int) -> int:
    return lib().oracle_budget_cap(budget, n_ic)
