"""Python binding of the REI library (include/rei.h), argument marshalling only.

Every step of the search runs in the CUDA kernels of ``librei.so``; this module
only converts Python values to the C structures of the ABI and back.  There is
no fallback: if the library cannot be loaded, every call raises.

The functions keep the C names (``rei_ctx_create``, ``rei_solve``, ...); the
``Context`` class and ``solve()`` wrap them for convenience.  PyTorch, when it
is importable, supplies device memory (its caching allocator, through the
``rei_alloc`` callbacks) and the stream (its current stream).
"""
from __future__ import annotations

import ctypes as C
import itertools
import struct
import os
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

from . import build as _build

LIB_PATH = _build.LIB

(REI_OK, REI_NOT_FOUND, REI_OOM, REI_EINVAL, REI_EBUFSZ, REI_ECUDA, REI_ETIMEOUT, REI_EBUSY,
 REI_ESCRATCH) = range(9)
STATUS_NAMES = {REI_OK: "ok", REI_NOT_FOUND: "not_found", REI_OOM: "oom", REI_EINVAL: "einval",
                REI_EBUFSZ: "ebufsz", REI_ECUDA: "ecuda", REI_ETIMEOUT: "etimeout", REI_EBUSY: "ebusy",
                REI_ESCRATCH: "escratch"}
REI_NOALLOC_SCRATCH_BYTES = 64 << 20
REI_F_DEVICE_INPUT = 1
REI_F_ONTHEFLY = 2
REI_OPT_CHUNK, REI_OPT_GRID, REI_OPT_KEEP_CACHE, REI_OPT_CACHE_INIT, REI_OPT_SOLO_TILES = 1, 2, 3, 4, 5
REI_OPT_SMALL_ROWS = 6
REI_OPT_FUSED_STAGE = 7
REI_OPT_EXACT_KEYS = 8
REI_OPT_HANDOVER = 9
REI_OPT_YIELD_US = 10
REI_MAX_IC, REI_MAX_STRLEN, REI_MAX_COST = 4096, 4095, 255

# every entry point include/rei.h declares
EXPORTS = ["rei_ctx_create", "rei_ctx_destroy", "rei_ctx_set_option", "rei_ctx_launches",
           "rei_solve", "rei_solve_problem", "rei_stage", "rei_cache_dump", "rei_solve_batch",
           "rei_server_create", "rei_server_submit", "rei_server_poll", "rei_server_destroy",
           "rei_solve_noalloc"]


class rei_costs(C.Structure):
    _fields_ = [("c_sym", C.c_uint32), ("c_opt", C.c_uint32), ("c_star", C.c_uint32),
                ("c_cat", C.c_uint32), ("c_alt", C.c_uint32)]


class rei_str(C.Structure):
    _fields_ = [("ptr", C.c_void_p), ("len", C.c_uint32)]


class rei_stats(C.Structure):
    _fields_ = [("candidates", C.c_uint64), ("unique", C.c_uint64), ("levels", C.c_uint32),
                ("n_ic", C.c_uint32), ("words", C.c_uint32), ("max_len", C.c_uint32),
                ("guide_pairs", C.c_uint64), ("ms_stage", C.c_double), ("ms_total", C.c_double),
                ("launches", C.c_uint64), ("bytes_h2d", C.c_uint64), ("bytes_d2h", C.c_uint64),
                ("cand_op", C.c_uint64 * 5), ("star_pairs", C.c_uint64),
                ("ms_search_kernel", C.c_double), ("ms_stage_kernel", C.c_double),
                ("search_launches", C.c_uint32), ("grid", C.c_uint32)]


class rei_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("cost", C.c_uint32), ("regex", C.c_void_p),
                ("regex_cap", C.c_size_t), ("regex_len", C.c_size_t), ("tree", C.c_void_p),
                ("tree_cap", C.c_size_t), ("tree_len", C.c_size_t), ("stats", rei_stats)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)


class rei_alloc(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class rei_problem(C.Structure):
    _fields_ = [("alphabet", C.c_void_p), ("n_sym", C.c_uint32), ("bytes", C.c_void_p),
                ("offsets", C.c_void_p), ("n_pos", C.c_uint32), ("n_neg", C.c_uint32),
                ("total_bytes", C.c_uint64), ("costs", rei_costs), ("max_cost", C.c_uint32),
                ("mem_budget", C.c_uint64), ("max_errors", C.c_uint32), ("flags", C.c_uint32),
                ("sym_costs", C.c_void_p)]


class rei_staged(C.Structure):
    _fields_ = [("n_ic", C.c_uint32), ("words", C.c_uint32), ("max_len", C.c_uint32),
                ("guide_pairs", C.c_uint64), ("word_start", C.c_void_p), ("word_len", C.c_void_p),
                ("gt_off", C.c_void_p), ("gt_pair", C.c_void_p), ("pos_mask", C.c_void_p),
                ("neg_mask", C.c_void_p), ("leaf", C.c_void_p), ("cap_words", C.c_uint32),
                ("cap_pairs", C.c_uint32), ("cap_w", C.c_uint32)]


class rei_tune(C.Structure):
    _fields_ = [("warps_per_cta", C.c_uint32), ("chunk", C.c_uint32), ("yield_us", C.c_uint32)]


_lib = None


def load(build_if_missing: bool = True):
    """Load librei.so (building it first when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"REI CUDA library missing: {LIB_PATH} (run paper_2305_18575_gb300/build.py)")
    L = C.CDLL(LIB_PATH)
    vp, u64p = C.c_void_p, C.POINTER(C.c_uint64)
    sig = {
        "rei_ctx_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(rei_alloc), vp]),
        "rei_ctx_destroy": (None, [vp]),
        "rei_ctx_set_option": (C.c_int, [vp, C.c_int, C.c_int64]),
        "rei_ctx_launches": (C.c_uint64, [vp]),
        "rei_solve": (C.c_int, [vp, C.c_char_p, C.c_uint32, C.POINTER(rei_str), C.c_uint32,
                                C.POINTER(rei_str), C.c_uint32, rei_costs, C.c_uint32, C.c_uint64,
                                C.POINTER(rei_result)]),
        "rei_solve_problem": (C.c_int, [vp, C.POINTER(rei_problem), C.POINTER(rei_result)]),
        "rei_stage": (C.c_int, [vp, C.POINTER(rei_problem), C.POINTER(rei_staged)]),
        "rei_cache_dump": (C.c_int, [vp, vp, vp, vp, vp, u64p, vp, vp, C.c_uint32]),
        "rei_solve_batch": (C.c_int, [vp, C.POINTER(rei_problem), C.c_uint32, C.POINTER(rei_result),
                                      C.POINTER(rei_tune)]),
        "rei_server_create": (C.c_int, [vp, C.c_uint64, C.c_uint32, C.POINTER(C.c_void_p)]),
        "rei_server_submit": (C.c_int, [vp, C.POINTER(rei_problem), u64p]),
        "rei_server_poll": (C.c_int, [vp, C.c_uint64, C.POINTER(rei_result), C.c_int]),
        "rei_server_destroy": (None, [vp]),
        "rei_solve_noalloc": (C.c_int, [C.POINTER(rei_problem), vp, C.POINTER(rei_result)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


# ----------------------------------------------------------------------------
# C-named wrappers (same names as include/rei.h)

def rei_ctx_create(device: int = 0, alloc: Optional[rei_alloc] = None, stream: Optional[int] = None):
    h = C.c_void_p()
    s = load().rei_ctx_create(C.byref(h), device, C.byref(alloc) if alloc is not None else None,
                              C.c_void_p(stream) if stream else None)
    if s != REI_OK:
        raise RuntimeError(f"rei_ctx_create failed: {STATUS_NAMES.get(s, s)}")
    return h


def rei_ctx_destroy(ctx) -> None:
    load().rei_ctx_destroy(ctx)


def rei_ctx_set_option(ctx, option: int, value: int) -> int:
    return load().rei_ctx_set_option(ctx, option, value)


def rei_ctx_launches(ctx) -> int:
    return load().rei_ctx_launches(ctx)


def rei_solve(ctx, alphabet: bytes, P: Sequence[bytes], N: Sequence[bytes], costs, max_cost: int,
              mem_budget: int, out: rei_result) -> int:
    strs = list(P) + list(N)
    n = len(strs)
    keep = C.create_string_buffer(b"".join(strs))  # every string, back to back
    base = C.addressof(keep)
    lens = [len(x) for x in strs]
    starts = list(itertools.accumulate(lens, initial=base))[:n]
    # the rei_str array {pointer, length} in one pack
    flat = [v for pair in zip(starts, lens) for v in pair]
    arr = (rei_str * max(n, 1)).from_buffer_copy(struct.pack("<" + "QI4x" * n, *flat) or bytes(C.sizeof(rei_str)))
    nP = len(P)
    pP = C.cast(arr, C.POINTER(rei_str))
    pN = C.cast(C.byref(arr, nP * C.sizeof(rei_str)), C.POINTER(rei_str))
    return load().rei_solve(ctx, alphabet, len(alphabet), pP, nP, pN, len(N), rei_costs(*costs),
                            max_cost, mem_budget, C.byref(out))


def rei_solve_problem(ctx, prob: rei_problem, out: rei_result) -> int:
    return load().rei_solve_problem(ctx, C.byref(prob), C.byref(out))


def rei_stage(ctx, prob: rei_problem, out: rei_staged) -> int:
    return load().rei_stage(ctx, C.byref(prob), C.byref(out))


def rei_cache_dump(ctx, cs, op, left, right, count: C.c_uint64, level_start, level_count, n_levels) -> int:
    return load().rei_cache_dump(ctx, cs, op, left, right, C.byref(count), level_start, level_count, n_levels)


def rei_solve_batch(ctx, probs, n: int, outs, tune: Optional[rei_tune] = None) -> int:
    return load().rei_solve_batch(ctx, probs, n, outs, C.byref(tune) if tune is not None else None)


def rei_server_create(ctx, budget_bytes: int, max_live: int):
    h = C.c_void_p()
    s = load().rei_server_create(ctx, budget_bytes, max_live, C.byref(h))
    if s != REI_OK:
        raise RuntimeError(f"rei_server_create failed: {STATUS_NAMES.get(s, s)}")
    return h


def rei_server_submit(srv, prob: rei_problem) -> int:
    t = C.c_uint64()
    s = load().rei_server_submit(srv, C.byref(prob), C.byref(t))
    if s != REI_OK:
        raise RuntimeError(f"rei_server_submit failed: {STATUS_NAMES.get(s, s)}")
    return t.value


def rei_server_poll(srv, ticket: int, out: rei_result, block_ms: int) -> int:
    return load().rei_server_poll(srv, ticket, C.byref(out), block_ms)


def rei_server_destroy(srv) -> None:
    load().rei_server_destroy(srv)


def rei_solve_noalloc(prob: rei_problem, stream: Optional[int], out: rei_result) -> int:
    """Solve without allocating (see include/rei.h); `stream` is a cudaStream_t or None."""
    return load().rei_solve_noalloc(C.byref(prob), C.c_void_p(stream) if stream else None, C.byref(out))


# ----------------------------------------------------------------------------
# convenience layer

@dataclass
class Result:
    status: int
    cost: int
    regex: Optional[str]
    tree: Optional[bytes]
    candidates: int
    unique: int
    levels: int
    n_ic: int
    words: int
    guide_pairs: int
    ms_stage: float
    ms_total: float
    launches: int
    bytes_h2d: int
    bytes_d2h: int
    cand_op: tuple = ()
    star_pairs: int = 0
    ms_search_kernel: float = 0.0
    ms_stage_kernel: float = 0.0
    search_launches: int = 0
    grid: int = 0

    @property
    def status_name(self) -> str:
        return STATUS_NAMES.get(self.status, str(self.status))


class _OutBuf:
    """Caller-owned output buffers of one rei_result."""

    def __init__(self, regex_cap: int = 8192, tree_cap: int = 2 * (REI_MAX_COST + 1)):
        self.rbuf = C.create_string_buffer(regex_cap)
        self.tbuf = C.create_string_buffer(tree_cap)
        self.raddr = C.addressof(self.rbuf)
        self.taddr = C.addressof(self.tbuf)
        self.res = rei_result()
        self.reset()

    def reset(self):
        r = self.res
        r.regex = self.raddr
        r.regex_cap = len(self.rbuf)
        r.tree = self.taddr
        r.tree_cap = len(self.tbuf)

    def result(self, status: int) -> Result:
        return _result(self.res, status, self.raddr, self.taddr)


def _result(r: "rei_result", status: int, raddr: int, taddr: int) -> Result:
    ok = status == REI_OK
    st = r.stats
    # (only the bytes written are copied out of the buffers)
    return Result(status, r.cost if ok else 0,
                  C.string_at(raddr, r.regex_len).decode("utf-8") if ok else None,
                  C.string_at(taddr, r.tree_len) if ok else None, st.candidates, st.unique,
                  st.levels, st.n_ic, st.words, st.guide_pairs, st.ms_stage, st.ms_total,
                  st.launches, st.bytes_h2d, st.bytes_d2h, tuple(st.cand_op), st.star_pairs,
                  st.ms_search_kernel, st.ms_stage_kernel, st.search_launches, st.grid)


class _BatchBufs:
    """Caller-owned outputs of a batch of n problems: one rei_result array and
    one regex and one tree buffer for all of them (the pointers are set once;
    the library writes only lengths, statistics and the text).  A regex of at
    most REI_MAX_COST + 1 nodes prints at most 3 bytes per node (a symbol or
    an operator, and its parentheses), so 1024 bytes hold any of them."""

    def __init__(self, n: int, regex_cap: int = 1024, tree_cap: int = 2 * (REI_MAX_COST + 1)):
        self.n = n
        self.rcap, self.tcap = regex_cap, tree_cap
        self.rbuf = C.create_string_buffer(regex_cap * max(n, 1))
        self.tbuf = C.create_string_buffer(tree_cap * max(n, 1))
        self.outs = (rei_result * max(n, 1))()
        ra, ta = C.addressof(self.rbuf), C.addressof(self.tbuf)
        self.raddr = [ra + i * regex_cap for i in range(n)]
        self.taddr = [ta + i * tree_cap for i in range(n)]
        for i in range(n):
            o = self.outs[i]
            o.regex = self.raddr[i]
            o.regex_cap = regex_cap
            o.tree = self.taddr[i]
            o.tree_cap = tree_cap

    def results(self) -> List[Result]:
        # every record unpacked at once (field by field through ctypes would
        # cost more than the batch's search)
        raw = C.string_at(C.addressof(self.outs), _RESULT_SIZE * self.n)
        rtext = C.string_at(self.raddr[0], self.rcap * self.n) if self.n else b""
        ttext = C.string_at(self.taddr[0], self.tcap * self.n) if self.n else b""
        res = []
        for i, f in enumerate(_RESULT_FMT.iter_unpack(raw)):
            (status, cost, _, _, rlen, _, _, tlen, cand, uniq, levels, n_ic, words, _max_len, gp, ms_stage,
             ms_total, launches, h2d, d2h, o0, o1, o2, o3, o4, star, ms_sk, ms_stk, s_l, grid) = f
            ok = status == REI_OK
            r0, t0 = i * self.rcap, i * self.tcap
            res.append(Result(status, cost if ok else 0,
                              rtext[r0:r0 + rlen].decode("utf-8") if ok else None,
                              ttext[t0:t0 + tlen] if ok else None, cand, uniq, levels, n_ic, words,
                              gp, ms_stage, ms_total, launches, h2d, d2h, (o0, o1, o2, o3, o4), star, ms_sk,
                              ms_stk, s_l, grid))
        return res


# rei_result as stored (x86-64 and aarch64 alike: natural alignment, no padding)
_RESULT_FMT = struct.Struct("=iIQQQQQQ" "QQIIIIQddQQQ5QQddII")
_RESULT_SIZE = _RESULT_FMT.size
assert _RESULT_SIZE == C.sizeof(rei_result), (_RESULT_SIZE, C.sizeof(rei_result))


def pack(pos: Sequence[bytes], neg: Sequence[bytes]):
    buf = b"".join(list(pos) + list(neg))
    offs = [0]
    for s in list(pos) + list(neg):
        offs.append(offs[-1] + len(s))
    return buf, offs


class Problem:
    """A packed problem (rei_problem) with its host or device storage kept alive."""

    def __init__(self, alphabet: bytes, pos: Sequence[bytes], neg: Sequence[bytes],
                 costs=(1, 1, 1, 1, 1), max_cost: int = 20, mem_budget: int = 1 << 30,
                 max_errors: int = 0, flags: int = 0, device_tensors=None, sym_costs=None):
        self.alphabet = bytes(alphabet)
        self._abuf = C.create_string_buffer(self.alphabet, max(len(self.alphabet), 1))
        buf, offs = pack(pos, neg)
        self.total = len(buf)
        p = rei_problem()
        p.alphabet = C.cast(self._abuf, C.c_void_p)
        p.n_sym = len(self.alphabet)
        p.n_pos, p.n_neg = len(pos), len(neg)
        p.total_bytes = len(buf)
        p.costs = rei_costs(*costs)
        p.max_cost = max_cost
        p.mem_budget = mem_budget
        p.max_errors = max_errors
        p.flags = flags
        if sym_costs is not None:
            if len(sym_costs) != len(self.alphabet):
                raise ValueError("sym_costs: one cost per alphabet symbol")
            self._sbuf = (C.c_uint32 * max(len(sym_costs), 1))(*sym_costs)
            p.sym_costs = C.cast(self._sbuf, C.c_void_p)
        if device_tensors is not None:
            # (uint8 tensor of bytes, int32 tensor of offsets), already on the device
            tb, to = device_tensors
            self._dev = (tb, to)
            p.bytes = tb.data_ptr()
            p.offsets = to.data_ptr()
            p.flags = flags | REI_F_DEVICE_INPUT
        else:
            self._bbuf = C.create_string_buffer(buf, max(len(buf), 1))
            self._obuf = (C.c_uint32 * len(offs))(*offs)
            p.bytes = C.cast(self._bbuf, C.c_void_p)
            p.offsets = C.cast(self._obuf, C.c_void_p)
        self.p = p

    @classmethod
    def on_device(cls, alphabet, pos, neg, device: int = 0, **kw) -> "Problem":
        import torch
        buf, offs = pack(pos, neg)
        tb = torch.tensor(list(buf) or [0], dtype=torch.uint8, device=f"cuda:{device}")
        to = torch.tensor(offs, dtype=torch.int32, device=f"cuda:{device}")
        return cls(alphabet, pos, neg, device_tensors=(tb, to), **kw)


def torch_allocator(device: int = 0):
    """rei_alloc callbacks backed by PyTorch's CUDA caching allocator."""
    import torch

    def _alloc(user, nbytes, stream):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, int(stream or 0))
        except Exception:  # noqa: BLE001 -- reported to the library as NULL
            return None

    def _free(user, ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(ptr)

    a = rei_alloc(ALLOC_FN(_alloc), FREE_FN(_free), None)
    return a


class Context:
    """One library context (device, allocator, stream)."""

    def __init__(self, device: int = 0, use_torch: bool = True, stream: Optional[int] = None):
        self._alloc = None
        if use_torch:
            try:
                import torch
                if torch.cuda.is_available():
                    self._alloc = torch_allocator(device)
                    if stream is None:
                        stream = torch.cuda.current_stream(device).cuda_stream
            except ImportError:
                pass
        self.h = rei_ctx_create(device, self._alloc, stream)
        self._out = _OutBuf()

    def close(self):
        if getattr(self, "h", None):
            rei_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_option(self, option: int, value: int):
        if rei_ctx_set_option(self.h, option, value) != REI_OK:
            raise ValueError(f"bad option {option}={value}")

    @property
    def launches(self) -> int:
        return rei_ctx_launches(self.h)

    def solve(self, alphabet: bytes, pos, neg, costs=(1, 1, 1, 1, 1), max_cost: int = 20,
              mem_budget: int = 1 << 30) -> Result:
        o = self._out
        o.reset()
        s = rei_solve(self.h, alphabet, pos, neg, costs, max_cost, mem_budget, o.res)
        return o.result(s)

    def solve_problem(self, prob: Problem) -> Result:
        o = self._out
        o.reset()
        s = rei_solve_problem(self.h, prob.p, o.res)
        return o.result(s)

    def stage(self, prob: Problem, cap_words: int = REI_MAX_IC, cap_pairs: int = 1 << 20):
        """Staged form: dict with ic words, guide table, masks and leaves."""
        W = (REI_MAX_IC + 31) // 32
        ws = (C.c_uint32 * cap_words)()
        wl = (C.c_uint32 * cap_words)()
        go = (C.c_uint32 * (cap_words + 1))()
        gp = (C.c_uint32 * cap_pairs)()
        pm = (C.c_uint32 * W)()
        nm = (C.c_uint32 * W)()
        lf = (C.c_uint32 * (W * max(prob.p.n_sym, 1)))()
        st = rei_staged(0, 0, 0, 0, C.cast(ws, C.c_void_p), C.cast(wl, C.c_void_p),
                        C.cast(go, C.c_void_p), C.cast(gp, C.c_void_p), C.cast(pm, C.c_void_p),
                        C.cast(nm, C.c_void_p), C.cast(lf, C.c_void_p), cap_words, cap_pairs, W)
        s = rei_stage(self.h, prob.p, st)
        if s != REI_OK:
            return s, None
        n, G, Wn = st.n_ic, st.guide_pairs, st.words
        return s, dict(n=n, W=Wn, max_len=st.max_len, G=G, word_start=list(ws[:n]),
                       word_len=list(wl[:n]), gt_off=list(go[: n + 1]), gt_pair=list(gp[:G]),
                       pos=list(pm[:Wn]), neg=list(nm[:Wn]),
                       leaf=[list(lf[a * W: a * W + Wn]) for a in range(prob.p.n_sym)])

    def cache_dump(self, n_levels: int, raw: bool = False):
        """(cs words per row, op, left, right, level_start, level_count) of the last solve;
        raw=True gives the four arrays as little-endian bytes instead of lists."""
        cnt = C.c_uint64(0)
        s = rei_cache_dump(self.h, None, None, None, None, cnt, None, None, 0)
        if s not in (REI_OK, REI_EBUFSZ):
            raise RuntimeError(f"rei_cache_dump: {STATUS_NAMES.get(s, s)}")
        k = cnt.value
        W = self._last_words
        cs = (C.c_uint32 * max(k * W, 1))()
        op = (C.c_uint8 * max(k, 1))()
        lf = (C.c_uint32 * max(k, 1))()
        rt = (C.c_uint32 * max(k, 1))()
        ls = (C.c_uint64 * n_levels)()
        lc = (C.c_uint64 * n_levels)()
        cnt = C.c_uint64(k)
        s = rei_cache_dump(self.h, C.cast(cs, C.c_void_p), C.cast(op, C.c_void_p), C.cast(lf, C.c_void_p),
                           C.cast(rt, C.c_void_p), cnt, C.cast(ls, C.c_void_p), C.cast(lc, C.c_void_p),
                           n_levels)
        if s != REI_OK:
            raise RuntimeError(f"rei_cache_dump: {STATUS_NAMES.get(s, s)}")
        if raw:
            return (bytes(cs)[:4 * k * W], bytes(op)[:k], bytes(lf)[:4 * k], bytes(rt)[:4 * k], list(ls), list(lc))
        rows = [list(cs[i * W:(i + 1) * W]) for i in range(k)]
        return rows, list(op[:k]), list(lf[:k]), list(rt[:k]), list(ls), list(lc)

    def solve_batch(self, probs: Sequence[Problem], warps_per_cta: int = 0, chunk: int = 0,
                    yield_us: int = 0) -> List[Result]:
        """rei_solve_batch over `probs` (one staging and one search launch);
        a rei_tune field left 0 is chosen by the library (see include/rei.h)."""
        n = len(probs)
        arr = (rei_problem * max(n, 1))(*[p.p for p in probs])
        # (the output buffers of a batch of the same size are reused)
        if getattr(self, "_batch_bufs", None) is None or self._batch_bufs.n != n:
            self._batch_bufs = _BatchBufs(n)
        tune = rei_tune(warps_per_cta, chunk, yield_us) if (warps_per_cta or chunk or yield_us) else None
        s = rei_solve_batch(self.h, arr, n, self._batch_bufs.outs, tune)
        if s != REI_OK:
            raise RuntimeError(f"rei_solve_batch: {STATUS_NAMES.get(s, s)}")
        return self._batch_bufs.results()

    def solve_keep(self, prob: Problem) -> Result:
        """solve_problem with the cache kept for cache_dump()."""
        self.set_option(REI_OPT_KEEP_CACHE, 1)
        r = self.solve_problem(prob)
        self._last_words = r.words
        return r


class Server:
    """Served form: problems submitted at any time are solved by one persistent
    launch as its CTAs free up (continuous batching).  `budget_bytes` bounds the
    cache the live problems may hold together, `max_live` how many are live."""

    def __init__(self, ctx: Context, budget_bytes: int = 8 << 30, max_live: int = 1 << 12):
        self.ctx = ctx
        self.h = rei_server_create(ctx.h, budget_bytes, max_live)
        self._probs = {}

    def submit(self, prob: Problem) -> int:
        t = rei_server_submit(self.h, prob.p)
        self._probs[t] = prob
        return t

    def result(self, ticket: int, block_ms: int = -1) -> Optional[Result]:
        """The ticket's Result, or None when it is not finished within block_ms."""
        o = _OutBuf()
        s = rei_server_poll(self.h, ticket, o.res, block_ms)
        if s == REI_EBUSY:
            return None
        if s != REI_OK:
            raise RuntimeError(f"rei_server_poll: {STATUS_NAMES.get(s, s)}")
        self._probs.pop(ticket, None)
        return o.result(o.res.status)

    def close(self):
        if getattr(self, "h", None):
            rei_server_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def solve(alphabet: bytes, pos, neg, **kw) -> Result:
    with Context() as ctx:
        return ctx.solve(alphabet, pos, neg, **kw)
