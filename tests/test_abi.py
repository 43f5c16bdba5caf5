"""The C ABI library builds for sm_103a, loads, and exports every entry
point include/rei.h declares (no GPU needed)."""
import ctypes
import os
import re

import paper_2305_18575_gb300 as rei
from paper_2305_18575_gb300 import build as b

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "rei.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rei_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_entry_point():
    lib = ctypes.CDLL(b.build())
    names = declared()
    assert len(names) >= 13
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(rei.EXPORTS) == names


def test_binding_structs_match_header_layout(tmp_path):
    """ctypes mirrors of the ABI structs have the sizes and field offsets the
    C compiler gives include/rei.h."""
    import subprocess
    structs = {"rei_costs": rei.rei_costs, "rei_str": rei.rei_str, "rei_stats": rei.rei_stats,
               "rei_result": rei.rei_result, "rei_alloc": rei.rei_alloc,
               "rei_problem": rei.rei_problem, "rei_staged": rei.rei_staged, "rei_tune": rei.rei_tune}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rei.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(got[f"{name}.{fname}"]) == getattr(cls, fname).offset, f"{name}.{fname}"


def test_no_cpu_fallback_without_gpu():
    """Without a GPU the library refuses to create a context: there is no CPU path."""
    import torch
    if torch.cuda.is_available():
        return
    h = ctypes.c_void_p()
    assert rei.load().rei_ctx_create(ctypes.byref(h), 0, None, None) != rei.REI_OK


def test_binding_constants_match_header(tmp_path):
    """Status codes, flags, options and limits of the binding are the values
    the C compiler sees in include/rei.h."""
    import subprocess
    src = open(os.path.join(ROOT, "include", "rei.h")).read()
    names = sorted(set(re.findall(r"^#define (REI_(?:F|OPT|MAX)_[A-Z_]+)\b", src, flags=re.M)))
    names += ["REI_NOALLOC_SCRATCH_BYTES"]
    names += sorted(set(re.findall(r"^\s+(REI_[A-Z_]+)\s*=\s*\d+", src, flags=re.M)))  # rei_status
    assert {"REI_OK", "REI_ETIMEOUT", "REI_OPT_YIELD_US", "REI_F_ONTHEFLY", "REI_MAX_IC"} <= set(names)
    lines = ['#include <stdio.h>', '#include "rei.h"', "int main(void) {"]
    lines += [f'printf("{n} %llu\\n", (unsigned long long)({n}));' for n in names]
    lines.append("return 0; }")
    c = tmp_path / "consts.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "consts"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().splitlines())
    for n in names:
        assert hasattr(rei, n), n
        assert int(got[n]) == getattr(rei, n), n


def _noalloc(prob):
    buf = rei._OutBuf()
    s = rei.rei_solve_noalloc(prob.p, None, buf.res)
    return s, buf.res.status


def test_noalloc_refuses_bad_arguments_before_any_launch():
    """rei_solve_noalloc applies the argument rules of every other entry point
    and answers REI_EINVAL, in the return value and in out->status, before it
    makes any CUDA call (so this runs without a GPU)."""
    # device inputs: bytes missing while total_bytes > 0
    p = rei.Problem(b"01", [b"01"], [b"1"])
    p.p.flags |= rei.REI_F_DEVICE_INPUT
    p.p.bytes = None
    p.p.total_bytes = 3
    assert _noalloc(p) == (rei.REI_EINVAL, rei.REI_EINVAL)
    # host inputs: bytes missing while the strings are not empty
    p = rei.Problem(b"01", [b"01"], [b"1"])
    p.p.bytes = None
    assert _noalloc(p) == (rei.REI_EINVAL, rei.REI_EINVAL)
    # example counts whose 32-bit sum wraps around: beyond the 2^24 limit
    p = rei.Problem(b"01", [b"01"], [b"1"])
    p.p.n_pos, p.p.n_neg = 0xFFFFFFFF, 2
    assert _noalloc(p) == (rei.REI_EINVAL, rei.REI_EINVAL)
    # a zero cost, a repeated symbol, max_cost beyond the limit
    assert _noalloc(rei.Problem(b"01", [b"01"], [b"1"], costs=(1, 0, 1, 1, 1))) == (rei.REI_EINVAL, rei.REI_EINVAL)
    assert _noalloc(rei.Problem(b"00", [b"0"], [b""])) == (rei.REI_EINVAL, rei.REI_EINVAL)
    assert _noalloc(rei.Problem(b"01", [b"0"], [b""], max_cost=256)) == (rei.REI_EINVAL, rei.REI_EINVAL)


def test_batch_results_unpack_every_field():
    """The batch binding reads all rei_result records with one unpack (a packed
    format of the struct): every field of every record, and each record's own
    regex and tree bytes, come out as field-by-field reading gives them."""
    import ctypes as C
    n = 37
    b = rei._BatchBufs(n)
    for i in range(n):
        o = b.outs[i]
        o.status = rei.REI_OK if i % 3 else rei.REI_NOT_FOUND
        o.cost = 5 + i
        text = b"0*(1%d)?" % i
        o.regex_len = len(text)
        C.memmove(b.raddr[i], text, len(text))
        tree = bytes((i + k) & 255 for k in range(2 * (i % 7 + 1)))
        o.tree_len = len(tree)
        C.memmove(b.taddr[i], tree, len(tree))
        st = o.stats
        st.candidates, st.unique, st.levels, st.n_ic, st.words = 1000 + i, 100 + i, 9, 40 + i, 2
        st.guide_pairs, st.ms_stage, st.ms_total, st.launches = 300 + i, 0.25 * i, 0.5 * i, i
        st.bytes_h2d, st.bytes_d2h, st.star_pairs = 7 * i, 11 * i, 3 * i
        for k in range(5):
            st.cand_op[k] = i * 10 + k
        st.ms_search_kernel, st.ms_stage_kernel, st.search_launches, st.grid = 0.125 * i, 0.0625 * i, 1 + i % 2, 152
    got = b.results()
    assert len(got) == n
    for i in range(n):
        want = rei._result(b.outs[i], b.outs[i].status, b.raddr[i], b.taddr[i])
        assert got[i] == want, i
    assert got[4].regex == "0*(14)?" and got[3].regex is None
