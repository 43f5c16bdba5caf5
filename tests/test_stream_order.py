"""Every device operation of the library is ordered on one of its streams.

The context's stream and the served form's launch stream are created
non-blocking, so work on the legacy default stream (cudaMemset, cudaMemcpy and
the like without a stream) is not ordered against them: a buffer emptied that
way can still hold its previous contents when the next launch reads it.  The
served form's slot tables were once emptied like that, and its first searches
could read stale entries.  This check keeps such calls out of the library's
sources (the separate peak probe, which runs on the default stream alone, is
not part of the library).
"""
import os
import re

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2305_18575_gb300", "csrc")
LEGACY = re.compile(r"\bcuda(Memset|Memcpy|Memset2D|Memcpy2D|MemcpyToSymbol|MemcpyFromSymbol)\s*\(")


def library_sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h")) and f != "peak.cu")


@pytest.mark.parametrize("name", library_sources())
def test_no_legacy_stream_copies_or_sets(name):
    with open(os.path.join(CSRC, name)) as fh:
        text = fh.read()
    hits = [m.group(0) for m in LEGACY.finditer(text)]
    assert not hits, f"{name}: {hits}"


def test_server_setup_waits_for_its_emptying():
    with open(os.path.join(CSRC, "host.cu")) as fh:
        text = fh.read()
    body = text[text.index("rei_status server_setup("):]
    body = body[: body.index("\n}\n")]
    sets = [m.start() for m in re.finditer(r"cudaMemsetAsync\([^;]*S->kstream\)", body)]
    assert len(sets) >= 3  # tables, bitmaps, queue heads
    assert body.find("cudaStreamSynchronize(S->kstream)") > max(sets)
