import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU check")


def _word(tok: str) -> bytes:
    return b"" if tok == "_" else tok.encode()


def load_golden(name: str) -> dict:
    """Parse a tests/golden fixture: 'key: words' lines and tagged rows."""
    out = {"rows": []}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith(("P:", "N:", "words:")):
                k, v = line.split(":", 1)
                out[k] = [_word(t) for t in v.split()]
            elif line.startswith("lang "):
                k, v = line[5:].split(":", 1)
                out.setdefault("lang", {})[k.strip()] = [_word(t) for t in v.split()]
            else:
                out["rows"].append(line.split())
    return out


@pytest.fixture(scope="session")
def golden():
    return load_golden


def load_expected(name: str):
    """Rows of a stored-oracle-results fixture (written by a script under
    tests/golden that calls only the oracle): seed -> (status, cost,
    candidates, unique, n_ic, tree)."""
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            sd, st, cost, cand, uniq, n_ic, *tree = line.split()
            rows[int(sd)] = (int(st), int(cost), int(cand), int(uniq), int(n_ic),
                             bytes.fromhex(tree[0]) if tree else b"")
    return rows
