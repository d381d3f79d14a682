import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


GOLDEN = os.path.join(ROOT, "tests", "golden")


def read_golden_sections(name):
    """Parse a golden text file with [section] headers and '#' comments."""
    out, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("[") and line.endswith("]"):
                cur = line[1:-1]
                out[cur] = []
                continue
            out.setdefault(cur, []).append([int(x) for x in line.split()])
    return out


def read_hub_rows(name):
    """Stored oracle rows of a graph's top-degree vertices (written by
    tests/golden/make_hub_rows.py): header values, then per vertex its id,
    raw row and net row."""
    import numpy as np
    head, rows = {}, []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "vertex":
                rows.append([int(t[1]), None, None])
            elif t[0] in ("raw", "net"):
                rows[-1][1 if t[0] == "raw" else 2] = np.array([int(x) for x in t[1:]], dtype=np.int64)
            else:
                head[t[0]] = t[1]
    return head, rows
