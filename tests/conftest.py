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


# Table I columns whose definitions need only a vertex's neighbourhood and its
# neighbours' lists (degrees, 2-paths, triangles on each incident edge):
# d1 = p1, d2 = p2, d3 = C(p1, 2), d4 = c3, d5 = p3, d6 = p2 (p1 - 1) - 2 c3,
# d7 = [A ((p1 - 1) o (p1 - 2)) / 2], d8 = C(p1, 3), d10 = [C3 (p1 - 2)],
# d11 = (p1 - 2) c3, d14 = [D4,3 e / 2] (Table I, Sec. 4.2-4.3).
TABLE1_LOCAL_COLUMNS = (1, 2, 3, 4, 5, 6, 7, 8, 10, 11, 14)


def table1_local_terms(rowptr, colidx, v, chunk=1 << 26):
    """The TABLE1_LOCAL_COLUMNS of vertex v's raw row, from the definitions,
    with plain torch tensor operations (CPU or CUDA tensors; rowptr int64,
    colidx int32 or int64). The neighbours' lists are gathered in chunks of
    at most `chunk` entries: per neighbour u, C3(v, u) = |N(u) ∩ N(v)| and the
    sum of the degrees over N(u)."""
    import torch
    dev = rowptr.device
    n = rowptr.numel() - 1
    d = rowptr[1:] - rowptr[:-1]
    b, e = int(rowptr[v]), int(rowptr[v + 1])
    nb = colidx[b:e].long()
    mask = torch.zeros(n, dtype=torch.bool, device=dev)
    mask[nb] = True
    du = d[nb]
    c3u = torch.zeros_like(du)
    s2u = torch.zeros_like(du)
    ends = torch.cumsum(du, 0)
    i0 = 0
    while i0 < nb.numel():
        base = int(ends[i0 - 1]) if i0 > 0 else 0
        i1 = int(torch.searchsorted(ends, torch.tensor(base + chunk, device=dev), right=True))
        i1 = max(i1, i0 + 1)
        lens = du[i0:i1]
        total = int(lens.sum())
        if total:
            excl = torch.cumsum(lens, 0) - lens
            idx = torch.repeat_interleave(rowptr[nb[i0:i1]] - excl, lens) + torch.arange(total, device=dev)
            w = colidx[idx].long()
            seg = torch.repeat_interleave(torch.arange(i1 - i0, device=dev), lens)
            c3u[i0:i1] = torch.zeros(i1 - i0, dtype=torch.int64, device=dev).index_add_(0, seg, mask[w].long())
            s2u[i0:i1] = torch.zeros(i1 - i0, dtype=torch.int64, device=dev).index_add_(0, seg, d[w])
        i0 = i1
    p1 = e - b
    p2 = int((du - 1).sum())
    twice_c3 = int(c3u.sum())
    assert twice_c3 % 2 == 0
    c3 = twice_c3 // 2
    p3 = int((s2u - du).sum()) - p1 * (p1 - 1) - 2 * c3
    return {
        1: p1, 2: p2, 3: p1 * (p1 - 1) // 2, 4: c3, 5: p3, 6: p2 * (p1 - 1) - 2 * c3,
        7: int(((du - 1) * (du - 2) // 2).sum()), 8: p1 * (p1 - 1) * (p1 - 2) // 6,
        10: int((c3u * (du - 2)).sum()), 11: (p1 - 2) * c3, 14: int((c3u * (c3u - 1) // 2).sum()),
    }
