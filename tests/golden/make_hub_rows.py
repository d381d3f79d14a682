#!/usr/bin/env python3
"""Writes the oracle's raw and net rows of the highest-degree vertices of a
seeded benchmark graph to tests/golden/hub_rows_<workload>.txt.

The rows come from the CPU oracle alone (``oracle.fglt`` in sampled mode:
Table I on the closed neighbourhoods of the requested vertices, then Table II);
the graph comes from the seeded input generators. Nothing here touches the
CUDA library. The file records a SHA-256 digest of the graph's CSR arrays, so
a test can check that it compares against the same graph.

Usage: python tests/golden/make_hub_rows.py [--top 16] [--threads 0]
(R-MAT scale 20, edge factor 16, seed 0; about half an hour on 8 cores).
"""
from __future__ import annotations

import argparse
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402


def csr_digest(rowptr: np.ndarray, colidx: np.ndarray) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(rowptr, dtype=np.int64).tobytes())
    h.update(np.ascontiguousarray(colidx, dtype=np.int32).tobytes())
    return h.hexdigest()


def top_degree_vertices(rowptr: np.ndarray, k: int) -> np.ndarray:
    """The k vertices of largest degree, ties broken by the smaller id."""
    deg = np.diff(rowptr)
    order = np.lexsort((np.arange(deg.size), -deg))
    return np.sort(order[:k]).astype(np.int64)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--top", type=int, default=16)
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args()
    g = gg.rmat(20, 16, seed=0)
    verts = top_degree_vertices(g.rowptr, args.top)
    t0 = time.time()
    raw, net = oracle.fglt(g, vertices=verts, threads=args.threads)
    dt = time.time() - t0
    deg = np.diff(g.rowptr)
    path = os.path.join(HERE, "hub_rows_rmat-s20-ef16.txt")
    with open(path, "w") as f:
        f.write("# Oracle rows (raw then net, Sigma16 columns d0..d15) of the top-degree vertices of\n")
        f.write("# R-MAT scale 20, edge factor 16, a=.57 b=.19 c=.19, seed 0 (graphgen.rmat).\n")
        f.write(f"# Written by tests/golden/make_hub_rows.py --top {args.top} ({dt:.0f} s of oracle time).\n")
        f.write(f"n {g.n}\nnnz {g.nnz}\nsha256 {csr_digest(g.rowptr, g.colidx)}\n")
        for r, v in enumerate(verts):
            f.write(f"vertex {v} degree {deg[v]}\n")
            f.write("raw " + " ".join(str(x) for x in raw[r]) + "\n")
            f.write("net " + " ".join(str(x) for x in net[r]) + "\n")
    print(f"wrote {path}: {len(verts)} rows in {dt:.0f} s")


if __name__ == "__main__":
    main()
