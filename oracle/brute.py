"""Brute-force graphlet frequencies on tiny graphs (pure Python).

TEST INFRASTRUCTURE ONLY. Independent of both the C oracle and the CUDA path:
it uses neither Table I nor Table II. It enumerates every vertex set S of size
1..4 (the naive enumeration the paper mentions in Sec. 1) and, for each S,

  * every edge subset F of the induced edges E(S) that connects S -> raw counts
    (a raw frequency counts sigma-pattern subgraphs, induced or not, Sec. 4), and
  * the induced edge set F = E(S) alone -> net counts (for the complete
    families of Sigma16 the net frequency is the induced count, Sec. 4).

Each connected (S, F) is classified into sigma_0..sigma_15 and the orbit of every
vertex of S is read off its degree inside F, following the dictionary of Fig. 1
and the names in Table I:

  |S|=1                    : sigma0
  |S|=2, 1 edge            : sigma1 (either end)
  |S|=3, 2 edges (2-path)  : ends sigma2, middle (bi-fork root) sigma3
  |S|=3, 3 edges (triangle): sigma4
  |S|=4, 3 edges, a degree-3 vertex (claw): leaves sigma7, centre sigma8
  |S|=4, 3 edges otherwise (3-path): ends sigma5, interior sigma6
  |S|=4, 4 edges, all degree 2 (4-cycle): sigma12
  |S|=4, 4 edges otherwise (paw): handle tip (deg 1) sigma9, base (deg 2) sigma10,
                                  centre (deg 3) sigma11
  |S|=4, 5 edges (diamond): off-cord (deg 2) sigma13, on-cord (deg 3) sigma14
  |S|=4, 6 edges (K4): sigma15
"""
from __future__ import annotations

from itertools import combinations

import numpy as np


def _connected(verts, edges) -> bool:
    verts = list(verts)
    adj = {v: [] for v in verts}
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    seen = {verts[0]}
    stack = [verts[0]]
    while stack:
        x = stack.pop()
        for y in adj[x]:
            if y not in seen:
                seen.add(y)
                stack.append(y)
    return len(seen) == len(verts)


def _orbits(verts, edges):
    """Return {vertex: sigma index} for a connected pattern (verts, edges)."""
    deg = {v: 0 for v in verts}
    for a, b in edges:
        deg[a] += 1
        deg[b] += 1
    k, m = len(verts), len(edges)
    if k == 1:
        return {v: 0 for v in verts}
    if k == 2:
        return {v: 1 for v in verts}
    if k == 3:
        if m == 2:
            return {v: (3 if deg[v] == 2 else 2) for v in verts}
        return {v: 4 for v in verts}
    # k == 4
    if m == 3:
        if max(deg.values()) == 3:
            return {v: (8 if deg[v] == 3 else 7) for v in verts}
        return {v: (6 if deg[v] == 2 else 5) for v in verts}
    if m == 4:
        if all(x == 2 for x in deg.values()):
            return {v: 12 for v in verts}
        return {v: {1: 9, 2: 10, 3: 11}[deg[v]] for v in verts}
    if m == 5:
        return {v: (14 if deg[v] == 3 else 13) for v in verts}
    return {v: 15 for v in verts}


def brute_fglt(n: int, edges):
    """Raw and net frequencies by exhaustive enumeration; int64 [n, 16]."""
    adj = [set() for _ in range(n)]
    for a, b in edges:
        if a != b:
            adj[a].add(b)
            adj[b].add(a)
    raw = np.zeros((n, 16), dtype=np.int64)
    net = np.zeros((n, 16), dtype=np.int64)
    for k in range(1, 5):
        for S in combinations(range(n), k):
            ES = [(a, b) for a, b in combinations(S, 2) if b in adj[a]]
            if len(ES) < k - 1:
                continue
            # raw: every connected spanning edge subset of the induced edges
            for r in range(k - 1, len(ES) + 1):
                for F in combinations(ES, r):
                    if k > 1 and not _connected(S, F):
                        continue
                    for v, s in _orbits(S, F).items():
                        raw[v, s] += 1
            # net: the induced subgraph itself, if connected
            if k == 1 or _connected(S, ES):
                for v, s in _orbits(S, ES).items():
                    net[v, s] += 1
    return raw, net


def edges_of(graph):
    """Undirected edge list (i < j) of a CSR graph."""
    out = []
    for i in range(graph.n):
        for e in range(int(graph.rowptr[i]), int(graph.rowptr[i + 1])):
            j = int(graph.colidx[e])
            if i < j:
                out.append((i, j))
    return out
