"""Seeded synthetic graph generators shared by the tests, the benchmark and the oracle tests.

This module only builds input graphs; it holds none of the graphlet-transform arithmetic.
Every generator returns a simple undirected graph (no self-loops, no multi-edges) as a
symmetric CSR with sorted neighbour lists:

    Graph(n, rowptr: int64[n+1], colidx: int32[rowptr[n]])

Vertex ids are 0-based. The paper numbers vertices from 1 (Sec. 1, notation paragraph);
only the labels differ.
"""
from __future__ import annotations

from typing import NamedTuple, Sequence

import numpy as np


class Graph(NamedTuple):
    n: int
    rowptr: np.ndarray  # int64[n+1]
    colidx: np.ndarray  # int32[nnz], nnz = 2m

    @property
    def m(self) -> int:
        return int(self.rowptr[-1]) // 2

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.rowptr)


def csr_from_pairs(n: int, src, dst) -> Graph:
    """Symmetrise, drop self-loops, deduplicate and sort an edge list into CSR."""
    src = np.asarray(src, dtype=np.int64).ravel()
    dst = np.asarray(dst, dtype=np.int64).ravel()
    keep = src != dst
    src, dst = src[keep], dst[keep]
    if n > 0 and src.size:
        if src.min() < 0 or dst.min() < 0 or src.max() >= n or dst.max() >= n:
            raise ValueError("vertex id out of range")
    keys = np.concatenate([src * n + dst, dst * n + src])
    keys.sort()
    if keys.size:
        keys = keys[np.concatenate([[True], keys[1:] != keys[:-1]])]
    rows = keys // max(n, 1)
    cols = (keys - rows * n).astype(np.int32)
    counts = np.bincount(rows, minlength=n) if n > 0 else np.zeros(0, np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return Graph(int(n), rowptr, cols)


def from_edge_list(n: int, edges: Sequence[Sequence[int]]) -> Graph:
    if len(edges) == 0:
        return csr_from_pairs(n, [], [])
    e = np.asarray(edges, dtype=np.int64)
    return csr_from_pairs(n, e[:, 0], e[:, 1])


# ---------------------------------------------------------------------------
# Small structured graphs (closed forms are known for these)
# ---------------------------------------------------------------------------

def empty(n: int) -> Graph:
    return csr_from_pairs(n, [], [])


def complete(n: int) -> Graph:
    i, j = np.triu_indices(n, k=1)
    return csr_from_pairs(n, i, j)


def star(k: int) -> Graph:
    """K_{1,k}: vertex 0 is the centre, 1..k the leaves."""
    return csr_from_pairs(k + 1, np.zeros(k, np.int64), np.arange(1, k + 1))


def path(n: int) -> Graph:
    i = np.arange(n - 1)
    return csr_from_pairs(n, i, i + 1)


def cycle(n: int) -> Graph:
    i = np.arange(n)
    return csr_from_pairs(n, i, (i + 1) % n)


# ---------------------------------------------------------------------------
# Random graph families
# ---------------------------------------------------------------------------

def erdos_renyi(n: int, avg_degree: float, seed: int) -> Graph:
    """G(n, p) with p = avg_degree / (n - 1): every unordered pair is an edge
    independently with probability p (one uniform draw per pair, pairs in
    row-major upper-triangle order)."""
    rng = np.random.default_rng(seed)
    p = avg_degree / max(n - 1, 1)
    i, j = np.triu_indices(n, k=1)
    keep = rng.random(i.size) < p
    return csr_from_pairs(n, i[keep], j[keep])


def rmat_pairs(scale: int, edge_factor: int, a: float, b: float, c: float,
               seed: int, permute: bool = True, chunk: int = 1 << 24):
    """Sample the 2^scale * edge_factor R-MAT (Kronecker) pairs.

    Each pair picks one quadrant per level with probabilities (a, b, c, d=1-a-b-c);
    the source takes the row bit and the destination the column bit. A seeded
    random vertex permutation is applied afterwards (Graph500 style) so that
    vertex id carries no degree information."""
    rng = np.random.default_rng(seed)
    n = 1 << scale
    total = n * edge_factor
    ab, abc = a + b, a + b + c
    srcs, dsts = [], []
    done = 0
    while done < total:
        cnt = min(chunk, total - done)
        s = np.zeros(cnt, dtype=np.int64)
        d = np.zeros(cnt, dtype=np.int64)
        for lvl in range(scale):
            r = rng.random(cnt, dtype=np.float64)
            bit = np.int64(1) << np.int64(scale - 1 - lvl)
            sbit = r >= ab
            dbit = ((r >= a) & (r < ab)) | (r >= abc)
            s += sbit * bit
            d += dbit * bit
        srcs.append(s)
        dsts.append(d)
        done += cnt
    src = np.concatenate(srcs)
    dst = np.concatenate(dsts)
    if permute:
        perm = rng.permutation(n).astype(np.int64)
        src = perm[src]
        dst = perm[dst]
    return n, src, dst


def rmat(scale: int, edge_factor: int, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 0, permute: bool = True) -> Graph:
    n, src, dst = rmat_pairs(scale, edge_factor, a, b, c, seed, permute)
    return csr_from_pairs(n, src, dst)


def _ba_pairs(n: int, m: int, seed: int):
    """Edge pairs of barabasi_albert (n > m).

    Preferential attachment (Barabasi-Albert): vertices m..n-1 arrive in
    order and each draws m targets with probability proportional to degree,
    i.e. uniformly from the list of all edge endpoints so far (the m initial
    vertices listed once each). Repeated draws of the same target merge into
    one edge. Vectorised: a draw that lands on the target end of an earlier
    edge takes that edge's target, resolved by pointer doubling."""
    rng = np.random.default_rng(seed)
    E = m * (n - m)
    e = np.arange(E, dtype=np.int64)
    src = m + e // m                          # the arriving vertex of draw e
    L = m + 2 * m * (src - m)                  # endpoint-list length before src arrives
    p = (rng.random(E) * L).astype(np.int64)
    q = p - m
    tgt = np.where(p < m, p, -1).astype(np.int64)
    is_src = (p >= m) & (q % 2 == 0)
    tgt[is_src] = m + (q[is_src] // 2) // m    # the arriving end of an earlier edge
    ref = np.where(tgt < 0, q // 2, e)         # the target end: copy that edge's target
    while True:
        todo = tgt < 0
        if not todo.any():
            break
        r = ref[todo]
        tgt[todo] = tgt[r]
        ref[todo] = ref[r]
    return src, tgt


def barabasi_albert(n: int, m: int, seed: int) -> Graph:
    """Barabasi-Albert graph with n vertices and m attachments per arriving vertex."""
    if n <= m:
        return complete(n)
    src, tgt = _ba_pairs(n, m, seed)
    return csr_from_pairs(n, src, tgt)


def _rgg_pairs(n: int, radius: float, seed: int):
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 2))
    try:
        from scipy.spatial import cKDTree
        pairs = cKDTree(pts).query_pairs(radius, output_type="ndarray")
        if pairs.size:
            return pairs[:, 0].astype(np.int64), pairs[:, 1].astype(np.int64)
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    except ImportError:
        i, j = np.triu_indices(n, k=1)
        dd = ((pts[i] - pts[j]) ** 2).sum(axis=1)
        keep = dd < radius * radius
        return i[keep], j[keep]


def random_geometric(n: int, radius: float, seed: int) -> Graph:
    """n points uniform in the unit square; an edge joins points closer than radius."""
    i, j = _rgg_pairs(n, radius, seed)
    return csr_from_pairs(n, i, j)


def rgg_radius(n: int, mean_degree: float = 8.0) -> float:
    return float(np.sqrt(mean_degree / (np.pi * max(n, 1))))


# ---------------------------------------------------------------------------
# Batches of small graphs, packed block-diagonally
# ---------------------------------------------------------------------------

class Batch(NamedTuple):
    graph: Graph             # block-diagonal union
    offsets: np.ndarray      # int64[num_graphs+1], first vertex of each graph


def dense_neighbourhoods(core: int, p: float, roots: Sequence[float], boosters: int, q: float,
                         seed: int) -> Graph:
    """A random graph G(core, p) on vertices 0..core-1, plus one root vertex per
    entry f of `roots`, joined to a random fraction f of the core, plus
    `boosters` vertices each joined to a random fraction q of the core (they
    raise the core's degrees above the roots', so that in degree order the
    roots' higher neighbours are exactly their core neighbours, and the
    subgraph induced on them is dense)."""
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(core, 1)
    keep = rng.random(iu.size) < p
    src, dst = [iu[keep]], [ju[keep]]
    v = core
    for f in roots:
        nb = np.flatnonzero(rng.random(core) < f)
        src.append(np.full(nb.size, v))
        dst.append(nb)
        v += 1
    for _ in range(boosters):
        nb = np.flatnonzero(rng.random(core) < q)
        src.append(np.full(nb.size, v))
        dst.append(nb)
        v += 1
    return csr_from_pairs(v, np.concatenate(src), np.concatenate(dst))


def pack_block_diagonal(graphs: Sequence[Graph]) -> Batch:
    ns = np.array([g.n for g in graphs], dtype=np.int64)
    offsets = np.zeros(len(graphs) + 1, dtype=np.int64)
    np.cumsum(ns, out=offsets[1:])
    n = int(offsets[-1])
    rowptr = np.zeros(n + 1, dtype=np.int64)
    cols = []
    base_e = 0
    for g, off in zip(graphs, offsets[:-1]):
        rowptr[off + 1: off + g.n + 1] = g.rowptr[1:] + base_e
        cols.append(g.colidx.astype(np.int64) + off)
        base_e += g.nnz
    colidx = (np.concatenate(cols) if cols else np.zeros(0, np.int64)).astype(np.int32)
    return Batch(Graph(n, rowptr, colidx), offsets)


def small_graph_batch(num_graphs: int, seed: int, n_lo: int = 10, n_hi: int = 500) -> Batch:
    """Graph g has n ~ U{n_lo..n_hi} and seed seed+g; even g are Barabasi-Albert with
    m ~ U{2..5}, odd g random-geometric with mean degree 8. Packed block-diagonally."""
    ns = np.zeros(num_graphs, np.int64)
    srcs, dsts = [], []
    off = 0
    for g in range(num_graphs):
        rng = np.random.default_rng(seed + g)
        n = int(rng.integers(n_lo, n_hi + 1))
        if g % 2 == 0:
            m = int(rng.integers(2, 6))
            if n <= m:
                i, j = np.triu_indices(n, k=1)
            else:
                i, j = _ba_pairs(n, m, seed + g)
        else:
            i, j = _rgg_pairs(n, rgg_radius(n), seed + g)
        srcs.append(np.asarray(i, np.int64) + off)
        dsts.append(np.asarray(j, np.int64) + off)
        ns[g] = n
        off += n
    offsets = np.zeros(num_graphs + 1, dtype=np.int64)
    np.cumsum(ns, out=offsets[1:])
    src = np.concatenate(srcs) if srcs else np.zeros(0, np.int64)
    dst = np.concatenate(dsts) if dsts else np.zeros(0, np.int64)
    return Batch(csr_from_pairs(int(offsets[-1]), src, dst), offsets)


def permute_vertices(g: Graph, perm: np.ndarray) -> Graph:
    """Relabel vertex v as perm[v]."""
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.rowptr))
    perm = np.asarray(perm, dtype=np.int64)
    return csr_from_pairs(g.n, perm[rows], perm[g.colidx.astype(np.int64)])


# ---------------------------------------------------------------------------
# Large R-MAT graphs generated on a CUDA device (scale 22-26): the host
# generator above needs tens of minutes and tens of GB for scale 24.
# ---------------------------------------------------------------------------

class DeviceGraph(NamedTuple):
    n: int
    rowptr: "object"  # torch int64[n+1] on the device
    colidx: "object"  # torch int32[nnz] on the device

    @property
    def nnz(self) -> int:
        return int(self.colidx.numel())

    @property
    def m(self) -> int:
        return self.nnz // 2

    def to_host(self) -> Graph:
        return Graph(self.n, self.rowptr.cpu().numpy(), self.colidx.cpu().numpy())


def rmat_device(scale: int, edge_factor: int, a: float = 0.57, b: float = 0.19, c: float = 0.19,
                seed: int = 0, device: str = "cuda", chunk: int = 1 << 26) -> DeviceGraph:
    """R-MAT graph of the same family as rmat() (quadrant per level with
    probabilities a, b, c, d = 1-a-b-c; seeded vertex permutation; self-loops
    dropped; symmetrised; deduplicated; sorted CSR), drawn with torch's
    counter-based device generator. The draws differ from rmat()'s for the same
    seed, so the two give different graphs of the same distribution. Rows are
    int64 row pointers and int32 column indices on the device."""
    import torch

    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    n = 1 << scale
    total = n * edge_factor
    ab, abc = a + b, a + b + c
    perm = torch.randperm(n, generator=gen, device=dev)
    keys = []
    done = 0
    while done < total:
        cnt = min(chunk, total - done)
        s = torch.zeros(cnt, dtype=torch.int64, device=dev)
        d = torch.zeros(cnt, dtype=torch.int64, device=dev)
        for lvl in range(scale):
            r = torch.rand(cnt, generator=gen, device=dev, dtype=torch.float64)
            bit = 1 << (scale - 1 - lvl)
            s += (r >= ab).to(torch.int64) * bit
            d += (((r >= a) & (r < ab)) | (r >= abc)).to(torch.int64) * bit
            del r
        s = perm[s]
        d = perm[d]
        keep = s != d
        s, d = s[keep], d[keep]
        keys.append(torch.unique(torch.cat([(s << scale) | d, (d << scale) | s])))
        del s, d, keep
        done += cnt
    k = torch.unique(torch.cat(keys)) if len(keys) > 1 else keys[0]
    del keys
    rows = k >> scale
    colidx = (k & (n - 1)).to(torch.int32)
    del k
    counts = torch.bincount(rows, minlength=n)
    del rows
    rowptr = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    torch.cumsum(counts, 0, out=rowptr[1:])
    return DeviceGraph(n, rowptr, colidx)
