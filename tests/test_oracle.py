"""Pins of the CPU oracle against values fixed by the paper and by mathematics.

None of these compare the oracle with itself: the references are the printed
worked example (Fig. 2), exhaustive enumeration of induced and non-induced
subgraphs (oracle/brute.py), closed forms, orbit-size invariants, and library
routines (networkx) for the special cases they cover.
"""
import itertools
from math import comb

import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle.brute import brute_fglt, edges_of
from conftest import read_golden_sections, read_hub_rows


def _fig2():
    sec = read_golden_sections("fig2_example.txt")
    edges = [(a - 1, b - 1) for a, b in sec["edges"]]
    raw = np.array([r[1:] for r in sec["raw"]], dtype=np.int64)
    net = np.array([r[1:] for r in sec["net"]], dtype=np.int64)
    return gg.from_edge_list(6, edges), edges, raw, net


def _random_small(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(4, 12))
    p = float(rng.uniform(0.15, 0.85))
    i, j = np.triu_indices(n, 1)
    keep = rng.random(i.size) < p
    return gg.csr_from_pairs(n, i[keep], j[keep])


# --------------------------------------------------------------------------
# Fig. 2 worked example (printed raw and net tables)
# --------------------------------------------------------------------------

def test_fig2_raw_and_net_tables():
    g, _, raw_ref, net_ref = _fig2()
    raw, net = oracle.fglt(g)
    np.testing.assert_array_equal(raw, raw_ref)
    np.testing.assert_array_equal(net, net_ref)


def test_fig2_observations():
    """Fig. 2 caption: f(v2) = f(v5); 5 triangles (sum d4 / 3); no 4-cycles; no claws."""
    g, _, _, _ = _fig2()
    _, net = oracle.fglt(g)
    np.testing.assert_array_equal(net[1], net[4])
    assert net[:, 4].sum() // 3 == 5
    assert net[:, 12].sum() == 0
    assert net[:, 7].sum() == 0 and net[:, 8].sum() == 0


def test_table2_golden_is_stored_table():
    ref = np.array(read_golden_sections("u16_table2.txt")[None], dtype=np.int64)
    np.testing.assert_array_equal(oracle.u16(), ref)


def test_table2_against_enumeration():
    """U16 f = f^ holds for brute-force raw and net counts (Table II vs mathematics)."""
    U = oracle.u16()
    for seed in range(40):
        g = _random_small(seed)
        raw, net = brute_fglt(g.n, edges_of(g))
        np.testing.assert_array_equal(net @ U.T, raw)


def test_inverse_has_same_pattern_integer():
    """Sec. 5: U16^{-1} has exactly the sparsity pattern of U16 (and is integer)."""
    U = oracle.u16()
    inv = oracle.raw_to_net(np.eye(16, dtype=np.int64)).T  # column k = U^{-1} e_k
    np.testing.assert_array_equal(U @ inv, np.eye(16, dtype=np.int64))
    np.testing.assert_array_equal(inv != 0, U != 0)
    assert int((U != 0).sum()) == 50


# --------------------------------------------------------------------------
# Brute-force enumeration on random tiny graphs
# --------------------------------------------------------------------------

@pytest.mark.parametrize("block", range(6))
def test_brute_force_random(block):
    for seed in range(block * 40, block * 40 + 40):
        g = _random_small(seed)
        raw_b, net_b = brute_fglt(g.n, edges_of(g))
        raw, net = oracle.fglt(g)
        np.testing.assert_array_equal(raw, raw_b, err_msg=f"seed {seed}")
        np.testing.assert_array_equal(net, net_b, err_msg=f"seed {seed}")


def test_brute_force_hub_graphs():
    """A hub joined to every other vertex (degree ratios above 8): the oracle's
    binary-search intersections against enumeration."""
    from test_oracle_mutants import hub_graph
    for seed in range(30):
        g = hub_graph(seed)
        deg = np.diff(g.rowptr)
        assert (deg.max() > 8 * deg[deg > 0]).any()
        raw_b, net_b = brute_fglt(g.n, edges_of(g))
        raw, net = oracle.fglt(g)
        np.testing.assert_array_equal(raw, raw_b)
        np.testing.assert_array_equal(net, net_b)


def test_brute_force_structured():
    cases = [gg.complete(5), gg.star(5), gg.path(6), gg.cycle(4), gg.cycle(6),
             gg.from_edge_list(5, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4)]),
             gg.empty(3)]
    for g in cases:
        raw_b, net_b = brute_fglt(g.n, edges_of(g))
        raw, net = oracle.fglt(g)
        np.testing.assert_array_equal(raw, raw_b)
        np.testing.assert_array_equal(net, net_b)


# --------------------------------------------------------------------------
# Closed forms
# --------------------------------------------------------------------------

def _vec(**kw):
    v = np.zeros(16, dtype=np.int64)
    v[0] = 1
    for k, x in kw.items():
        v[int(k[1:])] = x
    return v


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 12])
def test_complete_graph(n):
    _, net = oracle.fglt(gg.complete(n))
    want = _vec(d1=n - 1, d4=comb(n - 1, 2), d15=comb(n - 1, 3))
    for row in net:
        np.testing.assert_array_equal(row, want)


@pytest.mark.parametrize("k", [1, 2, 3, 6, 40])
def test_star(k):
    _, net = oracle.fglt(gg.star(k))
    np.testing.assert_array_equal(net[0], _vec(d1=k, d3=comb(k, 2), d8=comb(k, 3)))
    for row in net[1:]:
        np.testing.assert_array_equal(row, _vec(d1=1, d2=k - 1, d7=comb(k - 1, 2)))


@pytest.mark.parametrize("n", [5, 6, 9, 50])
def test_long_cycle(n):
    _, net = oracle.fglt(gg.cycle(n))
    for row in net:
        np.testing.assert_array_equal(row, _vec(d1=2, d2=2, d3=1, d5=2, d6=2))


def test_short_cycles():
    _, net = oracle.fglt(gg.cycle(4))
    for row in net:
        np.testing.assert_array_equal(row, _vec(d1=2, d2=2, d3=1, d12=1))
    _, net = oracle.fglt(gg.cycle(3))
    for row in net:
        np.testing.assert_array_equal(row, _vec(d1=2, d4=1))


def test_path8():
    _, net = oracle.fglt(gg.path(8))
    want = [_vec(d1=1, d2=1, d5=1), _vec(d1=2, d2=1, d3=1, d5=1, d6=1),
            _vec(d1=2, d2=2, d3=1, d5=1, d6=2), _vec(d1=2, d2=2, d3=1, d5=2, d6=2)]
    for v in range(4):
        np.testing.assert_array_equal(net[v], want[v])
        np.testing.assert_array_equal(net[7 - v], want[v])


def test_isolated_and_empty():
    raw, net = oracle.fglt(gg.empty(5))
    for row in np.concatenate([raw, net]):
        np.testing.assert_array_equal(row, _vec())
    raw, net = oracle.fglt(gg.empty(0))
    assert raw.shape == (0, 16) and net.shape == (0, 16)


# --------------------------------------------------------------------------
# Invariants on medium graphs
# --------------------------------------------------------------------------

def _medium_graphs():
    return [gg.erdos_renyi(300, 12, seed=1), gg.rmat(10, 8, seed=3),
            gg.barabasi_albert(400, 4, seed=5), gg.random_geometric(400, gg.rgg_radius(400, 12), seed=7)]


def test_orbit_sum_identities():
    """Orbit sizes of Fig. 1: each induced copy adds its orbit multiplicities."""
    for g in _medium_graphs():
        raw, net = oracle.fglt(g)
        s = net.sum(axis=0)
        assert s[1] == 2 * g.m
        assert s[2] == 2 * s[3]
        assert s[4] % 3 == 0
        assert s[5] == s[6]
        assert s[7] == 3 * s[8]
        assert s[10] == 2 * s[9] and s[9] == s[11]
        assert s[12] % 4 == 0
        assert s[13] == s[14]
        assert s[15] % 4 == 0
        assert (net >= 0).all()
        np.testing.assert_array_equal(net @ oracle.u16().T, raw)


def test_networkx_triangles_cycles_cliques():
    nx = pytest.importorskip("networkx")
    for g in [gg.erdos_renyi(60, 9, seed=11), gg.rmat(7, 6, seed=2), gg.complete(7)]:
        G = nx.Graph()
        G.add_nodes_from(range(g.n))
        G.add_edges_from(edges_of(g))
        raw, _ = oracle.fglt(g)
        tri = nx.triangles(G)
        np.testing.assert_array_equal(raw[:, 4], [tri[v] for v in range(g.n)])
        c4 = np.zeros(g.n, np.int64)
        for cyc in nx.simple_cycles(G, length_bound=4):
            if len(cyc) == 4:
                for v in cyc:
                    c4[v] += 1
        np.testing.assert_array_equal(raw[:, 12], c4)
        k4 = np.zeros(g.n, np.int64)
        for cl in nx.enumerate_all_cliques(G):
            if len(cl) == 4:
                for v in cl:
                    k4[v] += 1
            elif len(cl) > 4:
                break
        np.testing.assert_array_equal(raw[:, 15], k4)
        np.testing.assert_array_equal(raw[:, 1], [G.degree(v) for v in range(g.n)])


def test_permutation_equivariance():
    g = gg.rmat(9, 8, seed=4)
    rng = np.random.default_rng(0)
    perm = rng.permutation(g.n)
    h = gg.permute_vertices(g, perm)
    raw_g, net_g = oracle.fglt(g)
    raw_h, net_h = oracle.fglt(h)
    np.testing.assert_array_equal(raw_h[perm], raw_g)
    np.testing.assert_array_equal(net_h[perm], net_g)


def test_disjoint_union_is_concatenation():
    parts = [gg.erdos_renyi(50, 6, seed=s) for s in range(3)] + [gg.complete(6), gg.empty(2)]
    batch = gg.pack_block_diagonal(parts)
    raw_u, net_u = oracle.fglt(batch.graph)
    for k, p in enumerate(parts):
        raw_p, net_p = oracle.fglt(p)
        lo, hi = batch.offsets[k], batch.offsets[k + 1]
        np.testing.assert_array_equal(raw_u[lo:hi], raw_p)
        np.testing.assert_array_equal(net_u[lo:hi], net_p)


def test_vertex_subset_rows_match_full():
    """The sampled mode computes C3 only around the requested rows; every
    requested row must equal the full computation's (hubs, leaves, repeats)."""
    g = gg.rmat(10, 8, seed=9)
    raw, net = oracle.fglt(g)
    verts = np.array([0, 5, g.n - 1, 17, 17, 300])
    raw_s, net_s = oracle.fglt(g, vertices=verts)
    np.testing.assert_array_equal(raw_s, raw[verts])
    np.testing.assert_array_equal(net_s, net[verts])
    # a hub-heavy graph: degree ratios far above 8 take the binary-search intersection
    h = gg.rmat(12, 16, seed=4)
    raw, net = oracle.fglt(h)
    deg = np.diff(h.rowptr)
    rng = np.random.default_rng(7)
    for verts in (np.argsort(deg)[-5:], rng.integers(0, h.n, 30), np.array([int(np.argmax(deg))])):
        raw_s, net_s = oracle.fglt(h, vertices=verts)
        np.testing.assert_array_equal(raw_s, raw[verts])
        np.testing.assert_array_equal(net_s, net[verts])


def test_threads_do_not_change_result():
    g = gg.rmat(11, 8, seed=1)
    a = oracle.fglt(g, threads=1)
    b = oracle.fglt(g, threads=4)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


# --------------------------------------------------------------------------
# Sub-dictionaries (Table II caption: s has the conversion matrix U16(s,s))
# --------------------------------------------------------------------------

def _golden_u16():
    return np.array(read_golden_sections("u16_table2.txt")[None], dtype=np.int64)


def _closed(mask, U):
    """s is closed when every graphlet that raw rows in s count (U[k][l] != 0)
    is itself in s; then the induced counts of s need no graphlet outside s."""
    s = [k for k in range(16) if (mask >> k) & 1]
    return all((mask >> l) & 1 for k in s for l in range(16) if U[k, l])


CLOSED = [0x1F, 0x13, 0x3, 0x1 | 0x2 | (1 << 8) | (1 << 11) | (1 << 14) | (1 << 15),
          0x3 | (1 << 12) | (1 << 13) | (1 << 14) | (1 << 15), 0x3 | (1 << 15)]


def test_sub_dictionary_closed_sets_are_induced_counts():
    """For a closed s (Sigma5 among them), net(s) are the induced orbit counts
    of the graphlets in s: brute-force enumeration, no Table I or II."""
    U = _golden_u16()
    for mask in CLOSED:
        assert _closed(mask, U), hex(mask)
    cols = lambda m: [k for k in range(16) if (m >> k) & 1]  # noqa: E731
    for seed in range(60):
        g = _random_small(seed)
        raw_b, net_b = brute_fglt(g.n, edges_of(g))
        for mask in CLOSED:
            raw, net = oracle.fglt(g, dictionary=mask)
            np.testing.assert_array_equal(raw, raw_b[:, cols(mask)], err_msg=f"{hex(mask)} seed {seed}")
            np.testing.assert_array_equal(net, net_b[:, cols(mask)], err_msg=f"{hex(mask)} seed {seed}")


def test_sigma5_fig2_tables():
    """Sigma5 on the Fig. 2 example: the first five columns of both printed tables."""
    g, _, raw_ref, net_ref = _fig2()
    raw, net = oracle.fglt(g, dictionary=0x1F)
    np.testing.assert_array_equal(raw, raw_ref[:, :5])
    np.testing.assert_array_equal(net, net_ref[:, :5])


def test_sub_dictionary_any_set_solves_its_conversion():
    """Any s containing {0,1}: U16(s,s) net(s) = raw(s), with U16 from the
    golden Table II and raw from brute-force enumeration."""
    U = _golden_u16()
    rng = np.random.default_rng(5)
    masks = [0x3 | (int(rng.integers(0, 1 << 14)) << 2) for _ in range(25)] + [0x3 | (1 << 5), 0x3 | (1 << 12)]
    for seed in range(12):
        g = _random_small(100 + seed)
        raw_b, _ = brute_fglt(g.n, edges_of(g))
        for mask in masks:
            s = [k for k in range(16) if (mask >> k) & 1]
            raw, net = oracle.fglt(g, dictionary=mask)
            np.testing.assert_array_equal(raw, raw_b[:, s])
            np.testing.assert_array_equal(net @ U[np.ix_(s, s)].T, raw)


def test_sub_dictionary_rejects_sets_without_sigma0_sigma1():
    g = gg.complete(4)
    for mask in (0x1, 0x2, 0x1C, 1 << 16 | 0x3):
        with pytest.raises(ValueError):
            oracle.fglt(g, dictionary=mask)


def test_stored_hub_rows_are_consistent():
    """The stored oracle rows of R-MAT scale 20's top-degree vertices belong to
    the generator's current graph, are those of its 16 largest degrees, and
    satisfy raw = U16 net, net >= 0 and d1 = degree."""
    import os
    import sys
    sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
    from make_hub_rows import csr_digest, top_degree_vertices
    head, rows = read_hub_rows("hub_rows_rmat-s20-ef16.txt")
    g = gg.rmat(20, 16, seed=0)
    assert head["sha256"] == csr_digest(g.rowptr, g.colidx)
    assert [v for v, _, _ in rows] == list(top_degree_vertices(g.rowptr, 16))
    u = oracle.u16()
    deg = np.diff(g.rowptr)
    for v, raw, net in rows:
        assert raw[0] == 1 and raw[1] == deg[v]
        assert (net >= 0).all()
        np.testing.assert_array_equal(u @ net, raw)


def test_table1_local_terms_match_the_oracle():
    """The definition-based columns used for the largest hubs of the full-size
    graph (tests/conftest.py) agree with the oracle's raw rows, on the hubs and
    on low-degree vertices of a power-law graph and on small special graphs,
    with a chunk size small enough that the gathers are split."""
    torch = pytest.importorskip("torch")
    from conftest import TABLE1_LOCAL_COLUMNS, table1_local_terms
    for g in (gg.rmat(11, 16, seed=3), gg.complete(40), gg.star(30)):
        deg = np.diff(g.rowptr)
        verts = np.unique(np.concatenate([np.argsort(-deg, kind="stable")[:4], np.flatnonzero(deg == 1)[:2],
                                          np.flatnonzero(deg == 0)[:1]]))
        raw, _ = oracle.fglt(g, vertices=verts)
        rp = torch.from_numpy(g.rowptr.astype(np.int64))
        ci = torch.from_numpy(g.colidx.astype(np.int32))
        for row, v in zip(raw, verts):
            t = table1_local_terms(rp, ci, int(v), chunk=97)
            for c in TABLE1_LOCAL_COLUMNS:
                assert t[c] == row[c], (g.n, int(v), c, t[c], row[c])


def test_spmv_chain_relations_hold_on_the_oracle():
    """The per-row relations the full-size GPU test checks on every row
    (Sec. 4.2: d2 = A (p1 - 1), d7 = A C(p1 - 1, 2), d5 = A d2 - p1 (p1 - 1) - 2 d4,
    d9 = A d4 - 2 d4) hold on the oracle's rows of power-law and random graphs."""
    for g in (gg.rmat(10, 8, seed=1), gg.erdos_renyi(300, 6, seed=2), gg.barabasi_albert(400, 4, seed=3)):
        raw, _ = oracle.fglt(g)
        deg = np.diff(g.rowptr).astype(np.int64)
        rows = np.repeat(np.arange(g.n), deg)
        nbr = g.colidx.astype(np.int64)

        def spmv(x):  # (A x)_i = sum of x over N(i)
            out = np.zeros(g.n, dtype=np.int64)
            np.add.at(out, rows, x[nbr])
            return out

        p1 = deg
        np.testing.assert_array_equal(raw[:, 2], spmv(p1 - 1))
        np.testing.assert_array_equal(raw[:, 7], spmv((p1 - 1) * (p1 - 2) // 2))
        np.testing.assert_array_equal(raw[:, 5], spmv(raw[:, 2]) - p1 * (p1 - 1) - 2 * raw[:, 4])
        np.testing.assert_array_equal(raw[:, 9], spmv(raw[:, 4]) - 2 * raw[:, 4])
