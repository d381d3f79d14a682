"""GPU path vs the CPU oracle, element by element (all counts are integers:
the bar is bit-exact). Every call goes through the C ABI (libfglt.so)."""
from math import comb

import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle.brute import brute_fglt, edges_of
from conftest import read_golden_sections, read_hub_rows

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def handle():
    import paper_2007_11111_gb300 as fg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    h = fg.Handle(device=0, validate=False)
    yield h
    h.close()


def gpu(handle, g, rp64=True):
    dev = torch.device("cuda:0")
    rp = torch.from_numpy(g.rowptr.astype(np.int64 if rp64 else np.int32)).to(dev)
    ci = torch.from_numpy(g.colidx if g.colidx.size else np.zeros(1, np.int32)).to(dev)
    raw, net = handle.transform(rp, ci, g.n)
    return raw.cpu().numpy(), net.cpu().numpy()


def assert_same(got, want, what=""):
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        r, c = bad[0]
        raise AssertionError(f"{what}: {len(bad)} mismatches; first at vertex {r} column {c}: "
                             f"got {got[r, c]} want {want[r, c]}")


def check_vs_oracle(handle, g, what, rp64=True):
    raw, net = gpu(handle, g, rp64)
    oraw, onet = oracle.fglt(g)
    assert_same(raw, oraw, what + " raw")
    assert_same(net, onet, what + " net")


def test_fig2_tables(handle):
    sec = read_golden_sections("fig2_example.txt")
    g = gg.from_edge_list(6, [(a - 1, b - 1) for a, b in sec["edges"]])
    raw, net = gpu(handle, g)
    assert_same(raw, np.array([r[1:] for r in sec["raw"]]), "fig2 raw")
    assert_same(net, np.array([r[1:] for r in sec["net"]]), "fig2 net")


@pytest.mark.parametrize("rp64", [True, False])
def test_random_small_graphs(handle, rp64):
    for seed in range(60):
        rng = np.random.default_rng(seed)
        n = int(rng.integers(2, 40))
        i, j = np.triu_indices(n, 1)
        keep = rng.random(i.size) < rng.uniform(0.05, 0.9)
        g = gg.csr_from_pairs(n, i[keep], j[keep])
        check_vs_oracle(handle, g, f"seed {seed}", rp64)


def test_brute_force_tiny(handle):
    for seed in range(30):
        rng = np.random.default_rng(500 + seed)
        n = int(rng.integers(3, 10))
        i, j = np.triu_indices(n, 1)
        keep = rng.random(i.size) < rng.uniform(0.2, 0.9)
        g = gg.csr_from_pairs(n, i[keep], j[keep])
        raw, net = gpu(handle, g)
        braw, bnet = brute_fglt(g.n, edges_of(g))
        assert_same(raw, braw, f"brute raw {seed}")
        assert_same(net, bnet, f"brute net {seed}")


def test_degenerate_inputs(handle):
    for g in [gg.empty(1), gg.empty(7), gg.path(2), gg.path(3), gg.complete(3), gg.star(1),
              gg.from_edge_list(5, [(0, 1)]), gg.complete(4)]:
        check_vs_oracle(handle, g, f"n={g.n} m={g.m}")


def test_c1_erdos_renyi(handle):
    """ER G(n=2000, avg degree 10), seed 0."""
    g = gg.erdos_renyi(2000, 10, seed=0)
    check_vs_oracle(handle, g, "ER 2000", rp64=False)
    check_vs_oracle(handle, g, "ER 2000", rp64=True)


@pytest.mark.parametrize("scale,ef,seed", [(8, 8, 1), (10, 16, 2), (12, 16, 3), (14, 8, 4)])
def test_rmat_vs_oracle(handle, scale, ef, seed):
    g = gg.rmat(scale, ef, seed=seed)
    check_vs_oracle(handle, g, f"rmat s{scale} ef{ef}")


def test_small_graph_families(handle):
    for seed in range(4):
        check_vs_oracle(handle, gg.barabasi_albert(300, 2 + seed, seed), f"BA {seed}")
        check_vs_oracle(handle, gg.random_geometric(300, gg.rgg_radius(300, 12), seed), f"RGG {seed}")


def test_heavy_rows_and_boundaries(handle):
    """Degrees around the 8-lane / whole-block switch (512), out-degrees around the
    register / shared-memory sort switch (32), stars with large centres."""
    for k in [31, 32, 33, 511, 512, 513, 2000]:
        check_vs_oracle(handle, gg.star(k), f"star {k}")
    for n in [31, 32, 33, 34, 65, 100]:
        check_vs_oracle(handle, gg.complete(n), f"K{n}")
    # a hub attached to a denser random graph
    base = gg.erdos_renyi(1500, 30, seed=9)
    rows = np.repeat(np.arange(base.n), np.diff(base.rowptr))
    hub = base.n
    src = np.concatenate([rows, np.full(base.n, hub)])
    dst = np.concatenate([base.colidx.astype(np.int64), np.arange(base.n)])
    check_vs_oracle(handle, gg.csr_from_pairs(base.n + 1, src, dst), "hub+ER")


@pytest.mark.parametrize("n", [700, 1300])
def test_large_cliques_closed_form(handle, n):
    """K_n: net f = [1, n-1, 0, 0, C(n-1,2), 0 ... 0, C(n-1,3)] (out-degrees up to
    n-1 exercise the global-memory adjacency bitmap above ~1100)."""
    raw, net = gpu(handle, gg.complete(n))
    want = np.zeros(16, np.int64)
    want[0], want[1], want[4], want[15] = 1, n - 1, comb(n - 1, 2), comb(n - 1, 3)
    assert_same(net, np.tile(want, (n, 1)), f"K{n}")
    # raw = U16 net (Table II)
    assert_same(raw, net @ oracle.u16().T, f"K{n} raw")


def complete_bipartite(a, b):
    i, j = np.meshgrid(np.arange(a), np.arange(a, a + b), indexing="ij")
    return gg.csr_from_pairs(a + b, i.ravel(), j.ravel())


@pytest.mark.parametrize("a,b", [(3, 4), (40, 60), (1500, 1500)])
def test_complete_bipartite_closed_form(handle, a, b):
    """K_{a,b}, vertex on the a-side: d1=b, d2=b(a-1), d3=C(b,2), d7=b C(a-1,2),
    d8=C(b,3), d12=(a-1) C(b,2); everything else 0 (induced counts; the side is
    independent). Equal degrees make every vertex a wedge source with many
    distinct tops (4-cycle hash tables in global memory)."""
    raw, net = gpu(handle, complete_bipartite(a, b))

    def row(x, y):
        v = np.zeros(16, np.int64)
        v[0], v[1], v[2], v[3] = 1, y, y * (x - 1), comb(y, 2)
        v[7], v[8], v[12] = y * comb(x - 1, 2), comb(y, 3), (x - 1) * comb(y, 2)
        return v

    assert_same(net[:a], np.tile(row(a, b), (a, 1)), "a side")
    assert_same(net[a:], np.tile(row(b, a), (b, 1)), "b side")
    assert_same(raw, net @ oracle.u16().T, "raw = U16 net")


def test_output_pointers_optional(handle):
    import paper_2007_11111_gb300 as fg
    g = gg.rmat(9, 8, seed=7)
    oraw, onet = oracle.fglt(g)
    dev = torch.device("cuda:0")
    rp = torch.from_numpy(g.rowptr).to(dev)
    ci = torch.from_numpy(g.colidx).to(dev)
    raw = torch.zeros((g.n, 16), dtype=torch.int64, device=dev)
    fg.fglt_transform(handle.h, rp, 1, ci, g.n, raw, None)
    assert_same(raw.cpu().numpy(), oraw, "raw only")
    net = torch.zeros((g.n, 16), dtype=torch.int64, device=dev)
    fg.fglt_transform(handle.h, rp, 1, ci, g.n, None, net)
    assert_same(net.cpu().numpy(), onet, "net only")


def test_user_stream(handle):
    g = gg.rmat(10, 8, seed=8)
    oraw, onet = oracle.fglt(g)
    s = torch.cuda.Stream()
    dev = torch.device("cuda:0")
    with torch.cuda.stream(s):
        rp = torch.from_numpy(g.rowptr).to(dev)
        ci = torch.from_numpy(g.colidx).to(dev)
        raw, net = handle.transform(rp, ci, g.n, stream=s)
    s.synchronize()
    assert_same(raw.cpu().numpy(), oraw, "stream raw")
    assert_same(net.cpu().numpy(), onet, "stream net")


def test_repeated_calls_reuse_workspace(handle):
    """Workspace is reused and re-zeroed: a small graph after a large one, and the
    same graph twice, give identical results."""
    big = gg.rmat(13, 16, seed=5)
    small = gg.rmat(8, 8, seed=6)
    r1 = gpu(handle, small)
    gpu(handle, big)
    r2 = gpu(handle, small)
    assert_same(r1[0], r2[0], "repeat raw")
    assert_same(r1[1], r2[1], "repeat net")


def test_host_entry_point(handle):
    g = gg.rmat(11, 8, seed=12)
    oraw, onet = oracle.fglt(g)
    for rp in (g.rowptr.astype(np.int64), g.rowptr.astype(np.int32)):
        raw, net = handle.transform_host(rp, g.colidx, g.n)
        assert_same(raw, oraw, "host raw")
        assert_same(net, onet, "host net")


def test_batched_equals_per_graph(handle):
    batch = gg.small_graph_batch(60, seed=100, n_lo=10, n_hi=120)
    dev = torch.device("cuda:0")
    rp = torch.from_numpy(batch.graph.rowptr).to(dev)
    ci = torch.from_numpy(batch.graph.colidx).to(dev)
    raw, net = handle.transform_batched(rp, ci, batch.offsets)
    raw, net = raw.cpu().numpy(), net.cpu().numpy()
    oraw, onet = oracle.fglt(batch.graph)
    assert_same(raw, oraw, "batched raw")
    assert_same(net, onet, "batched net")


@pytest.mark.parametrize("span", [1, 64, 1024])
def test_cycle_paths_with_small_hub_span(span):
    """Shrinking the dense hub range routes 4-cycle work through the shared and
    global hash tables; the counts must not change."""
    import paper_2007_11111_gb300 as fg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with fg.Handle(device=0, cyc_hub_span=span) as h:
        for g in (gg.rmat(12, 16, seed=21), gg.barabasi_albert(2000, 6, seed=3), complete_bipartite(60, 90)):
            check_vs_oracle(h, g, f"span {span} n={g.n}")


def test_dense_neighbourhoods_hub_classes(handle):
    """Two roots whose higher-ranked neighbours induce a random subgraph of
    density 1/2 (the shape of the largest triangle classes on R-MAT s24):
    out-degree 1100 runs in the class with the bitmap in global memory and its
    tensor-core clique phase, 991 in the largest shared-memory class. The roots, a
    few core and booster vertices against the oracle; every row against the
    invariants."""
    g = gg.dense_neighbourhoods(1100, 0.5, (1.0, 0.9), 900, 0.75, seed=5)
    raw, net = gpu(handle, g)
    assert (net >= 0).all()
    assert_same(raw, net @ oracle.u16().T, "raw = U16 net")
    s = net.sum(axis=0)
    assert s[1] == 2 * g.m and s[2] == 2 * s[3] and s[5] == s[6] and s[7] == 3 * s[8]
    assert s[10] == 2 * s[9] and s[9] == s[11] and s[13] == s[14]
    assert s[4] % 3 == 0 and s[12] % 4 == 0 and s[15] % 4 == 0
    verts = np.array([1100, 1101, 0, 1, 1102, 1103])
    oraw, onet = oracle.fglt(g, vertices=verts)
    assert_same(raw[verts], oraw, "sampled raw")
    assert_same(net[verts], onet, "sampled net")


@pytest.fixture(scope="module")
def s20(handle):
    g = gg.rmat(20, 16, seed=0)
    raw, net = gpu(handle, g)
    return g, raw, net


def test_rmat_s20_top_hubs_vs_stored_oracle_rows(s20):
    """The 16 highest-degree vertices of R-MAT scale 20 (degrees up to 6.5e4;
    their rows take the oracle minutes each, so they are stored once by an
    oracle-only script) element by element, on the benchmark's graph."""
    import os
    import sys
    sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
    from make_hub_rows import csr_digest, top_degree_vertices
    g, raw, net = s20
    head, rows = read_hub_rows("hub_rows_rmat-s20-ef16.txt")
    assert int(head["n"]) == g.n and int(head["nnz"]) == g.nnz
    assert head["sha256"] == csr_digest(g.rowptr, g.colidx), "stored rows are for another graph"
    verts = [v for v, _, _ in rows]
    assert verts == list(top_degree_vertices(g.rowptr, 16))
    assert np.diff(g.rowptr).max() == max(np.diff(g.rowptr)[verts])  # the largest hub is among them
    for v, oraw, onet in rows:
        assert_same(raw[v:v + 1], oraw[None, :], f"hub {v} raw")
        assert_same(net[v:v + 1], onet[None, :], f"hub {v} net")


@pytest.mark.parametrize("pass2_from", [1, 2])
def test_pass2_listing_vertex(pass2_from):
    """The second triangle pass listed from each triangle's lowest vertex and
    from its middle vertex (through the in-lists) gives the oracle's counts,
    on R-MAT, BA, dense neighbourhoods and complete graphs."""
    import paper_2007_11111_gb300 as fg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with fg.Handle(device=0, tri_pass2_from=pass2_from) as h:
        for g in (gg.rmat(12, 16, seed=4), gg.barabasi_albert(3000, 7, seed=8), gg.complete(40), gg.star(50),
                  gg.dense_neighbourhoods(300, 0.4, (1.0, 0.7), 120, 0.8, seed=6)):
            check_vs_oracle(h, g, f"pass 2 from {pass2_from}, n={g.n}")


def test_rmat_s20_full_size_sampled(s20):
    """R-MAT scale 20, edge factor 16, seed 0, in the benchmark's launch
    configuration: every row checked against the invariants that hold at any
    size, and a vertex sample (high-degree, dense-class, low-degree and
    isolated vertices, uniform picks) element by element against the
    oracle."""
    g, raw, net = s20
    deg = np.diff(g.rowptr)
    # invariants on every row
    np.testing.assert_array_equal(raw[:, 0], 1)
    np.testing.assert_array_equal(raw[:, 1], deg)
    assert (net >= 0).all()
    assert_same(raw, net @ oracle.u16().T, "raw = U16 net")
    s = net.sum(axis=0)
    assert s[1] == 2 * g.m and s[2] == 2 * s[3] and s[5] == s[6] and s[7] == 3 * s[8]
    assert s[10] == 2 * s[9] and s[9] == s[11] and s[13] == s[14]
    assert s[4] % 3 == 0 and s[12] % 4 == 0 and s[15] % 4 == 0
    # sampled rows vs the oracle
    rng = np.random.default_rng(2024)
    order = np.argsort(deg)
    # a high-degree vertex (rank 300 from the top, degree ~4000), vertices of
    # the dense 4-cycle classes (ranks 1500 and 3000), the lowest, median and
    # random ones; the largest hubs cost the oracle minutes per row
    verts = np.unique(np.concatenate([order[[-300, -1500, -3000]], order[:4],
                                      order[len(order) // 2: len(order) // 2 + 4], rng.integers(0, g.n, 40)]))
    oraw, onet = oracle.fglt(g, vertices=verts)
    assert_same(raw[verts], oraw, "sampled raw")
    assert_same(net[verts], onet, "sampled net")
