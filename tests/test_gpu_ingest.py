"""Edge-list ingest on the GPU (fglt_csr_from_edges): any list of vertex pairs
becomes the simple undirected graph the paper assumes (Sec. 1), as a sorted
symmetric CSR, equal to the host construction (graphgen.csr_from_pairs) entry
for entry; the transform of the result matches the oracle.

Degree-ordered relabelling (fglt_csr_relabel_by_degree): the output is the
input relabelled by the returned permutation (host relabelling entry for
entry), new ids follow the degree order, and the transform of the relabelled
graph is the permuted transform (Sec. 2: invariance under isomorphism)."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _ingest(h, n, src, dst):
    dev = torch.device("cuda:0")
    s = torch.from_numpy(np.asarray(src, np.int32)).to(dev)
    d = torch.from_numpy(np.asarray(dst, np.int32)).to(dev)
    rp, ci = h.csr_from_edges(s, d, n)
    return rp.cpu().numpy(), ci.cpu().numpy()


def _messy_pairs(n, m, seed):
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, m)
    dst = rng.integers(0, n, m)
    # repeats in both directions and self-loops
    k = m // 4
    src = np.concatenate([src, dst[:k], src[:k], np.arange(min(n, k))])
    dst = np.concatenate([dst, src[:k], dst[:k], np.arange(min(n, k))])
    return src, dst


@pytest.fixture(scope="module")
def handle():
    import paper_2007_11111_gb300 as fg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    h = fg.Handle(device=0)
    yield h
    h.close()


@pytest.mark.parametrize("n,m,seed", [(1, 3, 0), (50, 400, 1), (3000, 20000, 2), (200000, 1500000, 3)])
def test_matches_host_construction(handle, n, m, seed):
    src, dst = _messy_pairs(n, m, seed)
    rp, ci = _ingest(handle, n, src, dst)
    want = gg.csr_from_pairs(n, src, dst)
    np.testing.assert_array_equal(rp, want.rowptr)
    np.testing.assert_array_equal(ci, want.colidx)


def test_long_rows_and_empty_graph(handle):
    # a hub with 40,000 distinct neighbours, each pair given three times
    leaves = np.arange(1, 40001)
    src = np.concatenate([np.zeros(40000, np.int64), leaves, np.zeros(40000, np.int64)])
    dst = np.concatenate([leaves, np.zeros(40000, np.int64), leaves[::-1]])
    rp, ci = _ingest(handle, 40001, src, dst)
    want = gg.star(40000)
    np.testing.assert_array_equal(rp, want.rowptr)
    np.testing.assert_array_equal(ci, want.colidx)
    rp, ci = _ingest(handle, 10, [], [])
    np.testing.assert_array_equal(rp, np.zeros(11, np.int64))
    assert ci.size == 0


def test_out_of_range_ids_rejected(handle):
    import paper_2007_11111_gb300 as fg
    with pytest.raises(fg.FgltError) as e:
        _ingest(handle, 10, [0, 3, 10], [1, 4, 2])
    assert e.value.status == fg.FGLT_ERR_INVALID_GRAPH


def test_ingest_then_transform_matches_oracle(handle):
    g = gg.rmat(12, 8, seed=6)
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    keep = rows < g.colidx  # one direction only, shuffled
    rng = np.random.default_rng(0)
    order = rng.permutation(int(keep.sum()))
    src, dst = rows[keep][order], g.colidx[keep][order]
    dev = torch.device("cuda:0")
    s = torch.from_numpy(src.astype(np.int32)).to(dev)
    d = torch.from_numpy(dst.astype(np.int32)).to(dev)
    rp, ci = handle.csr_from_edges(s, d, g.n)
    raw, net = handle.transform(rp, ci, g.n)
    oraw, onet = oracle.fglt(g)
    np.testing.assert_array_equal(raw.cpu().numpy(), oraw)
    np.testing.assert_array_equal(net.cpu().numpy(), onet)


# --- degree-ordered relabelling (fglt_csr_relabel_by_degree) -------------------

def _relabel(h, g, descending, rp64=True):
    dev = torch.device("cuda:0")
    rp = torch.from_numpy(g.rowptr.astype(np.int64 if rp64 else np.int32)).to(dev)
    ci = torch.from_numpy(g.colidx if g.colidx.size else np.zeros(1, np.int32)).to(dev)
    out_rp, out_ci, perm = h.relabel_by_degree(rp, ci, g.n, descending=descending)
    return out_rp.cpu().numpy(), out_ci.cpu().numpy(), perm.cpu().numpy()


@pytest.mark.parametrize("desc", [True, False])
@pytest.mark.parametrize("which", ["rmat", "ba", "star_hub", "empty"])
def test_relabel_is_the_degree_ordered_isomorphic_graph(handle, which, desc):
    g = {"rmat": lambda: gg.rmat(14, 16, seed=9), "ba": lambda: gg.barabasi_albert(5000, 4, seed=3),
         "star_hub": lambda: gg.star(40000), "empty": lambda: gg.empty(7)}[which]()
    rp, ci, perm = _relabel(handle, g, desc, rp64=(which != "ba"))
    # perm is a permutation, and new ids follow the degree order
    assert np.array_equal(np.sort(perm), np.arange(g.n))
    deg = np.diff(g.rowptr)
    new_deg = np.empty(g.n, np.int64)
    new_deg[perm] = deg
    steps = np.diff(new_deg)
    assert (steps <= 0).all() if desc else (steps >= 0).all()
    # the output is that relabelling of the input, rows sorted
    want = gg.permute_vertices(g, perm)
    np.testing.assert_array_equal(rp, want.rowptr)
    np.testing.assert_array_equal(ci, want.colidx)


def test_relabelled_transform_is_the_permuted_transform(handle):
    g = gg.rmat(12, 16, seed=11)
    dev = torch.device("cuda:0")
    rp = torch.from_numpy(g.rowptr).to(dev)
    ci = torch.from_numpy(g.colidx).to(dev)
    raw, net = handle.transform(rp, ci, g.n)
    out_rp, out_ci, perm = handle.relabel_by_degree(rp, ci, g.n)
    raw2, net2 = handle.transform(out_rp, out_ci, g.n)
    p = perm.cpu().numpy()
    np.testing.assert_array_equal(raw2.cpu().numpy()[p], raw.cpu().numpy())
    np.testing.assert_array_equal(net2.cpu().numpy()[p], net.cpu().numpy())
    oraw, onet = oracle.fglt(g)
    np.testing.assert_array_equal(raw.cpu().numpy(), oraw)


def test_relabel_rejects_out_of_range_columns(handle):
    import paper_2007_11111_gb300 as fg
    g = gg.Graph(3, np.array([0, 1, 2, 3], np.int64), np.array([1, 0, 5], np.int32))
    with pytest.raises(fg.FgltError) as e:
        _relabel(handle, g, True)
    assert e.value.status == fg.FGLT_ERR_INVALID_GRAPH


def test_many_long_rows(handle):
    # complete bipartite K(200, 17000): 200 rows longer than the shared-memory
    # row sort (16384 entries), sorted one block per row; pairs shuffled
    a, b = 200, 17000
    rng = np.random.default_rng(4)
    left = np.repeat(np.arange(a), b)
    right = a + np.tile(np.arange(b), a)
    order = rng.permutation(left.size)
    src, dst = left[order], right[order]
    flip = rng.random(left.size) < 0.5
    src, dst = np.where(flip, dst, src), np.where(flip, src, dst)
    rp, ci = _ingest(handle, a + b, src, dst)
    want = gg.csr_from_pairs(a + b, src, dst)
    np.testing.assert_array_equal(rp, want.rowptr)
    np.testing.assert_array_equal(ci, want.colidx)
    g = gg.Graph(a + b, rp, ci)
    rp2, ci2, perm = _relabel(handle, g, True)
    assert (np.sort(perm[:a]) == np.arange(a)).all()  # the 200 long rows come first
    want = gg.permute_vertices(g, perm)
    np.testing.assert_array_equal(rp2, want.rowptr)
    np.testing.assert_array_equal(ci2, want.colidx)
