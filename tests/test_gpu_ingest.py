"""Edge-list ingest on the GPU (fglt_csr_from_edges): any list of vertex pairs
becomes the simple undirected graph the paper assumes (Sec. 1), as a sorted
symmetric CSR, equal to the host construction (graphgen.csr_from_pairs) entry
for entry; the transform of the result matches the oracle."""
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
