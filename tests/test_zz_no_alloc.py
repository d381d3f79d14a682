"""fglt_transform_noalloc (the entry point for callers that cannot allocate
device memory at call time) against fglt_transform, through the C ABI.

Counts are integers, so the tolerance is zero: outputs must be identical. The
calls come in a row, so a call that left stale data in the shared scratch
array for the next one would show up here. This file is collected last.
"""
import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(g):
    dev = torch.device("cuda:0")
    rp = torch.from_numpy(g.rowptr).to(dev)
    ci = torch.from_numpy(g.colidx if g.colidx.size else np.zeros(1, np.int32)).to(dev)
    return rp, ci


def _reference(h, g):
    rp, ci = _dev(g)
    raw, net = h.transform(rp, ci, g.n)
    return raw.cpu().numpy(), net.cpu().numpy()


def _noalloc(g, rp64=True):
    import paper_2007_11111_gb300 as fg
    dev = torch.device("cuda:0")
    rp = torch.from_numpy(g.rowptr.astype(np.int64 if rp64 else np.int32)).to(dev)
    ci = torch.from_numpy(g.colidx if g.colidx.size else np.zeros(1, np.int32)).to(dev)
    raw = torch.full((g.n, 16), -7, dtype=torch.int64, device=dev)
    net = torch.full((g.n, 16), -7, dtype=torch.int64, device=dev)
    fg.fglt_transform_noalloc(rp, 1 if rp64 else 0, ci, g.n, raw, net)
    return raw.cpu().numpy(), net.cpu().numpy()


def test_noalloc_matches_transform_on_consecutive_calls():
    import paper_2007_11111_gb300 as fg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    graphs = [gg.rmat(13, 16, seed=31), gg.erdos_renyi(2000, 10, seed=0), gg.rmat(13, 16, seed=31),
              gg.barabasi_albert(3000, 5, seed=2),
              gg.rmat(15, 16, seed=5)]  # 32768 vertices, ~880K stored entries: near both limits
    with fg.Handle(device=0) as h:
        for k, g in enumerate(graphs):
            want_raw, want_net = _reference(h, g)
            got_raw, got_net = _noalloc(g, rp64=(k % 2 == 0))
            np.testing.assert_array_equal(got_raw, want_raw, err_msg=f"call {k} raw")
            np.testing.assert_array_equal(got_net, want_net, err_msg=f"call {k} net")


def test_noalloc_rejects_sizes_beyond_its_limit():
    import paper_2007_11111_gb300 as fg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = gg.empty(40000)  # more vertices than FGLT_NOALLOC_MAX_VERTICES (32768)
    with pytest.raises(fg.FgltError) as e:
        _noalloc(g)
    assert e.value.status == fg.FGLT_ERR_UNSUPPORTED
    big = gg.erdos_renyi(1500, 900, seed=1)  # more than 1,048,576 stored entries
    assert big.nnz > 1048576
    with pytest.raises(fg.FgltError) as e:
        _noalloc(big)
    assert e.value.status == fg.FGLT_ERR_UNSUPPORTED


def test_noalloc_at_both_limits_then_a_normal_call():
    """The largest inputs the limits admit (32768 vertices with about 1.05
    million stored entries; K_1024 with 1,047,552 entries, whose degree-order
    out-degrees reach the largest shared-memory triangle class) fit the
    scratch array and equal fglt_transform; a normal call after them too."""
    import paper_2007_11111_gb300 as fg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    graphs = [gg.erdos_renyi(32768, 31.9, seed=7), gg.complete(1024), gg.rmat(12, 8, seed=3)]
    assert graphs[0].nnz <= 1048576 and graphs[1].nnz <= 1048576
    with fg.Handle(device=0) as h:
        for g in graphs:
            want_raw, want_net = _reference(h, g)
            got_raw, got_net = _noalloc(g)
            np.testing.assert_array_equal(got_raw, want_raw)
            np.testing.assert_array_equal(got_net, want_net)
