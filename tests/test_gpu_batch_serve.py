"""Batched and served transforms through the C ABI.

Every result must equal (bit for bit) the single-graph transform of the same
graph run alone; for the batched entry also the oracle."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fg():
    import paper_2007_11111_gb300 as fg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return fg


def alone(h, g):
    dev = torch.device("cuda:0")
    rp = torch.from_numpy(g.rowptr).to(dev)
    ci = torch.from_numpy(g.colidx if g.colidx.size else np.zeros(1, np.int32)).to(dev)
    raw, net = h.transform(rp, ci, g.n)
    return raw.cpu().numpy(), net.cpu().numpy()


def test_batched_replay_and_recapture(fg):
    """Second call with the same buffers replays the captured CUDA graph; a
    different batch re-captures. Outputs are cleared between calls."""
    dev = torch.device("cuda:0")
    with fg.Handle(device=0) as h:
        for seed in (7, 7, 8):
            batch = gg.small_graph_batch(200, seed=seed, n_lo=10, n_hi=200)
            oraw, onet = oracle.fglt(batch.graph)
            rp = torch.from_numpy(batch.graph.rowptr).to(dev)
            ci = torch.from_numpy(batch.graph.colidx).to(dev)
            for _ in range(2):
                raw = torch.full((batch.graph.n, 16), -1, dtype=torch.int64, device=dev)
                net = torch.full((batch.graph.n, 16), -1, dtype=torch.int64, device=dev)
                h.transform_batched(rp, ci, batch.offsets, raw, net)
                np.testing.assert_array_equal(raw.cpu().numpy(), oraw)
                np.testing.assert_array_equal(net.cpu().numpy(), onet)


def test_batched_validation_rejects_cross_edges(fg):
    dev = torch.device("cuda:0")
    parts = [gg.complete(4), gg.complete(5)]
    batch = gg.pack_block_diagonal(parts)
    # join vertex 0 of graph 0 to vertex 4 (first vertex of graph 1)
    rows = np.repeat(np.arange(batch.graph.n), np.diff(batch.graph.rowptr))
    bad = gg.csr_from_pairs(batch.graph.n, np.concatenate([rows, [0]]),
                            np.concatenate([batch.graph.colidx.astype(np.int64), [4]]))
    with fg.Handle(device=0, validate=True) as h:
        rp = torch.from_numpy(bad.rowptr).to(dev)
        ci = torch.from_numpy(bad.colidx).to(dev)
        with pytest.raises(fg.FgltError) as e:
            h.transform_batched(rp, ci, batch.offsets)
        assert e.value.status == fg.FGLT_ERR_INVALID_GRAPH
        rp = torch.from_numpy(batch.graph.rowptr).to(dev)
        ci = torch.from_numpy(batch.graph.colidx).to(dev)
        raw, net = h.transform_batched(rp, ci, batch.offsets)
        np.testing.assert_array_equal(net.cpu().numpy(), oracle.fglt(batch.graph)[1])


def mixed_graphs():
    out = []
    for s in range(6):
        out.append(gg.rmat(8 + s % 5, 8, seed=40 + s))
        out.append(gg.barabasi_albert(100 + 150 * s, 3 + s % 3, seed=s))
        out.append(gg.erdos_renyi(50 + 30 * s, 6, seed=s))
    out += [gg.empty(5), gg.complete(30), gg.star(700), gg.path(2), gg.rmat(15, 16, seed=3)]
    return out


def test_served_results_equal_alone(fg):
    graphs = mixed_graphs()
    with fg.Handle(device=0) as h:
        want = [alone(h, g) for g in graphs]
    with fg.Handle(device=0) as h:
        outs, ids = [], []
        for g in graphs:  # submitted back to back: packs form while others run
            raw = np.full((g.n, 16), -1, np.int64)
            net = np.full((g.n, 16), -1, np.int64)
            rp = np.ascontiguousarray(g.rowptr, dtype=np.int64)
            ci = np.ascontiguousarray(g.colidx if g.colidx.size else np.zeros(1, np.int32), dtype=np.int32)
            outs.append((raw, net, rp, ci))
            ids.append(fg.fglt_stream_submit(h.h, g.n, rp, ci, raw, net))
        lat = []
        for k, rid in enumerate(ids):
            st, us = fg.fglt_stream_poll(h.h, rid, 60000)
            assert st == fg.FGLT_OK, (k, st)
            lat.append(us)
            np.testing.assert_array_equal(outs[k][0], want[k][0], err_msg=f"request {k} raw")
            np.testing.assert_array_equal(outs[k][1], want[k][1], err_msg=f"request {k} net")
        assert all(x > 0 for x in lat)
        st, _ = fg.fglt_stream_poll(h.h, ids[0], 0)
        assert st == fg.FGLT_ERR_NOT_FOUND  # collected ids are retired
    # and the served rows against the oracle directly
    for k, g in enumerate(graphs):
        oraw, onet = oracle.fglt(g)
        np.testing.assert_array_equal(outs[k][0], oraw, err_msg=f"request {k} raw vs oracle")
        np.testing.assert_array_equal(outs[k][1], onet, err_msg=f"request {k} net vs oracle")


def test_served_small_requests_overtake_a_large_one(fg):
    """A large request that does not fit the memory budget while others run
    does not hold back the small ones queued behind it (they may overtake it),
    and every result equals the oracle's."""
    big = gg.rmat(16, 16, seed=9)
    smalls = [gg.erdos_renyi(300, 6, seed=s) for s in range(40)]
    est_big = big.n * 512 + big.nnz * 24 + (4 << 20)
    with fg.Handle(device=0, serve_memory_budget=3 * est_big) as h:
        reqs = []
        for g in [big, big] + smalls:
            raw = np.full((g.n, 16), -1, np.int64)
            net = np.full((g.n, 16), -1, np.int64)
            rp = np.ascontiguousarray(g.rowptr, dtype=np.int64)
            ci = np.ascontiguousarray(g.colidx, dtype=np.int32)
            reqs.append((g, raw, net, rp, ci, fg.fglt_stream_submit(h.h, g.n, rp, ci, raw, net)))
        for g, raw, net, _, _, rid in reqs:
            st, _ = fg.fglt_stream_poll(h.h, rid, 120000)
            assert st == fg.FGLT_OK
        for g, raw, net, _, _, _ in reqs[2:7] + reqs[-3:]:
            oraw, onet = oracle.fglt(g)
            np.testing.assert_array_equal(raw, oraw)
            np.testing.assert_array_equal(net, onet)


def test_served_bad_request_is_isolated(fg):
    good = [gg.rmat(9, 8, seed=s) for s in range(6)]
    g0 = gg.complete(6)
    rows = np.repeat(np.arange(g0.n), np.diff(g0.rowptr))
    keep = ~((rows == 0) & (g0.colidx == 1))  # drop 0->1 but keep 1->0: asymmetric
    rp_bad = np.zeros(g0.n + 1, np.int64)
    np.cumsum(np.bincount(rows[keep], minlength=g0.n), out=rp_bad[1:])
    ci_bad = g0.colidx[keep].astype(np.int32)
    with fg.Handle(device=0, validate=True) as h:
        want = [alone(h, g) for g in good]
        bufs, ids = [], []
        for k, g in enumerate(good):
            if k == 3:
                raw = np.zeros((g0.n, 16), np.int64)
                ids.append(("bad", fg.fglt_stream_submit(h.h, g0.n, rp_bad, ci_bad, raw, None)))
                bufs.append((rp_bad, ci_bad, raw))
            raw = np.zeros((g.n, 16), np.int64)
            rp = np.ascontiguousarray(g.rowptr, dtype=np.int64)
            ids.append((k, fg.fglt_stream_submit(h.h, g.n, rp, g.colidx, raw, None)))
            bufs.append((rp, g.colidx, raw))
        for (tag, rid), b in zip(ids, bufs):
            st, _ = fg.fglt_stream_poll(h.h, rid, 60000)
            if tag == "bad":
                assert st == fg.FGLT_ERR_INVALID_GRAPH
            else:
                assert st == fg.FGLT_OK
                np.testing.assert_array_equal(b[2], want[tag][0])


def test_served_budget_and_cancel(fg):
    g = gg.rmat(12, 16, seed=1)
    rp = np.ascontiguousarray(g.rowptr, dtype=np.int64)
    raw = np.zeros((g.n, 16), np.int64)
    with fg.Handle(device=0, serve_memory_budget=4 << 20) as h:  # below any request's estimate
        with pytest.raises(fg.FgltError) as e:
            fg.fglt_stream_submit(h.h, g.n, rp, g.colidx, raw, None)
        assert e.value.status == fg.FGLT_ERR_BUSY
    with fg.Handle(device=0) as h:
        outs = [np.zeros((g.n, 16), np.int64) for _ in range(30)]  # must outlive the requests
        ids = [fg.fglt_stream_submit(h.h, g.n, rp, g.colidx, outs[k], None) for k in range(30)]
        st = fg.fglt_stream_cancel(h.h, ids[-1])
        assert st in (fg.FGLT_OK, fg.FGLT_ERR_BUSY)
        for rid in ids[:-1]:
            assert fg.fglt_stream_poll(h.h, rid, 60000)[0] == fg.FGLT_OK
        if st == fg.FGLT_OK:
            assert fg.fglt_stream_poll(h.h, ids[-1], 0)[0] == fg.FGLT_ERR_NOT_FOUND
        else:
            assert fg.fglt_stream_poll(h.h, ids[-1], 60000)[0] == fg.FGLT_OK


@pytest.mark.parametrize("hash_factor", [2, 4])
def test_batched_with_a_4096_vertex_member(fg, hash_factor):
    """A batch whose largest graph has 4096 vertices: the host-side bounds put
    the degree and out-degree bounds at 4095, so every triangle class up to
    the global-bitmap one is sized for that bound (both hash-table sizes)."""
    graphs = [gg.rmat(12, 8, seed=3), gg.barabasi_albert(300, 3, seed=1), gg.complete(40), gg.cycle(9)]
    batch = gg.pack_block_diagonal(graphs)
    oraw, onet = oracle.fglt(batch.graph)
    dev = torch.device("cuda:0")
    rp = torch.from_numpy(batch.graph.rowptr).to(dev)
    ci = torch.from_numpy(batch.graph.colidx).to(dev)
    with fg.Handle(device=0, tri_hash_factor=hash_factor) as h:
        for _ in range(2):  # captured run, then replay
            raw, net = h.transform_batched(rp, ci, batch.offsets)
            np.testing.assert_array_equal(raw.cpu().numpy(), oraw)
            np.testing.assert_array_equal(net.cpu().numpy(), onet)


def _dev(g):
    dev = torch.device("cuda:0")
    return torch.from_numpy(g.rowptr).to(dev), torch.from_numpy(g.colidx if g.colidx.size else
                                                                 np.zeros(1, np.int32)).to(dev)


def test_fused_batch_20000_graphs_vs_oracle_and_sequence(fg):
    """The benchmark's batch (20,000 BA and random-geometric graphs of 10..500
    vertices) through the fused one-block-per-graph launch, element by element
    against the oracle, then against the stage sequence (batch_small_max=-1),
    and once more as a replay."""
    batch = gg.small_graph_batch(20000, seed=0, n_lo=10, n_hi=500)
    oraw, onet = oracle.fglt(batch.graph)
    rp, ci = _dev(batch.graph)
    with fg.Handle(device=0) as h:
        for _ in range(2):
            raw, net = h.transform_batched(rp, ci, batch.offsets)
            np.testing.assert_array_equal(raw.cpu().numpy(), oraw)
            np.testing.assert_array_equal(net.cpu().numpy(), onet)
    with fg.Handle(device=0, batch_small_max=-1) as h:
        raw, net = h.transform_batched(rp, ci, batch.offsets)
        np.testing.assert_array_equal(net.cpu().numpy(), onet)


def test_fused_batch_limits_and_special_graphs(fg):
    """Graphs at the fused launch's size limit (512 vertices), complete graphs,
    stars, empty and single-vertex graphs; with a 513-vertex member the batch
    runs the stage sequence. Both against the oracle."""
    parts = [gg.complete(1), gg.empty(3), gg.complete(40), gg.star(300), gg.erdos_renyi(512, 30, seed=2),
             gg.barabasi_albert(512, 5, seed=4), gg.cycle(7), gg.path(2), gg.complete(64)]
    for extra in ([], [gg.erdos_renyi(513, 8, seed=5)]):
        batch = gg.pack_block_diagonal(parts + extra)
        oraw, onet = oracle.fglt(batch.graph)
        rp, ci = _dev(batch.graph)
        with fg.Handle(device=0) as h:
            raw, net = h.transform_batched(rp, ci, batch.offsets)
            np.testing.assert_array_equal(raw.cpu().numpy(), oraw)
            np.testing.assert_array_equal(net.cpu().numpy(), onet)


def test_fused_batch_sub_dictionary(fg):
    """A sub-dictionary through the fused launch: Sigma5, and a closed index
    set, equal the oracle's sub-dictionary conversion."""
    batch = gg.small_graph_batch(300, seed=3, n_lo=10, n_hi=300)
    oraw16, _ = oracle.fglt(batch.graph)
    rp, ci = _dev(batch.graph)
    for mask in (fg.DICT_SIGMA5, 0b1001000000011111):
        sraw, snet = oracle.sub_dictionary(oraw16, mask)
        with fg.Handle(device=0, dictionary=mask) as h:
            raw, net = h.transform_batched(rp, ci, batch.offsets)
            np.testing.assert_array_equal(raw.cpu().numpy(), sraw)
            np.testing.assert_array_equal(net.cpu().numpy(), snet)


def test_fused_batch_rejects_malformed_members(fg):
    """Without the validate option the fused launch still refuses an edge
    joining two graphs, a self-loop, a repeated entry and an asymmetric
    pattern; the handle then transforms a good batch."""
    base = gg.pack_block_diagonal([gg.complete(4), gg.cycle(6)])
    rows = np.repeat(np.arange(base.graph.n), np.diff(base.graph.rowptr))
    cols = base.graph.colidx.astype(np.int64)

    def raw_csr(r, c):  # rows as given, no symmetrisation or deduplication
        order = np.lexsort((c, r))
        r, c = r[order], c[order]
        rp = np.zeros(base.graph.n + 1, np.int64)
        np.cumsum(np.bincount(r, minlength=base.graph.n), out=rp[1:])
        return gg.Graph(base.graph.n, rp, c.astype(np.int32))

    bad = [raw_csr(np.concatenate([rows, [0, 4]]), np.concatenate([cols, [4, 0]])),  # cross edge
           raw_csr(np.concatenate([rows, [5]]), np.concatenate([cols, [5]])),        # self-loop
           raw_csr(np.concatenate([rows, [0]]), np.concatenate([cols, [1]])),        # repeated entry
           raw_csr(np.concatenate([rows, [4]]), np.concatenate([cols, [6]]))]        # asymmetric
    with fg.Handle(device=0) as h:
        for g in bad:
            rp, ci = _dev(g)
            with pytest.raises(fg.FgltError) as e:
                h.transform_batched(rp, ci, base.offsets)
            assert e.value.status == fg.FGLT_ERR_INVALID_GRAPH
        rp, ci = _dev(base.graph)
        _, net = h.transform_batched(rp, ci, base.offsets)
        np.testing.assert_array_equal(net.cpu().numpy(), oracle.fglt(base.graph)[1])
