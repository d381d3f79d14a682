"""Sub-dictionary transforms on the GPU (Table II caption: a sub-dictionary s
converts with U16(s,s)), element by element against the oracle, through the
single-graph, host and batched entry points. The pipeline skips the stages no
row of s needs (e.g. Sigma5 runs no 4-cycle, diamond or clique work)."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MASKS = [0x1F, 0x3, 0x3 | (1 << 12), 0x3 | (1 << 13) | (1 << 15), 0x3 | (1 << 5) | (1 << 9),
         0x3 | (1 << 10) | (1 << 14), 0xFFFF, 0x3 | (1 << 4) | (1 << 6) | (1 << 11), 0x7FFF, 0xFFFE | 0x1]


def _graphs():
    return [gg.rmat(11, 16, seed=8), gg.barabasi_albert(1500, 5, seed=2), gg.complete(40),
            gg.erdos_renyi(2000, 10, seed=0)]


@pytest.fixture(scope="module")
def cases():
    return [(g, oracle.fglt(g)[0]) for g in _graphs()]


@pytest.mark.parametrize("mask", MASKS, ids=[hex(m) for m in MASKS])
def test_sub_dictionary_matches_oracle(cases, mask):
    import paper_2007_11111_gb300 as fg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    with fg.Handle(device=0, dictionary=mask) as h:
        for g, raw16 in cases:
            want_raw, want_net = oracle.sub_dictionary(raw16, mask)
            rp = torch.from_numpy(g.rowptr).to(dev)
            ci = torch.from_numpy(g.colidx).to(dev)
            raw, net = h.transform(rp, ci, g.n)
            assert raw.shape == want_raw.shape
            np.testing.assert_array_equal(raw.cpu().numpy(), want_raw, err_msg=f"{hex(mask)} n={g.n}")
            np.testing.assert_array_equal(net.cpu().numpy(), want_net, err_msg=f"{hex(mask)} n={g.n}")
            hraw, hnet = h.transform_host(g.rowptr, g.colidx, g.n)
            np.testing.assert_array_equal(hnet, want_net)


def test_sigma5_batched_and_served():
    import paper_2007_11111_gb300 as fg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    batch = gg.small_graph_batch(300, seed=11, n_lo=10, n_hi=120)
    G = batch.graph
    want_raw, want_net = oracle.fglt(G, dictionary=fg.DICT_SIGMA5)
    dev = torch.device("cuda:0")
    with fg.Handle(device=0, dictionary=fg.DICT_SIGMA5) as h:
        rp = torch.from_numpy(G.rowptr).to(dev)
        ci = torch.from_numpy(G.colidx).to(dev)
        for _ in range(2):  # first run captures, second replays
            raw, net = h.transform_batched(rp, ci, batch.offsets)
            np.testing.assert_array_equal(net.cpu().numpy(), want_net)
            np.testing.assert_array_equal(raw.cpu().numpy(), want_raw)
        g = gg.rmat(10, 8, seed=3)
        r5, n5 = oracle.fglt(g, dictionary=fg.DICT_SIGMA5)
        out_raw = np.empty((g.n, 5), np.int64)
        out_net = np.empty((g.n, 5), np.int64)
        rid = fg.fglt_stream_submit(h.h, g.n, np.ascontiguousarray(g.rowptr), g.colidx, out_raw, out_net)
        st, _ = fg.fglt_stream_poll(h.h, rid, -1)
        assert st == fg.FGLT_OK
        np.testing.assert_array_equal(out_net, n5)
        np.testing.assert_array_equal(out_raw, r5)


def test_invalid_dictionaries_rejected():
    import paper_2007_11111_gb300 as fg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    for mask in (0x1, 0x2, 0x1C, (1 << 16) | 0x3):
        with pytest.raises(fg.FgltError) as e:
            fg.Handle(device=0, dictionary=mask)
        assert e.value.status == fg.FGLT_ERR_INVALID_ARG
