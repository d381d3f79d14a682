"""The tuning settings (degree-class bounds of the triangle passes, hash-table
sizes and block shapes of the 4-cycle classes, the dense hub span) move work
between kernels but never change a count: every setting must reproduce the
oracle bit for bit. The autotuner must return a valid setting, install it, and
leave the results unchanged."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SETTINGS = [
    dict(),
    dict(tri_class_bounds=(2, 3), tri_group_lanes=8),
    dict(tri_group_lanes=16, tri_probe_loads=2, tri_warp_max=32),
    dict(tri_warp_max=16, tri_class_bounds=(8, 20)),
    dict(tri_warp_max=-1, tri_class_bounds=(64, 256)),
    dict(tri_warp_max=32, tri_probe_loads=2, tri_class_bounds=(2, 3)),
    dict(tri_class_bounds=(8, 1024), tri_probe_loads=4, tri_hash_factor=4),
    dict(tri_class_bounds=(3, 2000), tri_probe_loads=4),
    dict(cyc_warp_bits=6),
    dict(cyc_warp_bits=8, cyc_mid_threads=(512, 1024, 512)),
    dict(cyc_mid_threads=(1024, 128, 1024), cyc_heavy_threads=256, tri_hash_factor=4),
    dict(cyc_heavy_threads=512, cyc_hub_span=64, cyc_dense_min=1),
    dict(cyc_dense_min=1024, cyc_mid_threads=(128, 128, 128), cyc_long_segment=2),
    dict(cyc_long_segment=512, cyc_heavy_threads=512, cyc_spill_bits=13),
    dict(cyc_spill_bits=12, cyc_hub_span=64, cyc_dense_min=1),
    dict(cyc_hub_span=1, cyc_warp_bits=7, tri_class_bounds=(16, 32)),
    dict(tri_pass2_from=1),
    dict(tri_pass2_from=2),
    dict(tri_pass2_from=2, tri_warp_max=-1, tri_class_bounds=(64, 256)),
    dict(tri_pass2_from=2, tri_class_bounds=(2, 3), tri_group_lanes=8, tri_probe_loads=2),
    dict(tri_pass2_from=2, tri_class_bounds=(3, 2000), tri_hash_factor=2),
]


def _graphs():
    def complete_bipartite(a, b):
        i = np.repeat(np.arange(a), b)
        j = a + np.tile(np.arange(b), a)
        return gg.csr_from_pairs(a + b, i, j)
    return [gg.rmat(12, 16, seed=21), gg.barabasi_albert(3000, 7, seed=3), complete_bipartite(70, 90),
            gg.rmat(13, 8, seed=5), gg.complete(300)]


@pytest.fixture(scope="module")
def cases():
    return [(g, oracle.fglt(g)) for g in _graphs()]


def _run(h, g):
    dev = torch.device("cuda:0")
    rp = torch.from_numpy(g.rowptr).to(dev)
    ci = torch.from_numpy(g.colidx).to(dev)
    raw, net = h.transform(rp, ci, g.n)
    return raw.cpu().numpy(), net.cpu().numpy()


@pytest.mark.parametrize("setting", SETTINGS, ids=[str(s) or "default" for s in SETTINGS])
def test_every_setting_matches_oracle(cases, setting):
    import paper_2007_11111_gb300 as fg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with fg.Handle(device=0, **setting) as h:
        for g, (oraw, onet) in cases:
            raw, net = _run(h, g)
            np.testing.assert_array_equal(raw, oraw, err_msg=f"{setting} n={g.n}")
            np.testing.assert_array_equal(net, onet, err_msg=f"{setting} n={g.n}")


def test_invalid_settings_rejected():
    import paper_2007_11111_gb300 as fg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    for bad in (dict(tri_class_bounds=(64, 32)), dict(tri_class_bounds=(1, 8)), dict(cyc_warp_bits=11),
                dict(cyc_warp_bits=5), dict(cyc_mid_threads=(96, 256, 256)), dict(cyc_heavy_threads=300),
                dict(cyc_hub_span=-1), dict(cyc_hub_span=90113), dict(tri_probe_loads=3),
                dict(tri_hash_factor=3), dict(cyc_mid_threads=(64, 256, 256)), dict(cyc_dense_min=5000),
                dict(tri_group_lanes=4), dict(cyc_long_segment=1), dict(tri_warp_max=33), dict(cyc_spill_bits=14),
                dict(tri_warp_max=-2), dict(tri_pass2_from=3), dict(tri_pass2_from=-1),
                dict(device_wait_limit_ns=-1)):
        with pytest.raises(fg.FgltError) as e:
            fg.Handle(device=0, **bad)
        assert e.value.status == fg.FGLT_ERR_INVALID_ARG


def test_autotune_installs_setting_and_keeps_results(cases):
    import paper_2007_11111_gb300 as fg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g, (oraw, onet) = cases[0]
    dev = torch.device("cuda:0")
    rp = torch.from_numpy(g.rowptr).to(dev)
    ci = torch.from_numpy(g.colidx).to(dev)
    with fg.Handle(device=0) as h:
        chosen, tuned_ms, default_ms = h.autotune(rp, ci, g.n, reps=1)
        assert tuned_ms > 0 and default_ms > 0
        t0, t1 = chosen["tri_class_bounds"]
        assert 2 <= t0 < t1
        assert 6 <= chosen["cyc_warp_bits"] <= 10
        assert all(x in (128, 256, 512, 1024) for x in chosen["cyc_mid_threads"])
        assert chosen["tri_hash_factor"] in (2, 4) and chosen["tri_probe_loads"] in (2, 4)
        assert chosen["cyc_heavy_threads"] in (256, 512, 1024)
        # results under the installed setting, on this graph and on another
        for gg_, (wr, wn) in (cases[0], cases[1]):
            raw, net = _run(h, gg_)
            np.testing.assert_array_equal(raw, wr)
            np.testing.assert_array_equal(net, wn)
        # a fresh handle created with the chosen setting gives the same counts
        kw = dict(tri_class_bounds=tuple(chosen["tri_class_bounds"]), cyc_warp_bits=chosen["cyc_warp_bits"],
                  tri_probe_loads=chosen["tri_probe_loads"], tri_hash_factor=chosen["tri_hash_factor"],
                  tri_group_lanes=chosen["tri_group_lanes"], tri_warp_max=chosen["tri_warp_max"],
                  cyc_mid_threads=tuple(chosen["cyc_mid_threads"]), cyc_heavy_threads=chosen["cyc_heavy_threads"],
                  cyc_hub_span=chosen["cyc_hub_span"], cyc_dense_min=chosen["cyc_dense_min"],
                  cyc_long_segment=chosen["cyc_long_segment"], cyc_spill_bits=chosen["cyc_spill_bits"],
                  tri_pass2_from=chosen["tri_pass2_from"])
        with fg.Handle(device=0, **kw) as h2:
            raw, net = _run(h2, g)
            np.testing.assert_array_equal(net, onet)


@pytest.mark.parametrize("bounds,lanes", [((3, 2000), 8), ((64, 256), 32)])
def test_global_bitmap_in_any_class_closed_form(bounds, lanes):
    """K_1200: every out-degree in the degree order is above the shared-memory
    bitmap limit, so with class bounds (3, 2000) a middle class runs on the
    global-memory bitmap. Net counts have the closed form of a clique."""
    import paper_2007_11111_gb300 as fg
    from math import comb
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = 1200
    g = gg.complete(n)
    with fg.Handle(device=0, tri_class_bounds=bounds, tri_group_lanes=lanes) as h:
        _, net = _run(h, g)
    want = np.zeros(16, np.int64)
    want[0], want[1], want[4], want[15] = 1, n - 1, comb(n - 1, 2), comb(n - 1, 3)
    np.testing.assert_array_equal(net, np.tile(want, (n, 1)))


def test_complete_multipartite_beyond_one_accumulator_segment():
    """Complete 6-partite graph with parts of 900 (vertex v in part v mod 6):
    every vertex has degree 4500, so out-degrees in the degree order reach
    4499 and the global-bitmap class forms S S on the tensor cores over more
    than 4096 columns of K (two accumulator read-outs), with S zero wherever
    two vertices share a part. All vertices are alike: triangles
    binom(5, 2) 900^2 and 4-cliques binom(5, 3) 900^3 at each, equal rows,
    and raw = U16 net."""
    import paper_2007_11111_gb300 as fg
    from math import comb
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    k, s = 6, 900
    n = k * s
    i, j = np.triu_indices(n, k=1)
    keep = (i % k) != (j % k)
    g = gg.csr_from_pairs(n, i[keep], j[keep])
    with fg.Handle(device=0) as h:
        raw, net = _run(h, g)
    assert (net == net[0]).all(), "all vertices alike"
    assert net[0, 1] == (k - 1) * s
    assert net[0, 4] == comb(k - 1, 2) * s ** 2
    assert net[0, 15] == comb(k - 1, 3) * s ** 3
    np.testing.assert_array_equal(raw, net @ oracle.u16().T)


def test_device_wait_that_runs_out_returns_timeout():
    """With a device wait limit of 1 (give up after the first unsuccessful
    test), the global-bitmap triangle class's first wait on its tensor-core
    work runs out (the MMAs were issued a moment before): the kernel leaves,
    after waiting for its own MMAs and freeing its tensor memory, and the call
    returns FGLT_ERR_TIMEOUT. The handle stays usable for a graph without that
    class, and a handle with the default limit gets K_1200 exact."""
    import paper_2007_11111_gb300 as fg
    from math import comb
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = 1200
    g = gg.complete(n)
    small = gg.rmat(12, 16, seed=21)
    want_small = oracle.fglt(small)
    with fg.Handle(device=0, device_wait_limit_ns=1) as h:
        with pytest.raises(fg.FgltError) as e:
            _run(h, g)
        assert e.value.status == fg.FGLT_ERR_TIMEOUT
        raw, net = _run(h, small)  # out-degrees below the global-bitmap class: no tensor-core waits
        np.testing.assert_array_equal(raw, want_small[0])
        np.testing.assert_array_equal(net, want_small[1])
    with fg.Handle(device=0) as h:
        _, net = _run(h, g)
    want = np.zeros(16, np.int64)
    want[0], want[1], want[4], want[15] = 1, n - 1, comb(n - 1, 2), comb(n - 1, 3)
    np.testing.assert_array_equal(net, np.tile(want, (n, 1)))
