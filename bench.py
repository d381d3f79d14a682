#!/usr/bin/env python3
"""FGLT benchmark: one JSON line on stdout (rank 0).

Default workload: R-MAT scale 24, edge factor 32 (a,b,c = .57,.19,.19, seed 0,
seeded vertex permutation, symmetrised, deduplicated, no self-loops; drawn by
the seeded device generator), int32 column indices, int64 row pointers,
synthetic: n = 16.8 M, m = 5.1e8. A step is one full transform (all 16 raw and
16 net frequencies for every vertex) through the C ABI with the inputs resident
in device memory. L2 is flushed (512 MiB write) before every timed step,
outside the timed events. R-MAT scale 20 is timed as well and reported under
"extras".

--impl reference times the CPU oracle (the reference arm of this build) on a
stratified vertex sample of the same graph on the host cores, with the full
transform's time extrapolated from per-row costs (OracleSampler).

Multi-GPU (torchrun, --gpus N): every rank transforms its own replica of the
graph (the single-graph path is not sharded); value = all ranks' edges / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402

METRIC = "FGLT edges/s & HBM GB/s vs peak; batched graphs/s, p50/p99 vs per-graph launch"
UNIT = "undirected edges/s"

WORKLOADS = {
    "rmat-s20-ef16": dict(kind="rmat", scale=20, ef=16, seed=0,
                          desc="R-MAT scale 20, edge factor 16, a=.57 b=.19 c=.19, seed 0, permuted, "
                               "symmetric simple CSR, int32 colidx, int64 rowptr"),
    "rmat-s18-ef16": dict(kind="rmat", scale=18, ef=16, seed=0,
                          desc="R-MAT scale 18, edge factor 16, a=.57 b=.19 c=.19, seed 0, permuted, "
                               "symmetric simple CSR (profiling size)"),
    "er-2000-d10": dict(kind="er", n=2000, deg=10, seed=0,
                        desc="Erdos-Renyi G(n=2000, avg degree 10), seed 0, symmetric simple CSR"),
    "rmat-s24-ef32": dict(kind="rmat_dev", scale=24, ef=32, seed=0,
                          desc="R-MAT scale 24, edge factor 32, a=.57 b=.19 c=.19, seed 0, permuted, "
                               "symmetric simple CSR generated on the device, int32 colidx, int64 rowptr"),
    "rmat-s21-ef32": dict(kind="rmat_dev", scale=21, ef=32, seed=0,
                          desc="R-MAT scale 21, edge factor 32, a=.57 b=.19 c=.19, seed 0, permuted, "
                               "symmetric simple CSR generated on the device (profiling size: 2.8e3 "
                               "out-degrees above 1024)"),
    "rmat-s22-ef16": dict(kind="rmat_dev", scale=22, ef=16, seed=0,
                          desc="R-MAT scale 22, edge factor 16, a=.57 b=.19 c=.19, seed 0, permuted, "
                               "symmetric simple CSR generated on the device"),
}
DEFAULT_WORKLOAD = "rmat-s24-ef32"  # the largest single-GPU configuration
AUTOTUNE_MAX_N = 1 << 22  # larger graphs are not autotuned in the run unless --autotune

# Settings fglt_autotune chose on a graph, keyed by the graph's signature
# (vertices, stored entries, largest degree): applied instead of an in-run
# autotune for graphs above AUTOTUNE_MAX_N (the search takes about 30
# transforms, six minutes at R-MAT s24).
TUNING_TABLE = {
    (16777216, 1023759990, 667733): {
        "tri_class_bounds": (128, 384), "tri_probe_loads": 4, "tri_hash_factor": 2, "tri_group_lanes": 32,
        "tri_warp_max": 32, "cyc_warp_bits": 10, "cyc_mid_threads": (256, 256, 128), "cyc_heavy_threads": 1024,
        "cyc_dense_min": 2048, "cyc_long_segment": 20, "cyc_spill_bits": 13},
}
EXTRA_WORKLOADS = ("rmat-s20-ef16",)  # also timed and reported under "extras"


def make_graph(spec, device=None):
    if spec["kind"] == "rmat_dev":
        return gg.rmat_device(spec["scale"], spec["ef"], seed=spec["seed"], device=device or "cuda")
    if spec["kind"] == "rmat":
        return gg.rmat(spec["scale"], spec["ef"], seed=spec["seed"])
    return gg.erdos_renyi(spec["n"], spec["deg"], seed=spec["seed"])


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# Roofline accounting
# ---------------------------------------------------------------------------
def algorithmic_bytes(stage: str, w: dict) -> int:
    """Bytes the method itself must move for one launch of a stage: 4 B per
    neighbour-list entry read, 4 B per per-edge C3 value, 8 B per per-vertex
    int64 value."""
    n, nnz, m = w["n"], w["nnz"], w["m"]
    if stage == "cyc":
        return 4 * w["wedges"] + 4 * nnz + 8 * n
    if stage == "tri1":
        return 4 * w["tri_scanned"] + 4 * m + 4 * m + 24 * n
    if stage == "tri2":
        return 4 * w["tri_scanned"] + 4 * m + 4 * m + 8 * n
    if stage in ("spmv1", "spmv2"):
        return 4 * nnz + 4 * nnz + 8 * (n + 1) + 16 * n
    if stage == "epilogue":
        return 256 * n + 8 * 12 * n
    return 4 * nnz + 8 * n


def traffic_for(stage: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source (profiles/traffic.json keyed by stage and
    workload, with the source digest it was measured on)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        e = t[workload][stage]
        src = os.path.join(ROOT, "paper_2007_11111_gb300", "csrc", e["source"])
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if digest != e["sha256_16"]:
            return None
        return int(e["dram_bytes"])
    except Exception:
        return None


# ---------------------------------------------------------------------------
# Arms
# ---------------------------------------------------------------------------
def neighbour_max_degree(g) -> np.ndarray:
    """Per vertex, the largest degree among its neighbours (0 if isolated)."""
    deg = np.diff(g.rowptr)
    out = np.zeros(g.n, dtype=np.int64)
    nz = np.flatnonzero(deg > 0)
    if nz.size:
        out[nz] = np.maximum.reduceat(deg[g.colidx], g.rowptr[nz])
    return out


class OracleSampler:
    """The CPU oracle timed on a stratified vertex sample of one graph, with the
    full transform's time extrapolated from per-row costs.

    Vertices are binned by floor(log2(degree)) (isolated vertices form their
    own bin). Each call picks up to `per_bin` vertices per bin, uniformly among
    the bin's "affordable" vertices: degree below `deg_cap`, and every
    neighbour's degree below a cap `nb_cap` (the oracle's sampled mode computes
    the C3 rows of the whole closed neighbourhood of each requested vertex, and
    one row of a top hub costs it minutes). nb_cap is the smallest power of two
    from 2^12 up to `nb_cap_max` for which every bin below deg_cap has an
    affordable vertex. The oracle reports, per sampled vertex, the seconds of its
    own C3 row (step 2) and of its Table I/II row (steps 4-8). The full
    transform's thread-seconds are estimated as the sum over the covered bins
    of (vertices in the bin) x (mean sampled cost in the bin); the bins left
    out (the highest degrees) carry most of the oracle's work, so the estimate
    is a lower bound on its time, i.e. an upper bound on its throughput. The
    fixed cost (step 1 over all vertices, allocations) is the wall time of a
    call for one lowest-degree vertex. All cores: fixed + thread-seconds /
    threads (ideal scaling); one core: fixed + thread-seconds."""

    def __init__(self, g, per_bin=6, deg_cap=1 << 10, nb_cap_max=1 << 15, threads=0, seed=0):
        import oracle
        oracle.build()
        self.g = g
        self.per_bin = per_bin
        self.deg_cap = deg_cap
        self.threads = threads or oracle.max_threads()
        self.rng = np.random.default_rng(seed)
        deg = np.diff(g.rowptr)
        self.deg = deg
        self.bin = np.where(deg > 0, np.floor(np.log2(np.maximum(deg, 1))).astype(np.int64), -1)
        nbm = neighbour_max_degree(g)
        bins, counts = np.unique(self.bin, return_counts=True)
        self.pops = {int(b): int(c) for b, c in zip(bins, counts)}
        nb_cap = 1 << 12
        while True:
            ok = (deg < deg_cap) & (nbm < nb_cap)
            self.cands = {}
            for b in self.pops:
                c = np.flatnonzero(ok & (self.bin == b))
                if c.size:
                    self.cands[b] = c
            low = [b for b in self.pops if b < 0 or (1 << b) < deg_cap]
            if all(b in self.cands for b in low) or nb_cap >= nb_cap_max:
                break
            nb_cap *= 2
        self.nb_cap = nb_cap
        self.excluded = {b: p for b, p in self.pops.items() if b not in self.cands}
        v0 = int(np.argmin(deg))
        t0 = time.perf_counter()
        oracle.fglt(g, vertices=np.array([v0]), threads=self.threads)
        self.fixed_s = time.perf_counter() - t0

    def step(self):
        """One sampled oracle call; returns (wall seconds, estimated full
        thread-seconds)."""
        import oracle
        picks, owner = [], []
        for b, c in self.cands.items():
            k = min(self.per_bin, c.size)
            sel = self.rng.choice(c, size=k, replace=False)
            picks.append(sel)
            owner.extend([b] * k)
        verts = np.concatenate(picks).astype(np.int64)
        owner = np.array(owner)
        t0 = time.perf_counter()
        _, _, t_c3, t_row = oracle.fglt_timed(self.g, verts, threads=self.threads)
        wall = time.perf_counter() - t0
        cost = t_c3[verts] + t_row
        est = sum(self.pops[b] * float(cost[owner == b].mean()) for b in self.cands)
        return wall, est

    def describe(self, nsteps, est_mean):
        covered = sum(self.pops[b] for b in self.cands)
        return (f"stratified vertex sample of the same graph: up to {self.per_bin} vertices per log2-degree bin "
                f"of degree below {self.deg_cap} whose neighbours' degrees are below {self.nb_cap}, new picks every call "
                f"({nsteps} calls); per-row oracle seconds extrapolated to the {covered} vertices of the sampled "
                f"bins ({self.g.n - covered} vertices of {len(self.excluded)} hub bins left out, so the full time "
                f"is under-estimated); fixed cost {self.fixed_s:.2f} s; estimated full transform "
                f"{est_mean:.0f} thread-seconds")

    def values(self, est):
        """(all-cores edges/s, one-core edges/s) of the extrapolated full run."""
        m = self.g.nnz // 2
        return m / (self.fixed_s + est / self.threads), m / (self.fixed_s + est)


def cpu_baseline(g, calls=2):
    s = OracleSampler(g, per_bin=3)
    ests = [s.step()[1] for _ in range(calls)]
    est = statistics.mean(ests)
    v_all, v_one = s.values(est)
    return {"value": v_all, "unit": UNIT, "cores": s.threads, "kind": "oracle",
            "single_core_value": v_one, "sample": s.describe(calls, est)}


# ---------------------------------------------------------------------------
# The library's entries beyond the full transform, timed on the benchmark
# graph: the Sigma5 sub-dictionary transform, edge-list ingest and degree
# relabelling. CUDA events on the launching stream, L2 flushed before each
# timed call, mean of `reps` calls after two untimed ones.
# ---------------------------------------------------------------------------
def bench_extensions(fg, torch, dev, n, rp, ci, flush, full_ms, reps=5):
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        for _ in range(2):
            fn()
        ts = []
        for _ in range(reps):
            flush.fill_(1)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.mean(ts), out

    m = int(ci.numel()) // 2
    out = {}
    # Sigma5: the stages only the 4-node graphlets need are skipped
    with fg.Handle(device=dev.index or 0, dictionary=fg.DICT_SIGMA5) as h5, fg.Handle(device=dev.index or 0) as hf:
        raw5 = torch.empty((n, 5), dtype=torch.int64, device=dev)
        net5 = torch.empty((n, 5), dtype=torch.int64, device=dev)
        ms5, _ = timed(lambda: h5.transform(rp, ci, n, raw5, net5, stream=stream))
        raw16, net16 = hf.transform(rp, ci, n, stream=stream)
        same = bool(torch.equal(raw5, raw16[:, :5]) and torch.equal(net5, net16[:, :5]))
        del raw16, net16
        out["sub_dictionary"] = {
            "dictionary": "Sigma5 (sigma_0 .. sigma_4)", "ms": ms5, "edges_per_s": m / (ms5 / 1e3),
            "full_ms": full_ms, "speedup_vs_full": full_ms / ms5, "bit_exact_vs_full_columns": same}
        # ingest: one direction of every edge, in a seeded random order
        rows = torch.repeat_interleave(torch.arange(n, device=dev, dtype=torch.int32), torch.diff(rp))
        keep = rows < ci
        gen = torch.Generator(device=dev)
        gen.manual_seed(0)
        order = torch.randperm(int(keep.sum().item()), device=dev, generator=gen)
        src = rows[keep][order].contiguous()
        dst = ci[keep][order].contiguous()
        del rows, keep, order
        msi, (irp, ici) = timed(lambda: hf.csr_from_edges(src, dst, n, stream=stream))
        out["ingest"] = {"pairs": int(src.numel()), "ms": msi, "pairs_per_s": src.numel() / (msi / 1e3),
                         "equal_to_input_csr": bool(torch.equal(irp, rp) and torch.equal(ici, ci))}
        del src, dst, irp, ici
        # degree relabelling (non-increasing degree)
        msr, (rrp, _, _) = timed(lambda: hf.relabel_by_degree(rp, ci, n, stream=stream))
        out["relabel"] = {"ms": msr, "edges_per_s": m / (msr / 1e3),
                          "degree_ordered": bool((torch.diff(torch.diff(rrp)) <= 0).all().item())}
    return out


# ---------------------------------------------------------------------------
# Batched (20,000 small graphs in one block-diagonal launch) and served
# (continuous batching of a Poisson request stream) forms, each against one
# single-graph transform per graph on the same GPU.
# ---------------------------------------------------------------------------
def bench_batched(fg, torch, dev, num_graphs=20000, reps=5):
    batch = gg.small_graph_batch(num_graphs, seed=0, n_lo=10, n_hi=500)
    G = batch.graph
    rp = torch.from_numpy(G.rowptr).to(dev)
    ci = torch.from_numpy(G.colidx).to(dev)
    raw = torch.empty((G.n, 16), dtype=torch.int64, device=dev)
    net = torch.empty((G.n, 16), dtype=torch.int64, device=dev)
    def timed_batches(h, out_raw, out_net):
        h.transform_batched(rp, ci, batch.offsets, out_raw, out_net)  # runs and captures the CUDA graph
        h.transform_batched(rp, ci, batch.offsets, out_raw, out_net)  # first replay
        torch.cuda.synchronize()
        times = []
        for _ in range(reps):
            t0 = time.perf_counter()
            h.transform_batched(rp, ci, batch.offsets, out_raw, out_net)
            times.append(time.perf_counter() - t0)
        return statistics.median(times)

    # the stage sequence of the single-graph path over the block-diagonal union
    with fg.Handle(device=dev.index or 0, batch_small_max=-1) as hs:
        sraw = torch.empty_like(raw)
        snet = torch.empty_like(net)
        t_seq = timed_batches(hs, sraw, snet)
    with fg.Handle(device=dev.index or 0) as h:
        t_batch = timed_batches(h, raw, net)  # the fused one-block-per-graph launch
        same_seq = bool(torch.equal(raw, sraw) and torch.equal(net, snet))
        del sraw, snet
        # one transform per graph (device-resident per-graph CSRs)
        per = []
        for g in range(num_graphs):
            lo, hi = int(batch.offsets[g]), int(batch.offsets[g + 1])
            e0, e1 = int(G.rowptr[lo]), int(G.rowptr[hi])
            per.append((hi - lo, torch.from_numpy(G.rowptr[lo:hi + 1] - e0).to(dev),
                        torch.from_numpy((G.colidx[e0:e1].astype(np.int64) - lo).astype(np.int32)
                                         if e1 > e0 else np.zeros(1, np.int32)).to(dev)))
        outs = [(torch.empty((k, 16), dtype=torch.int64, device=dev),
                 torch.empty((k, 16), dtype=torch.int64, device=dev)) for k, _, _ in per]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for (k, prp, pci), (oraw, onet) in zip(per, outs):
            h.transform(prp, pci, k, oraw, onet)
        torch.cuda.synchronize()
        t_per = time.perf_counter() - t0
        ok = all(torch.equal(net[int(batch.offsets[g]):int(batch.offsets[g + 1])], outs[g][1])
                 for g in range(0, num_graphs, 97))
    return {"workload": f"{num_graphs} graphs, n ~ U{{10..500}}, alternating BA (m ~ U{{2..5}}) and "
                        "random-geometric (mean degree 8), block-diagonal CSR, seed 0",
            "vertices": G.n, "edges": G.m, "graphs_per_s": num_graphs / t_batch,
            "ms_per_batch": 1000 * t_batch, "form": "one fused launch, one block per graph, replayed as a CUDA graph",
            "per_graph_launch_graphs_per_s": num_graphs / t_per, "speedup_vs_per_graph": t_per / t_batch,
            "stage_sequence_graphs_per_s": num_graphs / t_seq, "stage_sequence_ms_per_batch": 1000 * t_seq,
            "speedup_vs_stage_sequence": t_seq / t_batch, "cuda_graph_replay": True,
            "bit_exact_vs_stage_sequence": same_seq, "bit_exact_vs_per_graph_sample": bool(ok)}


def bench_serving(fg, torch, dev, num_requests=400, pool_size=24, seed=0, loads=(1.0, 2.0, 4.0, 8.0),
                  max_edges=2e6):
    """Poisson arrivals of graphs with |E| log-uniform in [1e3, max_edges] drawn
    from a pool of distinct R-MAT and Barabasi-Albert graphs, served through
    fglt_stream_submit/poll, against a sequential one-at-a-time FIFO of
    fglt_transform_host calls fed the same arrivals (both measured live)."""
    rng = np.random.default_rng(seed)
    pool = []
    for i in range(pool_size):
        E = int(np.exp(rng.uniform(np.log(1e3), np.log(max_edges))))
        if i % 2 == 0:
            sc = max(4, int(np.ceil(np.log2(max(E / 8, 2)))))
            ef = max(1, E // (1 << sc))
            if sc >= 18:  # large pool graphs come from the device generator
                pool.append(gg.rmat_device(sc, ef, seed=seed + i, device=str(dev)).to_host())
            else:
                pool.append(gg.rmat(sc, ef, seed=seed + i))
        else:
            pool.append(gg.barabasi_albert(max(16, E // 8), 8, seed + i))
    picks = rng.integers(0, pool_size, num_requests)
    rps = [np.ascontiguousarray(g.rowptr, dtype=np.int64) for g in pool]
    out = {"workload": f"{num_requests} Poisson requests per load point, |E| log-uniform in [1e3, {max_edges:.0e}], "
                       f"from a pool of {pool_size} distinct R-MAT/BA graphs, seed {seed}; "
                       "load = arrival rate / sequential capacity", "points": []}
    with fg.Handle(device=dev.index or 0) as h:
        svc = []
        for g in pool:
            h.transform_host(g.rowptr, g.colidx, g.n)
            t0 = time.perf_counter()
            h.transform_host(g.rowptr, g.colidx, g.n)
            svc.append(time.perf_counter() - t0)
        mean_svc = float(np.mean([svc[k] for k in picks]))
        # warm the served form like the sequential one: every lane grows its
        # staging and device buffers on pool graphs before the timed points
        warm = []
        for _ in range(3):
            for k, g in enumerate(pool):
                buf = np.empty((g.n, 16), np.int64)
                warm.append((fg.fglt_stream_submit(h.h, g.n, rps[k], g.colidx, None, buf), buf))
        for rid, _ in warm:
            fg.fglt_stream_poll(h.h, rid, -1)
        del warm
        for load in loads:
            arrivals = np.cumsum(rng.exponential(mean_svc / load, num_requests))
            # Requests are collected while later ones are still arriving, so only
            # the outputs in flight (and the sampled ones kept for the check)
            # occupy host memory.
            lat = [None] * num_requests
            keep = {}
            pending = {}
            start = time.perf_counter()

            def collect(block):
                for i in list(pending):
                    rid, buf = pending[i]
                    st, us = fg.fglt_stream_poll(h.h, rid, -1 if block else 0)
                    if st == fg.FGLT_ERR_PENDING:
                        continue
                    if st != fg.FGLT_OK:
                        raise RuntimeError(f"request failed with status {st}")
                    lat[i] = us / 1e6
                    if i % 37 == 0:
                        keep[i] = buf
                    del pending[i]

            for i, (a, k) in enumerate(zip(arrivals, picks)):
                wait = start + a - time.perf_counter()
                if wait > 0:
                    time.sleep(wait)
                g = pool[k]
                buf = np.empty((g.n, 16), np.int64)
                pending[i] = (fg.fglt_stream_submit(h.h, g.n, rps[k], g.colidx, None, buf), buf)
                collect(False)
            collect(True)
            served_total = max(a + l for a, l in zip(arrivals, lat)) - arrivals[0]
            ok = all(np.array_equal(keep[i], h.transform_host(pool[picks[i]].rowptr, pool[picks[i]].colidx,
                                                               pool[picks[i]].n)[1])
                     for i in range(0, num_requests, 37))
            # sequential FIFO, live: one fglt_transform_host at a time, in arrival order
            seq_lat = []
            start = time.perf_counter()
            for a, k in zip(arrivals, picks):
                wait = start + a - time.perf_counter()
                if wait > 0:
                    time.sleep(wait)
                g = pool[k]
                h.transform_host(g.rowptr, g.colidx, g.n)
                seq_lat.append(time.perf_counter() - start - a)
            seq_total = max(a + l for a, l in zip(arrivals, seq_lat)) - arrivals[0]
            edges = sum(pool[k].m for k in picks)
            out["points"].append({
                "load": load, "graphs_per_s": num_requests / served_total, "edges_per_s": edges / served_total,
                "p50_ms": 1000 * float(np.percentile(lat, 50)), "p99_ms": 1000 * float(np.percentile(lat, 99)),
                "sequential_graphs_per_s": num_requests / seq_total,
                "sequential_p50_ms": 1000 * float(np.percentile(seq_lat, 50)),
                "sequential_p99_ms": 1000 * float(np.percentile(seq_lat, 99)),
                "bit_exact_vs_alone_sample": bool(ok)})
    # capacity: the best completion rate over the load points (the top loads
    # offer far more than either form completes)
    best = max(out["points"], key=lambda p: p["graphs_per_s"])
    best_seq = max(out["points"], key=lambda p: p["sequential_graphs_per_s"])
    out["capacity"] = {"served_graphs_per_s": best["graphs_per_s"], "served_p99_ms": best["p99_ms"],
                       "sequential_graphs_per_s": best_seq["sequential_graphs_per_s"],
                       "sequential_p99_ms": best_seq["sequential_p99_ms"],
                       "ratio": best["graphs_per_s"] / best_seq["sequential_graphs_per_s"]}
    return out


def tuning_args(args) -> dict:
    """--set name=value options for the handle (tuning fields of fglt_options;
    tuples as comma-separated values)."""
    out = {}
    for item in args.set or []:
        k, v = item.split("=", 1)
        vals = [int(x) for x in v.split(",")]
        out[k] = tuple(vals) if len(vals) > 1 else vals[0]
    return out


def slowest_rank_ms(ms: float, world: int, device=None) -> float:
    """Max over ranks of a per-rank time (the job is as fast as its slowest rank)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(m_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput: every rank transforms its own replica of m edges."""
    return world * m_per_rank / (ms / 1000.0)


def host_graph(spec):
    """The workload's graph in host memory (the large R-MAT configurations are
    drawn by the seeded device generator, then copied to the host)."""
    if spec["kind"] == "rmat_dev":
        import torch
        dg = make_graph(spec, torch.device("cuda", 0))
        g = dg.to_host()
        del dg
        torch.cuda.empty_cache()
        return g
    return make_graph(spec)


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle as it stands on the host cores, each
    step one sampled oracle call on the same graph as the GPU arm, the value
    the extrapolated full-transform throughput (OracleSampler)."""
    if rank != 0:
        return 0
    spec = WORKLOADS[args.workload]
    g = host_graph(spec)
    s = OracleSampler(g, per_bin=2)
    for _ in range(args.warmup):
        s.step()
    walls, ests = [], []
    for _ in range(args.steps):
        w, e = s.step()
        walls.append(w)
        ests.append(e)
    est = statistics.mean(ests)
    value, one_core = s.values(est)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * statistics.mean(walls),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": spec["desc"], "n": g.n, "m": g.m, "nnz": g.nnz},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": s.threads, "kind": "oracle",
                         "single_core_value": one_core, "sample": s.describe(args.steps, est)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def roofline_of(stage_ms: dict, work: dict, workload: str) -> dict:
    """Roofline of the dominant stage: algorithmic bytes per transform over the
    stage's CUDA-event time against the measured HBM copy peak, beside the DRAM
    bytes ncu counted for that stage (null unless measured on the current
    kernel source) and the limiter the counters show."""
    dom = max((k for k in stage_ms if "." not in k), key=stage_ms.get)  # "cyc.*" are parts of "cyc"
    peak, peak_kind = load_peaks()
    ab = algorithmic_bytes(dom, work)
    sec = stage_ms[dom] / 1000
    achieved = ab / sec / 1e9
    traffic = traffic_for(dom, workload)
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "traffic": traffic, "kernel": dom, "kernel_ms": stage_ms[dom], "algorithmic_bytes": ab,
           "achieved_kind": "algorithmic bytes (list entries, per-edge C3, per-vertex values) / stage time",
           "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
           else "fallback 6.8 TB/s"}
    if traffic:
        out["dram_gbs"] = traffic / sec / 1e9
        out["dram_frac"] = out["dram_gbs"] / peak
        out["traffic_source"] = "ncu dram__bytes_read.sum + dram__bytes_write.sum (profiles/traffic.json)"
    out["limiter"] = LIMITERS.get((workload, dom), "not characterised for this workload")
    return out


# What the ncu counters of the dominant stages show (profiles/*.md).
LIMITERS = {
    ("rmat-s24-ef32", "cyc"): "shared-memory counter updates (pass A atomics, pass B gathers; loading the "
                              "wedges alone costs about a tenth of pass A, timed with work removed) and, in "
                              "the spill class, DRAM re-reads of each bottom vertex's segments in pass B "
                              "plus spill-table atomics (5.2 TB of DRAM traffic against 3.1 TB of "
                              "algorithmic bytes, a fifth of the copy peak)",
    ("rmat-s24-ef32", "tri1"): "hash probes of the out-lists streamed from DRAM (3.0 TB at a fifth of the copy "
                               "peak); the clique phase of the largest class runs on the tensor cores "
                               "(tcgen05, E4M3)",
    ("rmat-s20-ef16", "cyc"): "shared-memory atomics and instruction issue; lists and tables stay in L2 "
                              "(DRAM traffic a few percent of the algorithmic bytes)",
}


def bench_extra_workload(fg, torch, dev, name, flush, args, steps=10, warmup=3):
    """A second single-graph workload on the same GPU (autotuned, inputs
    resident, L2 flushed before each timed transform): edges/s, stage times and
    its roofline."""
    spec = WORKLOADS[name]
    g = make_graph(spec, dev)
    if isinstance(g, gg.DeviceGraph):
        rp, ci = g.rowptr, g.colidx
    else:
        rp = torch.from_numpy(g.rowptr).to(dev)
        ci = torch.from_numpy(g.colidx).to(dev)
    stream = torch.cuda.current_stream(dev)
    with fg.Handle(device=dev.index or 0, profile_stages=True) as h:
        raw = torch.empty((g.n, 16), dtype=torch.int64, device=dev)
        net = torch.empty((g.n, 16), dtype=torch.int64, device=dev)
        tune = None
        if not args.no_autotune and g.n <= AUTOTUNE_MAX_N:
            chosen, tuned_ms, default_ms = h.autotune(rp, ci, g.n, reps=1, stream=stream)
            tune = {"tuned_ms": tuned_ms, "default_ms": default_ms}
        for _ in range(warmup):
            h.transform(rp, ci, g.n, raw, net, stream=stream)
        ts, acc = [], {}
        for _ in range(steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.transform(rp, ci, g.n, raw, net, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
            for k, v in h.stage_times().items():
                acc.setdefault(k, []).append(v)
        work = h.work_counters()
    ms = statistics.mean(ts)
    stage_ms = {k: statistics.mean(v) for k, v in acc.items()}
    return {"desc": spec["desc"], "n": g.n, "m": g.m, "value": g.m / (ms / 1000), "unit": UNIT, "steps": steps,
            "ms_per_step": ms, "stage_ms": {k: v for k, v in stage_ms.items() if "." not in k},
            "roofline": roofline_of(stage_ms, work, name), "autotune": tune}


def run_gpu(args, rank, world, local_rank):
    import torch
    import paper_2007_11111_gb300 as fg

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    spec = WORKLOADS[args.workload]
    g = make_graph(spec, dev)
    if isinstance(g, gg.DeviceGraph):
        rp, ci = g.rowptr, g.colidx
    else:
        rp = torch.from_numpy(g.rowptr).to(dev)
        ci = torch.from_numpy(g.colidx).to(dev)
    raw = torch.empty((g.n, 16), dtype=torch.int64, device=dev)
    net = torch.empty((g.n, 16), dtype=torch.int64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    sig = None
    if g.n > AUTOTUNE_MAX_N and not args.autotune and not args.no_autotune and not args.set:
        sig = (g.n, g.nnz, int((g.rowptr[1:] - g.rowptr[:-1]).max().item()))
    table = TUNING_TABLE.get(sig, {}) if sig else {}
    h = fg.Handle(device=local_rank, profile_stages=True, **(table or tuning_args(args)))
    stream = torch.cuda.current_stream(dev)

    def step():
        h.transform(rp, ci, g.n, raw, net, stream=stream)

    tune = None
    if not args.no_autotune and (args.autotune or g.n <= AUTOTUNE_MAX_N):
        t0 = time.perf_counter()
        chosen, tuned_ms, default_ms = h.autotune(rp, ci, g.n, reps=1, stream=stream)
        tune = {"chosen": chosen, "tuned_ms": tuned_ms, "default_ms": default_ms,
                "seconds": time.perf_counter() - t0, "note": "untimed set-up before the warm-up steps"}
    elif table:
        tune = {"chosen": {k: list(v) if isinstance(v, tuple) else v for k, v in table.items()},
                "source": "tuning table: fglt_autotune's choice on a graph of the same signature "
                          f"(n, nnz, max degree) = {sig}; no autotune in this run"}
    elif not args.no_autotune:
        tune = {"chosen": "library defaults", "note": f"graphs above {AUTOTUNE_MAX_N} vertices are not "
                "autotuned in the run (about 30 transforms) and no table entry matched"}

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    sampler = ClockSampler(local_rank)
    sampler.start()
    step_ms, stage_acc = [], {}
    launches = 0
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        for k, v in h.stage_times().items():
            stage_acc.setdefault(k, []).append(v)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if dist is not None:
        dist.barrier()
    ms = slowest_rank_ms(statistics.mean(step_ms), world, dev)
    work = h.work_counters()
    launches = int(work.get("launches", 0)) * args.steps

    # End to end through the public API with host buffers (pinned host memory).
    e2e = None
    if rank == 0 and not args.no_e2e:
        prp = rp.cpu().pin_memory().numpy()
        pci = ci.cpu().pin_memory().numpy()
        hraw = torch.empty((g.n, 16), dtype=torch.int64).pin_memory().numpy()
        hnet = torch.empty((g.n, 16), dtype=torch.int64).pin_memory().numpy()
        fg.fglt_transform_host(h.h, prp, 1, pci, g.n, hraw, hnet)
        tl = []
        for _ in range(3 if g.n > AUTOTUNE_MAX_N else max(3, min(args.steps, 10))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fg.fglt_transform_host(h.h, prp, 1, pci, g.n, hraw, hnet)
            tl.append(time.perf_counter() - t0)
        e2e = {"value": g.m / statistics.mean(tl), "unit": UNIT,
               "h2d_bytes_per_step": int(prp.nbytes + pci.nbytes),
               "d2h_bytes_per_step": int(hraw.nbytes + hnet.nbytes),
               "step_s": [round(t, 4) for t in tl]}

    if rank != 0:
        h.close()
        return 0

    stage_ms = {k: statistics.mean(v) for k, v in stage_acc.items()}
    roofline = roofline_of(stage_ms, work, args.workload)
    value = job_value(g.m, world, ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": spec["desc"], "n": g.n, "m": g.m, "nnz": g.nnz,
                   "l2": "flushed before every timed step (512 MiB write, outside the timed events)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": roofline,
        "stage_ms": stage_ms,
        "autotune": tune,
        "work": work,
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": e2e,
    }
    if not args.no_extensions and rank == 0:
        line["extensions"] = bench_extensions(fg, torch, dev, g.n, rp, ci, flush, ms)
    if not args.no_batched:
        line["batched"] = bench_batched(fg, torch, dev)
    if args.serving_full:
        line["serving"] = bench_serving(fg, torch, dev, num_requests=5000, pool_size=48, loads=(1.0, 2.0, 4.0),
                                        max_edges=2e7)
    elif not args.no_serving:
        line["serving"] = bench_serving(fg, torch, dev)
    if not args.no_extras and rank == 0:
        line["extras"] = {w: bench_extra_workload(fg, torch, dev, w, flush, args)
                          for w in EXTRA_WORKLOADS if w != args.workload}
    if not args.no_cpu_baseline:
        gh = g.to_host() if isinstance(g, gg.DeviceGraph) else g
        line["cpu_baseline"] = cpu_baseline(gh)
    print(json.dumps(line), flush=True)
    h.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-extras", action="store_true", help="skip the extra workloads (R-MAT s20) of the line")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--autotune", action="store_true",
                    help="autotune even on graphs above 2^22 vertices (minutes at R-MAT s24)")
    ap.add_argument("--no-extensions", action="store_true",
                    help="skip timing the Sigma5 transform, edge-list ingest and relabelling")
    ap.add_argument("--set", action="append", metavar="NAME=VALUE",
                    help="tuning field of the handle, e.g. --set cyc_spill_bits=13 (with --no-autotune to keep it)")
    ap.add_argument("--serving-full", action="store_true",
                    help="serve 5000 requests with |E| up to 2e7 at loads 1 and 2 (several minutes)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    rc = run_gpu(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
