"""The oracle's pins catch plausible mistakes.

Each case plants one mistake (a dropped term, a wrong sign, coefficient or index,
a transposed operand) in a temporary copy of the oracle's C source, builds it on
the CPU and checks that the Fig. 2 tables or the brute-force enumeration reject
it. The committed oracle itself is never modified.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle.brute import brute_fglt, edges_of
from conftest import read_golden_sections

SRC = os.path.join(os.path.dirname(oracle.__file__), "fglt_oracle.c")

MUTANTS = {
    "p2 drops c2": ("p2[i] = rsub(s, p1[i]);", "p2[i] = s;"),
    "p3 keeps one triangle term": ("p3[i] = rsub(rsub(s, p1[i] * rsub(p1[i], 1)), 2 * c3[i]);",
                                   "p3[i] = rsub(rsub(s, p1[i] * rsub(p1[i], 1)), c3[i]);"),
    "p3 drops backtrack": ("p3[i] = rsub(rsub(s, p1[i] * rsub(p1[i], 1)), 2 * c3[i]);",
                           "p3[i] = rsub(s, 2 * c3[i]);"),
    "c3 not halved": ("c3[i] = s / 2;", "c3[i] = s;"),
    "d6 sign": ("f[6] = rsub(p2[i] * rsub(d, 1), 2 * c3[i]);", "f[6] = p2[i] * rsub(d, 1) + 2 * c3[i];"),
    "d7 uses own degree": ("Ap1m += rsub(p1[j], 1) * rsub(p1[j], 2);",
                           "Ap1m += rsub(p1[i], 1) * rsub(p1[j], 2);"),
    "d9 coefficient": ("f[9] = rsub(Ac3, 2 * c3[i]);", "f[9] = rsub(Ac3, c3[i]);"),
    "d10 offset": ("C3p1m2 += C3[e] * rsub(p1[j], 2);", "C3p1m2 += C3[e] * rsub(p1[j], 1);"),
    "d11 transposed": ("f[11] = rsub(d, 2) * c3[i];", "f[11] = rsub(d, 2) * p2[i];"),
    "c4 not halved": ("r.c4 = c42 / 2;", "r.c4 = c42;"),
    "c4 keeps l == i": ("if (l == i) continue;", ""),
    "D4c without -A": ("d4c += rsub(C3[g->rp[j] + qpos[s]], 1);", "d4c += C3[g->rp[j] + qpos[s]];"),
    "intersect (long first list) position": ("{ val[c] = b[y]; posb[c] = y; c++; }",
                                             "{ val[c] = b[y]; posb[c] = 0; c++; }"),
    "intersect (long second list) value": ("if (y >= 0) { val[c] = a[x]; posb[c] = y; c++; }",
                                           "if (y >= 0) { val[c] = b[0]; posb[c] = y; c++; }"),
    "C3 binary search misses": ("for (i64 x = 0; x < ns; x++) c += find_pos(l, nl, s[x]) >= 0;",
                                "for (i64 x = 1; x < ns; x++) c += find_pos(l, nl, s[x]) >= 0;"),
    "D4,3 wrong index": ("i64 p = acc[Ni[x]];", "i64 p = acc[x];"),
    "T divisor": ("f[15] = qt.T / 6;", "f[15] = qt.T / 3;"),
    "U16 entry": ("/* 5 */ { 0, 0, 0, 0, 0, 1, 0, 0, 0, 2, 1, 0, 2, 4, 2, 6 },",
                  "/* 5 */ { 0, 0, 0, 0, 0, 1, 0, 0, 0, 2, 1, 0, 2, 2, 2, 6 },"),
    "U16 transposed entry": ("/* 9 */ { 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0, 0, 2, 0, 3 },",
                             "/* 9 */ { 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0, 0, 0, 2, 3 },"),
}


def _build_mutant(tmpdir, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutant anchor not unique: {name}"
    path_c = os.path.join(tmpdir, "m.c")
    path_so = os.path.join(tmpdir, "m.so")
    with open(path_c, "w") as f:
        f.write(src.replace(old, new))
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-shared", "-fPIC", path_c, "-o", path_so],
                   check=True)
    return oracle._bind(path_so)


def _pins_pass(lib):
    sec = read_golden_sections("fig2_example.txt")
    g = gg.from_edge_list(6, [(a - 1, b - 1) for a, b in sec["edges"]])
    raw, net = oracle.fglt(g, _lib_override=lib)
    if not (np.array_equal(raw, [r[1:] for r in sec["raw"]])
            and np.array_equal(net, [r[1:] for r in sec["net"]])):
        return False
    for seed in range(30):
        rng = np.random.default_rng(1000 + seed)
        n = int(rng.integers(4, 10))
        i, j = np.triu_indices(n, 1)
        keep = rng.random(i.size) < rng.uniform(0.2, 0.8)
        h = gg.csr_from_pairs(n, i[keep], j[keep])
        rb, nb = brute_fglt(h.n, edges_of(h))
        r, nn = oracle.fglt(h, _lib_override=lib)
        if not (np.array_equal(r, rb) and np.array_equal(nn, nb)):
            return False
    for seed in range(12):  # hub graphs: degree ratios above 8 take the binary-search intersections
        h = hub_graph(seed)
        rb, nb = brute_fglt(h.n, edges_of(h))
        r, nn = oracle.fglt(h, _lib_override=lib)
        if not (np.array_equal(r, rb) and np.array_equal(nn, nb)):
            return False
    return True


def hub_graph(seed, n=27):
    """Vertex n//2 joined to every other vertex, plus a few random edges among
    the others (two of them stay pendant): the hub's degree is more than 8
    times that of the vertices of degree up to 3, and it sits in the middle of
    their sorted neighbour lists."""
    rng = np.random.default_rng(2000 + seed)
    hub = n // 2
    others = np.array([v for v in range(n) if v != hub], np.int64)
    i, j = np.triu_indices(n - 1, 1)
    keep = (rng.random(i.size) < 0.08) & (i >= 2)  # others[0] and others[1] stay pendant
    src = np.concatenate([np.full(n - 1, hub, np.int64), others[i[keep]]])
    dst = np.concatenate([others, others[j[keep]]])
    return gg.csr_from_pairs(n, src, dst)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name):
    old, new = MUTANTS[name]
    with tempfile.TemporaryDirectory() as d:
        lib = _build_mutant(d, name, old, new)
        assert not _pins_pass(lib), f"pins did not catch mutant: {name}"


def test_unmutated_copy_passes():
    with tempfile.TemporaryDirectory() as d:
        lib = _build_mutant(d, "identity", "r.c4 = c42 / 2;", "r.c4 = c42 / 2;")
        assert _pins_pass(lib)
