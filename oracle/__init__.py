"""CPU oracle of the Fast Graphlet Transform.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers. The product path (the CUDA
library and its Python binding) never imports this package.

``fglt(graph)`` runs the plain int64 C implementation in ``fglt_oracle.c``
(Table I formulas, then Table II back substitution). ``brute`` holds an
independent brute-force enumeration used to pin it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fglt_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libfglt_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over vertices)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(path):
    lib = ctypes.CDLL(path)
    i64p = ctypes.POINTER(ctypes.c_int64)
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib.oracle_fglt.argtypes = [ctypes.c_int64, i64p, i32p, i64p, ctypes.c_int64,
                                i64p, i64p, ctypes.c_int]
    lib.oracle_fglt.restype = ctypes.c_int
    f64p = ctypes.POINTER(ctypes.c_double)
    lib.oracle_fglt_timed.argtypes = [ctypes.c_int64, i64p, i32p, i64p, ctypes.c_int64,
                                      i64p, i64p, ctypes.c_int, f64p, f64p]
    lib.oracle_fglt_timed.restype = ctypes.c_int
    lib.oracle_raw_to_net.argtypes = [ctypes.c_int64, i64p, i64p]
    lib.oracle_raw_to_net.restype = None
    lib.oracle_raw_to_net_sub.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_int), i64p, i64p]
    lib.oracle_raw_to_net_sub.restype = None
    lib.oracle_u16.argtypes = [i64p]
    lib.oracle_u16.restype = None
    lib.oracle_max_threads.argtypes = []
    lib.oracle_max_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(_LIB_PATH)
    return _lib


def _p64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _p32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def fglt(graph, vertices=None, threads: int = 0, _lib_override=None, dictionary: int = 0):
    """Raw and net frequencies (int64, shape [rows, 16], or [rows, |s|] for a
    sub-dictionary).

    graph: any object with n, rowptr (int64[n+1]) and colidx (int32[nnz]).
    vertices: None for all vertices, else the rows to compute (in that order).
    threads: OpenMP threads (0 = all available).
    dictionary: 0 for Sigma16, else the bit mask of a sub-dictionary s (bit k
    = sigma_k): raw(s) are the Table I rows in s and net(s) = U16(s,s)^{-1}
    raw(s), the conversion the caption of Table II gives for s."""
    if dictionary not in (0, 0xFFFF):
        raw, _ = fglt(graph, vertices, threads, _lib_override)
        return sub_dictionary(raw, dictionary)
    lib = _lib_override if _lib_override is not None else _load()
    n = int(graph.n)
    rowptr = np.ascontiguousarray(graph.rowptr, dtype=np.int64)
    colidx = np.ascontiguousarray(graph.colidx, dtype=np.int32)
    if colidx.size == 0:
        colidx = np.zeros(1, np.int32)
    if vertices is None:
        rows = n
        vp = ctypes.POINTER(ctypes.c_int64)()
    else:
        verts = np.ascontiguousarray(vertices, dtype=np.int64)
        rows = verts.size
        vp = _p64(verts)
    raw = np.zeros((max(rows, 1), 16), dtype=np.int64)
    net = np.zeros((max(rows, 1), 16), dtype=np.int64)
    rc = lib.oracle_fglt(n, _p64(rowptr), _p32(colidx), vp, rows if vertices is not None else 0,
                         _p64(raw), _p64(net), int(threads))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return raw[:rows], net[:rows]


def fglt_timed(graph, vertices, threads: int = 0):
    """Sampled-mode rows (as ``fglt(graph, vertices)``) plus per-row wall
    seconds: t_c3[j] for the C3 row of every vertex j whose row step 2
    computed (0 elsewhere) and t_row[r] for steps 4-8 of output row r. The
    timers are measurements for the benchmark's CPU baseline; the results are
    the same as ``fglt``'s."""
    lib = _load()
    n = int(graph.n)
    rowptr = np.ascontiguousarray(graph.rowptr, dtype=np.int64)
    colidx = np.ascontiguousarray(graph.colidx, dtype=np.int32)
    if colidx.size == 0:
        colidx = np.zeros(1, np.int32)
    verts = np.ascontiguousarray(vertices, dtype=np.int64)
    rows = verts.size
    raw = np.zeros((max(rows, 1), 16), dtype=np.int64)
    net = np.zeros((max(rows, 1), 16), dtype=np.int64)
    t_c3 = np.zeros(max(n, 1), dtype=np.float64)
    t_row = np.zeros(max(rows, 1), dtype=np.float64)
    f64p = ctypes.POINTER(ctypes.c_double)
    rc = lib.oracle_fglt_timed(n, _p64(rowptr), _p32(colidx), _p64(verts), rows, _p64(raw), _p64(net),
                               int(threads), t_c3.ctypes.data_as(f64p), t_row.ctypes.data_as(f64p))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return raw[:rows], net[:rows], t_c3[:n], t_row[:rows]


def sub_dictionary(raw16: np.ndarray, mask: int):
    """(raw(s), net(s)) of sub-dictionary s (bit mask) from Sigma16 raw rows."""
    cols = [k for k in range(16) if (mask >> k) & 1]
    if mask >> 16 or 0 not in cols or 1 not in cols:
        raise ValueError("a sub-dictionary holds sigma_0 and sigma_1 and indices below 16")
    raw = np.ascontiguousarray(raw16[:, cols], dtype=np.int64)
    net = np.zeros_like(raw)
    c = (ctypes.c_int * len(cols))(*cols)
    _load().oracle_raw_to_net_sub(raw.shape[0], len(cols), c, _p64(raw), _p64(net))
    return raw, net


def raw_to_net(raw: np.ndarray) -> np.ndarray:
    lib = _load()
    raw = np.ascontiguousarray(raw, dtype=np.int64)
    net = np.zeros_like(raw)
    lib.oracle_raw_to_net(raw.shape[0], _p64(raw), _p64(net))
    return net


def u16() -> np.ndarray:
    """Table II as stored in the oracle (row = raw index, column = net index)."""
    lib = _load()
    out = np.zeros((16, 16), dtype=np.int64)
    lib.oracle_u16(_p64(out))
    return out


def max_threads() -> int:
    return int(_load().oracle_max_threads())
