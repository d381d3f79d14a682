"""Python binding of the GB300 Fast Graphlet Transform library (libfglt.so).

Argument marshalling only: every step of the transform runs in the library's
CUDA kernels. The names mirror the C ABI declared in include/fglt.h
(fglt_create, fglt_transform, ...). Device buffers are passed as torch CUDA
tensors (or raw integer device pointers); host buffers as numpy arrays.

There is no CPU fallback: if the library is missing or fails to load, every
call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import buildlib as _build

NUM_GRAPHLETS = 16
DICT_SIGMA5 = 0x1F  # sigma_0 .. sigma_4


def dictionary_mask(sigmas) -> int:
    """Bit mask of a sub-dictionary given as sigma indices (e.g. range(5))."""
    m = 0
    for k in sigmas:
        m |= 1 << int(k)
    return m


def dictionary_columns(mask: int) -> int:
    return 16 if mask in (0, 0xFFFF) else bin(mask).count("1")

FGLT_OK = 0
FGLT_ERR_INVALID_ARG = 1
FGLT_ERR_INVALID_GRAPH = 2
FGLT_ERR_OOM = 3
FGLT_ERR_OVERFLOW = 4
FGLT_ERR_CUDA = 5
FGLT_ERR_TIMEOUT = 6
FGLT_ERR_PENDING = 7
FGLT_ERR_NOT_FOUND = 8
FGLT_ERR_INTERNAL = 9
FGLT_ERR_UNSUPPORTED = 10
FGLT_ERR_BUSY = 11
FGLT_ERR_CANCELLED = 12


class FgltError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} (status {status})")
        self.status = status


class fglt_options(ctypes.Structure):
    _fields_ = [
        ("validate", ctypes.c_int),
        ("serve_memory_budget", ctypes.c_size_t),
        ("serve_max_batch", ctypes.c_int),
        ("serve_max_queue", ctypes.c_int),
        ("profile_stages", ctypes.c_int),
        ("cyc_hub_span", ctypes.c_int),
        ("tri_class_bounds", ctypes.c_int * 2),
        ("tri_probe_loads", ctypes.c_int),
        ("tri_hash_factor", ctypes.c_int),
        ("tri_group_lanes", ctypes.c_int),
        ("tri_warp_max", ctypes.c_int),
        ("cyc_warp_bits", ctypes.c_int),
        ("cyc_mid_threads", ctypes.c_int * 3),
        ("cyc_heavy_threads", ctypes.c_int),
        ("cyc_dense_min", ctypes.c_int),
        ("cyc_long_segment", ctypes.c_int),
        ("cyc_spill_bits", ctypes.c_int),
        ("dictionary_mask", ctypes.c_uint),
        ("batch_small_max", ctypes.c_int),
        ("tri_pass2_from", ctypes.c_int),
        ("device_wait_limit_ns", ctypes.c_longlong),
    ]

    def tuning(self) -> dict:
        """The tuning fields (0 = default)."""
        return {"cyc_hub_span": self.cyc_hub_span, "tri_class_bounds": list(self.tri_class_bounds),
                "tri_probe_loads": self.tri_probe_loads, "tri_hash_factor": self.tri_hash_factor,
                "tri_group_lanes": self.tri_group_lanes, "tri_warp_max": self.tri_warp_max,
                "cyc_warp_bits": self.cyc_warp_bits, "cyc_mid_threads": list(self.cyc_mid_threads),
                "cyc_heavy_threads": self.cyc_heavy_threads, "cyc_dense_min": self.cyc_dense_min,
                "cyc_long_segment": self.cyc_long_segment, "cyc_spill_bits": self.cyc_spill_bits,
                "tri_pass2_from": self.tri_pass2_from}


class fglt_graph_host(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("rowptr", ctypes.POINTER(ctypes.c_int64)),
        ("colidx", ctypes.POINTER(ctypes.c_int32)),
        ("out_raw", ctypes.POINTER(ctypes.c_int64)),
        ("out_net", ctypes.POINTER(ctypes.c_int64)),
    ]


EXPORTED = [
    "fglt_options_default", "fglt_create", "fglt_destroy", "fglt_status_string", "fglt_last_cuda_error",
    "fglt_transform", "fglt_transform_host", "fglt_transform_batched", "fglt_stage_times", "fglt_work_counters",
    "fglt_stream_submit", "fglt_stream_poll", "fglt_stream_cancel", "fglt_transform_noalloc", "fglt_autotune",
    "fglt_csr_from_edges", "fglt_csr_relabel_by_degree",
]

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libfglt.so (building it first if needed). Raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"the FGLT CUDA library is not built ({path}); run build()")
    lib = ctypes.CDLL(path)
    vp, i64, i32, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
    h_t = ctypes.c_void_p
    lib.fglt_options_default.argtypes = [ctypes.POINTER(fglt_options)]
    lib.fglt_create.argtypes = [ctypes.POINTER(h_t), ctypes.POINTER(fglt_options), c_int]
    lib.fglt_destroy.argtypes = [h_t]
    lib.fglt_status_string.argtypes = [c_int]
    lib.fglt_status_string.restype = ctypes.c_char_p
    lib.fglt_last_cuda_error.argtypes = [h_t]
    lib.fglt_last_cuda_error.restype = ctypes.c_char_p
    lib.fglt_transform.argtypes = [h_t, vp, c_int, vp, i64, vp, vp, vp]
    lib.fglt_transform_host.argtypes = [h_t, vp, c_int, vp, i64, vp, vp]
    lib.fglt_transform_batched.argtypes = [h_t, vp, c_int, vp, ctypes.POINTER(i64), i64, vp, vp, vp]
    lib.fglt_stage_times.argtypes = [h_t, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_float),
                                     c_int, ctypes.POINTER(c_int)]
    lib.fglt_transform_noalloc.argtypes = [vp, c_int, vp, i64, vp, vp, vp]
    lib.fglt_csr_from_edges.argtypes = [h_t, vp, vp, i64, i64, vp, vp, ctypes.POINTER(i64), vp]
    lib.fglt_csr_relabel_by_degree.argtypes = [h_t, vp, c_int, vp, i64, c_int, vp, vp, vp, vp]
    lib.fglt_autotune.argtypes = [h_t, vp, c_int, vp, i64, c_int, vp, ctypes.POINTER(fglt_options),
                                  ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]
    lib.fglt_work_counters.argtypes = [h_t, ctypes.POINTER(ctypes.c_int64), c_int, ctypes.POINTER(c_int)]
    lib.fglt_stream_submit.argtypes = [h_t, ctypes.POINTER(fglt_graph_host), ctypes.POINTER(ctypes.c_uint64)]
    lib.fglt_stream_poll.argtypes = [h_t, ctypes.c_uint64, c_int, ctypes.POINTER(ctypes.c_double)]
    lib.fglt_stream_cancel.argtypes = [h_t, ctypes.c_uint64]
    for name in EXPORTED:
        if name not in ("fglt_status_string", "fglt_last_cuda_error"):
            getattr(lib, name).restype = c_int
    _lib = lib
    return lib


def build() -> str:
    """Compile libfglt.so for sm_103a (in-tree) and return its path."""
    return _build.build()


def status_string(status: int) -> str:
    try:
        return load(build_if_missing=False).fglt_status_string(status).decode()
    except Exception:
        return f"status {status}"


def _check(status: int, what: str, h=None):
    if status != FGLT_OK:
        extra = ""
        if h is not None and status == FGLT_ERR_CUDA:
            extra = " [" + load().fglt_last_cuda_error(h).decode() + "]"
        raise FgltError(status, what + extra)


def _ptr(x) -> Optional[int]:
    """Device/host address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot take the address of {type(x)}")


CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy: the legacy default stream as an explicit handle


def _stream_ptr(stream) -> Optional[int]:
    """None -> NULL (the library uses the handle's own stream); a torch.cuda.Stream
    -> its handle, where torch's default stream (handle 0, the legacy default
    stream) is passed as cudaStreamLegacy so that the library orders its work
    after the caller's instead of taking NULL as "the handle's stream"."""
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    s = stream.cuda_stream  # torch.cuda.Stream
    return s if s != 0 else CUDA_STREAM_LEGACY


def _torch_stream(stream, tensor):
    """The stream a Handle method runs on: the caller's, else torch's current
    stream on the tensor's device (so that work queued there on the inputs
    comes first)."""
    if stream is not None:
        return stream
    import torch
    return torch.cuda.current_stream(tensor.device)


# ---------------------------------------------------------------------------
# C-ABI mirror
# ---------------------------------------------------------------------------

def fglt_options_default() -> fglt_options:
    opt = fglt_options()
    _check(load().fglt_options_default(ctypes.byref(opt)), "fglt_options_default")
    return opt


def fglt_create(opt: Optional[fglt_options] = None, device: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load().fglt_create(ctypes.byref(h), ctypes.byref(opt) if opt is not None else None, device),
           "fglt_create")
    return h.value


def fglt_destroy(h: int) -> None:
    _check(load().fglt_destroy(h), "fglt_destroy")


def fglt_transform(h, rowptr, rowptr_is_64bit: int, colidx, n: int, out_raw, out_net, stream=None) -> None:
    _check(load().fglt_transform(h, _ptr(rowptr), int(rowptr_is_64bit), _ptr(colidx), int(n), _ptr(out_raw),
                                 _ptr(out_net), _stream_ptr(stream)), "fglt_transform", h)


def fglt_transform_host(h, rowptr, rowptr_is_64bit: int, colidx, n: int, out_raw, out_net) -> None:
    _check(load().fglt_transform_host(h, _ptr(rowptr), int(rowptr_is_64bit), _ptr(colidx), int(n),
                                      _ptr(out_raw), _ptr(out_net)), "fglt_transform_host", h)


def fglt_transform_batched(h, rowptr, rowptr_is_64bit: int, colidx, graph_offsets: np.ndarray,
                           num_graphs: int, out_raw, out_net, stream=None) -> None:
    off = np.ascontiguousarray(graph_offsets, dtype=np.int64)
    _check(load().fglt_transform_batched(h, _ptr(rowptr), int(rowptr_is_64bit), _ptr(colidx),
                                         off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), int(num_graphs),
                                         _ptr(out_raw), _ptr(out_net), _stream_ptr(stream)),
           "fglt_transform_batched", h)


def fglt_transform_noalloc(rowptr, rowptr_is_64bit: int, colidx, n: int, out_raw, out_net, stream=None) -> None:
    """Transform without any device allocation (no handle). For callers that
    cannot allocate at call time; limited to small graphs (see include/fglt.h)."""
    _check(load().fglt_transform_noalloc(_ptr(rowptr), int(rowptr_is_64bit), _ptr(colidx), int(n), _ptr(out_raw),
                                         _ptr(out_net), _stream_ptr(stream)), "fglt_transform_noalloc")


def fglt_autotune(h, rowptr, rowptr_is_64bit: int, colidx, n: int, reps: int = 1, stream=None):
    """Runs the autotuner on one graph (device buffers) and installs the result
    on the handle. Returns (chosen fglt_options, tuned_ms, default_ms)."""
    opt = fglt_options()
    tuned = ctypes.c_float()
    default = ctypes.c_float()
    _check(load().fglt_autotune(h, _ptr(rowptr), int(rowptr_is_64bit), _ptr(colidx), int(n), int(reps),
                                _stream_ptr(stream), ctypes.byref(opt), ctypes.byref(tuned), ctypes.byref(default)),
           "fglt_autotune", h)
    return opt, tuned.value, default.value


def fglt_csr_from_edges(h, src, dst, num_edges: int, n: int, out_rowptr, out_colidx, stream=None) -> int:
    """Edge list -> sorted symmetric simple CSR (device buffers); returns nnz."""
    nnz = ctypes.c_int64()
    _check(load().fglt_csr_from_edges(h, _ptr(src), _ptr(dst), int(num_edges), int(n), _ptr(out_rowptr),
                                      _ptr(out_colidx), ctypes.byref(nnz), _stream_ptr(stream)),
           "fglt_csr_from_edges", h)
    return nnz.value


def fglt_csr_relabel_by_degree(h, rowptr, rowptr_is_64bit: int, colidx, n: int, descending: int, out_rowptr,
                               out_colidx, out_perm, stream=None) -> None:
    """Degree-ordered relabelling of a CSR (device buffers); perm[old] = new."""
    _check(load().fglt_csr_relabel_by_degree(h, _ptr(rowptr), int(rowptr_is_64bit), _ptr(colidx), int(n),
                                             int(descending), _ptr(out_rowptr), _ptr(out_colidx), _ptr(out_perm),
                                             _stream_ptr(stream)),
           "fglt_csr_relabel_by_degree", h)


def fglt_stage_times(h) -> dict:
    names = (ctypes.c_char_p * 32)()
    ms = (ctypes.c_float * 32)()
    cnt = ctypes.c_int()
    st = load().fglt_stage_times(h, names, ms, 32, ctypes.byref(cnt))
    if st == FGLT_ERR_NOT_FOUND:
        return {}
    _check(st, "fglt_stage_times")
    return {names[i].decode(): float(ms[i]) for i in range(min(cnt.value, 32))}


CYC_CLASSES = ["warp", "hash11", "hash12", "hash13", "dense", "dense_spill", "global"]
WORK_COUNTER_NAMES = (["n", "nnz", "m", "max_degree", "max_out_degree", "tri_scanned", "triangles",
                       "k4", "wedges", "max_wedges", "launches"] + [f"cls_vertices.{c}" for c in CYC_CLASSES]
                      + [f"cls_wedges.{c}" for c in CYC_CLASSES])


def fglt_work_counters(h) -> dict:
    vals = (ctypes.c_int64 * 32)()
    cnt = ctypes.c_int()
    st = load().fglt_work_counters(h, vals, 32, ctypes.byref(cnt))
    if st == FGLT_ERR_NOT_FOUND:
        return {}
    _check(st, "fglt_work_counters")
    return {WORK_COUNTER_NAMES[i]: int(vals[i]) for i in range(min(cnt.value, len(WORK_COUNTER_NAMES)))}


def fglt_stream_submit(h, n: int, rowptr: np.ndarray, colidx: np.ndarray, out_raw: Optional[np.ndarray],
                       out_net: Optional[np.ndarray]) -> int:
    g = fglt_graph_host()
    g.n = int(n)
    g.rowptr = rowptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    g.colidx = colidx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    g.out_raw = out_raw.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)) if out_raw is not None else None
    g.out_net = out_net.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)) if out_net is not None else None
    rid = ctypes.c_uint64()
    _check(load().fglt_stream_submit(h, ctypes.byref(g), ctypes.byref(rid)), "fglt_stream_submit", h)
    return rid.value


def fglt_stream_poll(h, request_id: int, timeout_ms: int):
    """Returns (status, latency_us). The status is the request's own result
    (FGLT_OK, or the error its transform returned) or FGLT_ERR_PENDING /
    FGLT_ERR_TIMEOUT / FGLT_ERR_NOT_FOUND; it is returned, not raised."""
    lat = ctypes.c_double()
    st = load().fglt_stream_poll(h, ctypes.c_uint64(request_id), int(timeout_ms), ctypes.byref(lat))
    return st, lat.value


def fglt_stream_cancel(h, request_id: int) -> int:
    return load().fglt_stream_cancel(h, ctypes.c_uint64(request_id))


# ---------------------------------------------------------------------------
# Convenience wrapper (still marshalling only)
# ---------------------------------------------------------------------------

class Handle:
    """Owns one fglt_t."""

    def __init__(self, device: int = 0, validate: bool = False, profile_stages: bool = False,
                 serve_memory_budget: int = 0, serve_max_batch: int = 0, serve_max_queue: int = 0,
                 cyc_hub_span: int = 0, tri_class_bounds=(0, 0), cyc_warp_bits: int = 0,
                 cyc_mid_threads=(0, 0, 0), cyc_heavy_threads: int = 0, dictionary: int = 0,
                 tri_probe_loads: int = 0, tri_hash_factor: int = 0, cyc_dense_min: int = 0,
                 tri_group_lanes: int = 0, cyc_long_segment: int = 0, tri_warp_max: int = 0,
                 cyc_spill_bits: int = 0, batch_small_max: int = 0, tri_pass2_from: int = 0,
                 device_wait_limit_ns: int = 0):
        """dictionary: sub-dictionary bit mask (0 = Sigma16; DICT_SIGMA5 = Sigma5)."""
        opt = fglt_options_default()
        opt.dictionary_mask = int(dictionary)
        self.cols = dictionary_columns(int(dictionary))
        opt.cyc_hub_span = int(cyc_hub_span)
        opt.tri_class_bounds[0], opt.tri_class_bounds[1] = (int(x) for x in tri_class_bounds)
        opt.cyc_warp_bits = int(cyc_warp_bits)
        for i, x in enumerate(cyc_mid_threads):
            opt.cyc_mid_threads[i] = int(x)
        opt.cyc_heavy_threads = int(cyc_heavy_threads)
        opt.tri_probe_loads = int(tri_probe_loads)
        opt.tri_hash_factor = int(tri_hash_factor)
        opt.cyc_dense_min = int(cyc_dense_min)
        opt.tri_group_lanes = int(tri_group_lanes)
        opt.cyc_long_segment = int(cyc_long_segment)
        opt.tri_warp_max = int(tri_warp_max)
        opt.cyc_spill_bits = int(cyc_spill_bits)
        opt.batch_small_max = int(batch_small_max)
        opt.tri_pass2_from = int(tri_pass2_from)
        opt.device_wait_limit_ns = int(device_wait_limit_ns)
        opt.validate = int(validate)
        opt.profile_stages = int(profile_stages)
        opt.serve_memory_budget = int(serve_memory_budget)
        opt.serve_max_batch = int(serve_max_batch)
        opt.serve_max_queue = int(serve_max_queue)
        self.h = fglt_create(opt, device)

    def close(self):
        if self.h:
            fglt_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def transform(self, rowptr, colidx, n: int, out_raw=None, out_net=None, stream=None):
        """Device transform; rowptr/colidx/out_* are torch CUDA tensors."""
        import torch
        if out_raw is None:
            out_raw = torch.empty((n, self.cols), dtype=torch.int64, device=rowptr.device)
        if out_net is None:
            out_net = torch.empty((n, self.cols), dtype=torch.int64, device=rowptr.device)
        rp64 = 1 if rowptr.dtype == torch.int64 else 0
        fglt_transform(self.h, rowptr, rp64, colidx, n, out_raw, out_net, _torch_stream(stream, rowptr))
        return out_raw, out_net

    def transform_host(self, rowptr: np.ndarray, colidx: np.ndarray, n: int):
        raw = np.empty((n, self.cols), dtype=np.int64)
        net = np.empty((n, self.cols), dtype=np.int64)
        rp = np.ascontiguousarray(rowptr)
        rp64 = 1 if rp.dtype == np.int64 else 0
        ci = np.ascontiguousarray(colidx, dtype=np.int32)
        if ci.size == 0:
            ci = np.zeros(1, np.int32)
        fglt_transform_host(self.h, rp, rp64, ci, n, raw, net)
        return raw, net

    def transform_batched(self, rowptr, colidx, graph_offsets, out_raw=None, out_net=None, stream=None):
        import torch
        off = np.ascontiguousarray(graph_offsets, dtype=np.int64)
        n = int(off[-1])
        if out_raw is None:
            out_raw = torch.empty((n, self.cols), dtype=torch.int64, device=rowptr.device)
        if out_net is None:
            out_net = torch.empty((n, self.cols), dtype=torch.int64, device=rowptr.device)
        rp64 = 1 if rowptr.dtype == torch.int64 else 0
        fglt_transform_batched(self.h, rowptr, rp64, colidx, off, len(off) - 1, out_raw, out_net,
                               _torch_stream(stream, rowptr))
        return out_raw, out_net

    def csr_from_edges(self, src, dst, n: int, stream=None):
        """Edge list (torch CUDA int32 tensors) -> (rowptr int64[n+1], colidx
        int32[nnz]) on the same device: symmetric, sorted, no self-loops or
        repeats."""
        import torch
        rowptr = torch.empty(n + 1, dtype=torch.int64, device=src.device)
        colidx = torch.empty(max(2 * src.numel(), 1), dtype=torch.int32, device=src.device)
        nnz = fglt_csr_from_edges(self.h, src, dst, src.numel(), n, rowptr, colidx, _torch_stream(stream, src))
        return rowptr, colidx[:nnz]

    def relabel_by_degree(self, rowptr, colidx, n: int, descending: bool = True, stream=None):
        """Degree-ordered relabelling (torch CUDA tensors) -> (rowptr int64[n+1],
        colidx int32[nnz], perm int32[n]) with perm[old id] = new id: new ids
        follow non-increasing (descending) or non-decreasing degree."""
        import torch
        rp64 = 1 if rowptr.dtype == torch.int64 else 0
        nnz = int(rowptr[n].item()) if n > 0 else 0
        out_rp = torch.empty(n + 1, dtype=torch.int64, device=rowptr.device)
        out_ci = torch.empty(max(nnz, 1), dtype=torch.int32, device=rowptr.device)
        perm = torch.empty(max(n, 1), dtype=torch.int32, device=rowptr.device)
        fglt_csr_relabel_by_degree(self.h, rowptr, rp64, colidx, n, 1 if descending else 0, out_rp, out_ci, perm,
                                   _torch_stream(stream, rowptr))
        return out_rp, out_ci[:nnz], perm[:n]

    def autotune(self, rowptr, colidx, n: int, reps: int = 1, stream=None):
        """Autotunes on this graph (torch CUDA tensors); returns (tuning dict,
        tuned ms, default ms). Later calls on this handle use the result."""
        import torch
        rp64 = 1 if rowptr.dtype == torch.int64 else 0
        opt, tuned, default = fglt_autotune(self.h, rowptr, rp64, colidx, n, reps, _torch_stream(stream, rowptr))
        return opt.tuning(), tuned, default

    def stage_times(self) -> dict:
        return fglt_stage_times(self.h)

    def work_counters(self) -> dict:
        return fglt_work_counters(self.h)
