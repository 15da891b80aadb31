"""Python binding of the GB300 single-source SimRank library (``libsrk.so``).

A thin ctypes layer over the C ABI declared in ``include/srk.h``: it only
marshals arguments (array pointers, sizes, the CUDA stream) and turns negative
return codes into ``SrkError``.  Every step of a query runs in the library's
CUDA kernels; there is no CPU fallback.  Importing this package loads
``libsrk.so`` and fails loudly (``ImportError``) when it has not been built
(``python -m paper_2304_04015_gb300.build``).

Arrays may be torch tensors (CUDA or CPU) or numpy arrays.  Device tensors are
passed as device pointers; host arrays as host pointers (the library then
copies results back and synchronises the stream before returning).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

__all__ = [
    "SrkError", "SrkOpts", "SrkStats", "Graph",
    "srk_graph_load", "srk_graph_free", "srk_graph_info", "srk_graph_layout", "srk_single_source",
    "srk_multi_source", "srk_multi_source_topk", "srk_single_source_noalloc", "srk_probe_gather",
    "srk_probe_gather_ex", "SRK_PROBE_DEFAULT", "SRK_PROBE_CG", "SRK_PROBE_NC", "SRK_PROBE_CA",
    "srk_linear_fwd", "srk_linear_bwd", "srk_linear_ctx_free", "LinearContext",
    "LinearSimRank", "linear_simrank", "SrkServerReport", "Server",
    "srk_server_create", "srk_server_submit", "srk_server_drain", "srk_server_stats",
    "srk_server_destroy", "srk_last_error", "srk_pool_stats",
    "library_path", "SRK_NOALLOC_SCRATCH_BYTES",
    "SRK_OK", "SRK_EINVAL", "SRK_ENOMEM", "SRK_ECUDA", "SRK_ETIMEOUT",
    "SRK_ENOTSUP", "SRK_DEVICE_PTRS", "SRK_VALIDATE", "SRK_ADJ_NARROW", "SRK_ADJ_WIDE", "SRK_OPT_NO_GRAPH", "SRK_OPT_WARMUP_RULE", "SRK_OPT_LITERAL_SHUFFLE", "SRK_OPT_SHARED_WALKS", "SRK_MAX_LEN",
    "SRK_MAX_WALKS",
]

SRK_OK, SRK_EINVAL, SRK_ENOMEM, SRK_ECUDA, SRK_ETIMEOUT, SRK_ENOTSUP = 0, -1, -2, -3, -4, -5
SRK_DEVICE_PTRS, SRK_VALIDATE, SRK_ADJ_NARROW, SRK_ADJ_WIDE, SRK_ADJ_CSR = 1, 2, 4, 8, 16
SRK_OPT_NO_GRAPH, SRK_OPT_WARMUP_RULE, SRK_OPT_LITERAL_SHUFFLE, SRK_OPT_SHARED_WALKS = 1, 2, 4, 8
SRK_PROBE_DEFAULT, SRK_PROBE_CG, SRK_PROBE_NC, SRK_PROBE_CA = 0, 1, 2, 3
SRK_MAX_LEN, SRK_MAX_WALKS = 255, 1 << 24
SRK_NOALLOC_SCRATCH_BYTES = 16 << 20

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "libsrk.so")

if not os.path.exists(library_path):
    raise ImportError(
        "libsrk.so is not built; run `python paper_2304_04015_gb300/build.py` "
        "or __graft_entry__.build() (needs nvcc).  There is no CPU fallback.")
_lib = ctypes.CDLL(library_path)


class SrkError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__("srk error %d: %s" % (code, message))
        self.code = code


class SrkStats(ctypes.Structure):
    _fields_ = [("z", ctypes.c_double), ("L", ctypes.c_int32),
                ("n_walks", ctypes.c_int32), ("n_active_pairs", ctypes.c_int32),
                ("batch_shape", ctypes.c_int32), ("source_steps", ctypes.c_uint64),
                ("target_steps", ctypes.c_uint64), ("graph_updates", ctypes.c_int64)]


class SrkOpts(ctypes.Structure):
    _fields_ = [("z_override", ctypes.c_double), ("L_override", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("p", ctypes.c_double),
                ("q", ctypes.c_double), ("step_counts", ctypes.c_void_p),
                ("stats", ctypes.POINTER(SrkStats)), ("timing_events", ctypes.c_void_p),
                ("target_begin", ctypes.c_int32), ("target_end", ctypes.c_int32)]


_vp = ctypes.c_void_p
_lib.srk_graph_load.argtypes = [_vp, _vp, ctypes.c_int32, ctypes.c_int64,
                                ctypes.c_int, _vp, ctypes.POINTER(_vp)]
_lib.srk_graph_free.argtypes = [_vp]
_lib.srk_graph_info.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32),
                                ctypes.POINTER(ctypes.c_int64)]
_lib.srk_single_source.argtypes = [_vp, ctypes.c_int32, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_uint64,
                                   ctypes.POINTER(SrkOpts), _vp, _vp, _vp, _vp]
_lib.srk_single_source_noalloc.argtypes = _lib.srk_single_source.argtypes
_lib.srk_multi_source.argtypes = [_vp, _vp, ctypes.c_int32, ctypes.c_double,
                                  _vp, ctypes.c_uint64, ctypes.POINTER(SrkOpts),
                                  _vp, _vp, _vp]
_lib.srk_graph_layout.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32)]
_lib.srk_probe_gather.argtypes = [_vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint32,
                                  _vp, ctypes.POINTER(ctypes.c_int64), _vp]
_lib.srk_probe_gather_ex.argtypes = [_vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint32,
                                     ctypes.c_int32, _vp, ctypes.POINTER(ctypes.c_int64), _vp]
_lib.srk_linear_fwd.argtypes = [_vp, _vp, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                _vp, ctypes.POINTER(_vp), _vp]
_lib.srk_linear_bwd.argtypes = [_vp, _vp, _vp, _vp]
_lib.srk_linear_ctx_free.argtypes = [_vp]


class SrkServerReport(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64),
                ("shed", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("target_steps", ctypes.c_uint64),
                ("reserved_peak", ctypes.c_uint64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("wall_s", ctypes.c_double),
                ("queries_per_s", ctypes.c_double)]


_lib.srk_server_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int32, ctypes.c_uint64,
                                   ctypes.c_int32, ctypes.c_double, ctypes.POINTER(_vp)]
_lib.srk_server_submit.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_uint64, _vp, ctypes.c_uint64,
                                   ctypes.POINTER(ctypes.c_int32)]
_lib.srk_server_drain.argtypes = [_vp]
_lib.srk_server_stats.argtypes = [_vp, ctypes.POINTER(SrkServerReport)]
_lib.srk_server_destroy.argtypes = [_vp]
_lib.srk_pool_stats.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_uint64),
                                ctypes.POINTER(ctypes.c_uint64),
                                ctypes.POINTER(ctypes.c_uint64), ctypes.c_int]
_lib.srk_last_error.restype = ctypes.c_char_p
_lib.srk_multi_source_topk.argtypes = [_vp, _vp, ctypes.c_int32, ctypes.c_double, _vp,
                                       ctypes.c_uint64, _vp, ctypes.c_int32, _vp, _vp, _vp,
                                       _vp, _vp]
for _f in ("srk_pool_stats", "srk_multi_source_topk", "srk_graph_load", "srk_graph_free", "srk_graph_info", "srk_graph_layout",
           "srk_single_source", "srk_single_source_noalloc", "srk_multi_source",
           "srk_probe_gather", "srk_probe_gather_ex", "srk_linear_fwd", "srk_linear_bwd", "srk_linear_ctx_free",
           "srk_server_create", "srk_server_submit", "srk_server_drain", "srk_server_stats",
           "srk_server_destroy"):
    getattr(_lib, _f).restype = ctypes.c_int


def srk_last_error() -> str:
    return (_lib.srk_last_error() or b"").decode(errors="replace")


def _check(rc: int) -> None:
    if rc != SRK_OK:
        raise SrkError(rc, srk_last_error())


# unsigned outputs may also be given as signed tensors of the same width
_SAME_WIDTH = {"uint32": ("uint32", "int32"), "uint64": ("uint64", "int64")}


def _ptr(a, dtype=None):
    """(pointer, is_device, keepalive) of a torch tensor or numpy array."""
    if a is None:
        return None, False, None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if dtype is not None and str(a.dtype)[6:] not in _SAME_WIDTH.get(dtype, (dtype,)):
                raise TypeError("expected a %s tensor, got %s" % (dtype, a.dtype))
            if not a.is_contiguous():
                raise ValueError("tensor must be contiguous")
            return a.data_ptr(), a.is_cuda, a
    except ImportError:  # pragma: no cover
        pass
    arr = np.asarray(a)
    if dtype is not None and arr.dtype != np.dtype(dtype):
        raise TypeError("expected a %s array, got %s" % (dtype, arr.dtype))
    if not arr.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return arr.ctypes.data, False, arr


def _stream_handle(stream) -> int:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:  # pragma: no cover
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Graph:
    """Handle of a resident graph (``srk_graph*``); frees itself when closed."""

    def __init__(self, handle: int, n: int, m: int, keep):
        self.handle = handle
        self.n = n
        self.m = m
        self._keep = keep

    def close(self) -> None:
        if self.handle:
            h, self.handle = self.handle, 0
            _check(_lib.srk_graph_free(h))
            self._keep = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def srk_graph_load(row_ptr, col, n: Optional[int] = None, m: Optional[int] = None,
                   flags: Optional[int] = None, edge_w=None,
                   layout: Optional[str] = None) -> Graph:
    """Load an in-neighbour CSR (see ``include/srk.h``).  Device tensors are
    borrowed (SRK_DEVICE_PTRS); host arrays are copied to the current device.
    ``layout``: None (chosen by size), "narrow" or "wide" adjacency entries."""
    rp, rp_dev, k1 = _ptr(row_ptr, "int32")
    cl, cl_dev, k2 = _ptr(col, "int32")
    ew, ew_dev, k3 = _ptr(edge_w, "float32")
    if n is None:
        n = (row_ptr.numel() if hasattr(row_ptr, "numel") else np.asarray(row_ptr).size) - 1
    if m is None:
        m = col.numel() if hasattr(col, "numel") else np.asarray(col).size
    if flags is None:
        flags = SRK_DEVICE_PTRS if rp_dev else 0
    if layout is not None:
        flags |= {"narrow": SRK_ADJ_NARROW, "wide": SRK_ADJ_WIDE, "csr": SRK_ADJ_CSR}[layout]
    if rp_dev != cl_dev or (edge_w is not None and ew_dev != rp_dev):
        raise ValueError("row_ptr, col and edge_w must all be on the device or all on the host")
    h = _vp()
    _check(_lib.srk_graph_load(rp, cl, int(n), int(m), int(flags), ew, ctypes.byref(h)))
    keep = (k1, k2, k3) if flags & SRK_DEVICE_PTRS else None
    return Graph(h.value, int(n), int(m), keep)


def srk_graph_free(g: Graph) -> None:
    g.close()


def srk_graph_layout(g: Graph) -> str:
    """The adjacency layout the walks read: "narrow", "wide" or "csr"."""
    v = ctypes.c_int32()
    _check(_lib.srk_graph_layout(g.handle, ctypes.byref(v)))
    return {SRK_ADJ_NARROW: "narrow", SRK_ADJ_WIDE: "wide", SRK_ADJ_CSR: "csr"}[v.value]


def srk_graph_info(g: Graph):
    n = ctypes.c_int32()
    m = ctypes.c_int64()
    _check(_lib.srk_graph_info(g.handle, ctypes.byref(n), ctypes.byref(m)))
    return n.value, m.value


def _opts(z_override=None, L_override=None, p=None, q=None, step_counts=None,
          stats: Optional[SrkStats] = None, timing_events=None, flags: int = 0,
          target_range=None, warmup_rule: bool = False, literal_shuffle: bool = False,
          shared_walks: bool = False):
    o = SrkOpts()
    if literal_shuffle:
        flags |= SRK_OPT_LITERAL_SHUFFLE
    if shared_walks:
        flags |= SRK_OPT_SHARED_WALKS
    if target_range is not None:
        o.target_begin, o.target_end = int(target_range[0]), int(target_range[1])
    if warmup_rule:
        flags |= SRK_OPT_WARMUP_RULE
    o.z_override = float(z_override) if z_override else 0.0
    o.L_override = int(L_override) if L_override is not None else -1
    o.flags = int(flags)
    o.p = float(p) if p else 0.0
    o.q = float(q) if q else 0.0
    sp, _, keep = _ptr(step_counts, "uint32")
    o.step_counts = sp
    o.stats = ctypes.pointer(stats) if stats is not None else None
    ev_keep = None
    if timing_events is not None:
        # two torch.cuda.Event objects (or raw cudaEvent_t handles)
        handles = [e.cuda_event if hasattr(e, "cuda_event") else int(e) for e in timing_events]
        ev_keep = (ctypes.c_void_p * 2)(*handles)
        o.timing_events = ctypes.cast(ev_keep, ctypes.c_void_p).value
    return o, (keep, ev_keep)


def srk_single_source(g: Graph, s: int, c: float, eps: float, seed: int,
                      scores, meet_counts=None, weight_sums=None, *,
                      z_override=None, L_override=None, p=None, q=None,
                      step_counts=None, stats: Optional[SrkStats] = None,
                      timing_events=None, target_range=None, warmup_rule: bool = False,
                      literal_shuffle: bool = False, shared_walks: bool = False,
                      stream=None) -> None:
    """One query (``srk_single_source``): fills ``scores`` (n float64) and,
    when given, ``meet_counts`` (n uint32), ``weight_sums`` (n uint64),
    ``step_counts`` (n uint32) and ``stats``.  ``timing_events``: two
    ``torch.cuda.Event(enable_timing=True)`` recorded around the target-walk
    kernel on the query's stream."""
    sc, _, k1 = _ptr(scores, "float64")
    mc, _, k2 = _ptr(meet_counts, "uint32")
    ws, _, k3 = _ptr(weight_sums, "uint64")
    o, k4 = _opts(z_override, L_override, p, q, step_counts, stats, timing_events,
                  target_range=target_range, warmup_rule=warmup_rule,
                  literal_shuffle=literal_shuffle, shared_walks=shared_walks)
    rc = _lib.srk_single_source(g.handle, int(s), float(c), float(eps),
                                int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.byref(o),
                                sc, mc, ws, _stream_handle(stream))
    del k1, k2, k3, k4
    _check(rc)


def srk_single_source_noalloc(g: Graph, s: int, c: float, eps: float, seed: int,
                              scores, meet_counts=None, weight_sums=None, *,
                              z_override=None, L_override=None, p=None, q=None,
                              step_counts=None, stats: Optional[SrkStats] = None,
                              timing_events=None, target_range=None,
                              warmup_rule: bool = False, literal_shuffle: bool = False,
                              shared_walks: bool = False, stream=None) -> None:
    """``srk_single_source`` for callers that must not allocate device memory
    while querying: the scratch is a static device array of
    ``SRK_NOALLOC_SCRATCH_BYTES``; outputs must be device tensors; calls that
    overlap on the GPU race on the shared scratch."""
    sc, _, k1 = _ptr(scores, "float64")
    mc, _, k2 = _ptr(meet_counts, "uint32")
    ws, _, k3 = _ptr(weight_sums, "uint64")
    o, k4 = _opts(z_override, L_override, p, q, step_counts, stats, timing_events,
                  target_range=target_range, warmup_rule=warmup_rule,
                  literal_shuffle=literal_shuffle, shared_walks=shared_walks)
    rc = _lib.srk_single_source_noalloc(g.handle, int(s), float(c), float(eps),
                                        int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.byref(o),
                                        sc, mc, ws, _stream_handle(stream))
    del k1, k2, k3, k4
    _check(rc)


def srk_multi_source(g: Graph, sources, c: float, eps, seed: int, scores,
                     meet_counts=None, *, z_override=None, L_override=None,
                     p=None, q=None, stats: Optional[SrkStats] = None,
                     no_graph: bool = False, warmup_rule: bool = False,
                     literal_shuffle: bool = False, shared_walks: bool = False,
                     stream=None) -> None:
    """k queries (``srk_multi_source``): ``sources`` and ``eps`` are host
    sequences of length k; ``scores`` is k x n float64.  ``no_graph``: enqueue
    the batch launches directly instead of through a captured CUDA graph.
    ``shared_walks``: every target's walks are drawn once for all sources of
    a batch (``SRK_OPT_SHARED_WALKS``).  ``literal_shuffle`` is passed through
    and rejected by the library."""
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32))
    k = src.size
    eps_a = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, dtype=np.float64), (k,)))
    sc, _, k1 = _ptr(scores, "float64")
    mc, _, k2 = _ptr(meet_counts, "uint32")
    o, _ = _opts(z_override, L_override, p, q, None, stats,
                 flags=SRK_OPT_NO_GRAPH if no_graph else 0, warmup_rule=warmup_rule,
                 literal_shuffle=literal_shuffle, shared_walks=shared_walks)
    rc = _lib.srk_multi_source(g.handle, src.ctypes.data, k, float(c), eps_a.ctypes.data,
                               int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.byref(o), sc, mc,
                               _stream_handle(stream))
    del k1, k2
    _check(rc)


def srk_multi_source_topk(g: Graph, sources, c: float, eps, seed: int, top: int,
                          top_nodes, top_scores, top_count=None, nnz=None, *,
                          z_override=None, L_override=None, p=None, q=None,
                          stats: Optional[SrkStats] = None, no_graph: bool = False,
                          warmup_rule: bool = False, shared_walks: bool = False,
                          stream=None) -> None:
    """Per source, the ``top`` targets of largest score (``srk_multi_source_topk``):
    ``top_nodes`` (k x top int32), ``top_scores`` (k x top float64) and
    optionally ``top_count`` (k int32) and ``nnz`` (k int64), all device
    tensors."""
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32))
    k = src.size
    eps_a = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, dtype=np.float64), (k,)))
    tn, _, k1 = _ptr(top_nodes, "int32")
    ts, _, k2 = _ptr(top_scores, "float64")
    tc, _, k3 = _ptr(top_count, "int32")
    nz, _, k4 = _ptr(nnz, "int64")
    o, k5 = _opts(z_override, L_override, p, q, None, stats,
                  flags=SRK_OPT_NO_GRAPH if no_graph else 0, warmup_rule=warmup_rule,
                  shared_walks=shared_walks)
    rc = _lib.srk_multi_source_topk(g.handle, src.ctypes.data, k, float(c), eps_a.ctypes.data,
                                    int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.byref(o), int(top),
                                    tn, ts, tc, nz, _stream_handle(stream))
    del k1, k2, k3, k4, k5
    _check(rc)


def srk_probe_gather(data, iters: int, seed: int, sink, stream=None,
                     cache_op: int = 0) -> int:
    """Enqueue the random-gather probe over ``data`` (device int32 tensor);
    returns the number of 4-byte loads it issues.  ``sink``: device int64[1].
    ``cache_op``: one of SRK_PROBE_* (``srk_probe_gather_ex``)."""
    dp, d_dev, k1 = _ptr(data, "int32")
    sp, s_dev, k2 = _ptr(sink, "uint64")
    if not (d_dev and s_dev):
        raise ValueError("data and sink must be device tensors")
    n = data.numel()
    loads = ctypes.c_int64()
    rc = _lib.srk_probe_gather_ex(dp, int(n), int(iters), int(seed) & 0xFFFFFFFF,
                                  int(cache_op), sp, ctypes.byref(loads),
                                  _stream_handle(stream))
    del k1, k2
    _check(rc)
    return loads.value


class LinearContext:
    """Owns an ``srk_linear_ctx*`` (the state srk_linear_bwd needs)."""

    def __init__(self, handle: int, graph: "Graph", m: int):
        self.handle = handle
        self.graph = graph   # the context refers to the graph
        self.m = m

    def free(self) -> None:
        if self.handle:
            h, self.handle = self.handle, 0
            _check(_lib.srk_linear_ctx_free(h))

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def srk_pool_stats(device: int = 0, reset_high: bool = False):
    """(reserved, used, used_high) bytes of the library's memory pool on
    ``device`` (``srk_pool_stats``); ``reset_high`` resets the high-water
    mark to the current use after reading it."""
    r, u, h = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(_lib.srk_pool_stats(int(device), ctypes.byref(r), ctypes.byref(u), ctypes.byref(h),
                               1 if reset_high else 0))
    return r.value, u.value, h.value


def srk_probe_gather_ex(data, iters: int, seed: int, cache_op: int, sink, stream=None) -> int:
    """``srk_probe_gather`` with the loads' PTX cache operator ``cache_op``
    (SRK_PROBE_DEFAULT, _CG, _NC or _CA)."""
    return srk_probe_gather(data, iters, seed, sink, stream=stream, cache_op=cache_op)


def srk_linear_fwd(g: Graph, edge_w, s: int, c: float, L: int, s_out, *,
                   keep_context: bool = True, stream=None):
    """Truncated linearised single-source SimRank into ``s_out`` (device
    float32, n).  ``edge_w``: device float32 weights aligned with col, or None
    for the weights given at load.  Returns a LinearContext (or None)."""
    wp, _, k1 = _ptr(edge_w, "float32")
    op, _, k2 = _ptr(s_out, "float32")
    h = _vp()
    rc = _lib.srk_linear_fwd(g.handle, wp, int(s), float(c), int(L), op,
                             ctypes.byref(h) if keep_context else None,
                             _stream_handle(stream))
    del k1, k2
    _check(rc)
    return LinearContext(h.value, g, g.m) if keep_context else None


def srk_linear_bwd(ctx: LinearContext, grad_s, grad_w, stream=None) -> None:
    """dLoss/dw into ``grad_w`` (device float32, m) from ``grad_s`` (n)."""
    gp, _, k1 = _ptr(grad_s, "float32")
    wp, _, k2 = _ptr(grad_w, "float32")
    rc = _lib.srk_linear_bwd(ctx.handle, gp, wp, _stream_handle(stream))
    del k1, k2
    _check(rc)


def srk_linear_ctx_free(ctx: LinearContext) -> None:
    ctx.free()


def _make_linear_function():
    import torch

    class LinearSimRank(torch.autograd.Function):
        """s_vec = sum_t c^t (P^T)^t D P^t e_s as a differentiable function of
        the edge weights (forward: srk_linear_fwd; backward: srk_linear_bwd)."""

        @staticmethod
        def forward(ctx, edge_w, graph, s, c, L):
            out = torch.empty(graph.n, dtype=torch.float32, device=edge_w.device)
            ctx.lin = srk_linear_fwd(graph, edge_w.detach().contiguous(), s, c, L, out)
            return out

        @staticmethod
        def backward(ctx, grad_out):
            grad_w = torch.empty(ctx.lin.m, dtype=torch.float32, device=grad_out.device)
            srk_linear_bwd(ctx.lin, grad_out.contiguous().to(torch.float32), grad_w)
            torch.cuda.current_stream(grad_out.device).synchronize()
            ctx.lin.free()
            return grad_w, None, None, None, None

    return LinearSimRank


try:
    LinearSimRank = _make_linear_function()
except ImportError:  # pragma: no cover
    LinearSimRank = None


def linear_simrank(graph: Graph, edge_w, s: int, c: float = 0.6, L: int = 10):
    """Differentiable linearised single-source SimRank (torch tensors)."""
    return LinearSimRank.apply(edge_w, graph, s, c, L)


class Server:
    """A query server (``srk_server*``) over resident graphs."""

    def __init__(self, handle: int, graphs):
        self.handle = handle
        self.graphs = list(graphs)   # the server refers to them
        self._buffers = []

    def close(self) -> None:
        if self.handle:
            h, self.handle = self.handle, 0
            _check(_lib.srk_server_destroy(h))
            self._buffers = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def srk_server_create(graphs, mem_budget: int, n_workers: int = 4,
                      latency_target_ms: float = 0.0) -> Server:
    """A server over ``graphs``; ``latency_target_ms`` > 0 adds estimated-
    finish-time admission and shortest-estimated-work-first service."""
    arr = (_vp * len(graphs))(*[g.handle for g in graphs])
    h = _vp()
    _check(_lib.srk_server_create(arr, len(graphs), int(mem_budget), int(n_workers),
                                  float(latency_target_ms), ctypes.byref(h)))
    return Server(h.value, graphs)


def srk_server_submit(srv: Server, graph: int, s: int, c: float, eps: float, seed: int,
                      host_scores=None, tag: int = 0) -> bool:
    """Submit one query; returns whether it was admitted.  ``host_scores``
    (numpy float64, n) is kept alive by the server object until close()."""
    hp = None
    if host_scores is not None:
        hp, dev, keep = _ptr(host_scores, "float64")
        if dev:
            raise ValueError("host_scores must be host memory")
        srv._buffers.append(keep)
    adm = ctypes.c_int32()
    _check(_lib.srk_server_submit(srv.handle, int(graph), int(s), float(c), float(eps),
                                  int(seed) & 0xFFFFFFFFFFFFFFFF, hp, int(tag),
                                  ctypes.byref(adm)))
    return bool(adm.value)


def srk_server_drain(srv: Server) -> None:
    _check(_lib.srk_server_drain(srv.handle))


def srk_server_stats(srv: Server) -> "SrkServerReport":
    st = SrkServerReport()
    _check(_lib.srk_server_stats(srv.handle, ctypes.byref(st)))
    return st


def srk_server_destroy(srv: Server) -> None:
    srv.close()
