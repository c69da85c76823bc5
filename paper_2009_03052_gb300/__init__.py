"""Python binding of libmotif, the GB300 colour-coding motif library.

Argument marshalling only: every step of the computation runs in the CUDA
library declared by include/motif.h.  PyTorch supplies device memory (the
caching allocator, through the library's allocator callback) and streams.
There is no CPU fallback: without the compiled library, or without a CUDA
device, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build_ext

LIB_PATH = build_ext.LIB
_lock = threading.Lock()
_lib = None

MC_OK, MC_E_INVALID, MC_E_NOMEM, MC_E_OVERFLOW, MC_E_CUDA, MC_E_TIMEOUT, MC_E_UNSUPPORTED, \
    MC_E_INTERNAL = range(8)
MC_GRAPH_DEVICE_PTRS = 1
MC_GRAPH_TRUSTED = 2
MC_BUILD_ZERO_ROOT = 1
MC_BUILD_SKIP_ROUND = 2
MC_BUILD_SUCCINCT = 4
MC_BUILD_VARLEN = 8
MC_REQ_SAMPLE = 0
MC_REQ_ESTIMATE = 1
MC_EST_UNIFORM = 0
MC_EST_AGS = 1

EXPORTED = [
    "mc_load_graph", "mc_free_graph", "mc_graph_info", "mc_color", "mc_build_tables",
    "mc_free_tables", "mc_total", "mc_table_layout", "mc_read_table", "mc_sample",
    "mc_estimate_counts", "mc_num_shapes", "mc_num_unrooted", "mc_num_classes", "mc_shape_info",
    "mc_class_codes", "mc_sigma", "mc_last_error", "mc_profile_enable", "mc_profile_reset",
    "mc_profile_read", "mc_launch_count", "mc_estimate_uniform_noalloc", "mc_total_range",
    "mc_sample_range", "mc_build_tables_batch", "mc_server_create", "mc_server_submit",
    "mc_server_wait", "mc_server_free", "mc_star_total", "mc_sample_stars", "mc_rebuild_tables",
    "mc_tables_status", "mc_color_biased", "mc_table_nonzeros", "mc_skip_round_info",
    "mc_autotune", "mc_autotune_choice", "mc_autotune_set", "mc_table_bytes",
]


class MotifError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libmotif status {status}: {msg}")
        self.status = status


class MotifOverflow(MotifError):
    pass


class Allocator(C.Structure):
    _fields_ = [("alloc", C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)),
                ("free", C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)),
                ("ctx", C.c_void_p)]


class EstimateParams(C.Structure):
    _fields_ = [("mode", C.c_int), ("h", C.c_int), ("seed", C.c_uint64),
                ("first_index", C.c_uint64), ("samples", C.c_int64), ("cbar", C.c_int64),
                ("eps", C.c_double), ("delta", C.c_double), ("batch", C.c_int64),
                ("node_lo", C.c_int64), ("node_hi", C.c_int64), ("colour_bias_q32", C.c_uint32),
                ("star_samples", C.c_int64)]


class Request(C.Structure):
    _fields_ = [("kind", C.c_int), ("table", C.c_int), ("h", C.c_int), ("unrooted_shape", C.c_int32),
                ("node_lo", C.c_int64), ("node_hi", C.c_int64), ("seed", C.c_uint64),
                ("first_index", C.c_uint64), ("count", C.c_int64), ("est", EstimateParams)]


class EstimateStats(C.Structure):
    _fields_ = [("samples", C.c_int64), ("switches", C.c_int64), ("covered", C.c_int64),
                ("batches", C.c_int64), ("discarded", C.c_int64)]


def load(path: str | None = None):
    """Load libmotif; raises if it has not been built (see build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libmotif is not built ({p} missing); run "
                               "paper_2009_03052_gb300.build()")
        lib = C.CDLL(p)
        P, i64, u64, i32 = C.c_void_p, C.c_int64, C.c_uint64, C.c_int32
        lib.mc_load_graph.argtypes = [i64, i64, P, P, C.c_uint32, P, P, C.POINTER(P)]
        lib.mc_free_graph.argtypes = [P]
        lib.mc_free_graph.restype = None
        lib.mc_graph_info.argtypes = [P, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
        lib.mc_color.argtypes = [P, C.c_int, u64, P, P]
        lib.mc_build_tables.argtypes = [P, P, C.c_int, C.c_int, C.c_uint32, P, P, C.POINTER(P)]
        lib.mc_free_tables.argtypes = [P]
        lib.mc_free_tables.restype = None
        lib.mc_total.argtypes = [P, C.c_int, i32, P, P, P]
        lib.mc_total_range.argtypes = [P, C.c_int, i32, i64, i64, P, P, P]
        lib.mc_sample_range.argtypes = [P, C.c_int, i32, i64, i64, u64, u64, i64, P, P, P, P, P]
        lib.mc_build_tables_batch.argtypes = [C.c_int, P, P, C.c_int, C.c_int, C.c_uint32, P, P,
                                              C.POINTER(P), P]
        lib.mc_table_layout.argtypes = [P, C.c_int, C.c_int, C.POINTER(i64), C.POINTER(C.c_int)]
        lib.mc_read_table.argtypes = [P, C.c_int, C.c_int, P, C.c_size_t, C.c_int, P]
        lib.mc_sample.argtypes = [P, C.c_int, i32, u64, u64, i64, P, P, P, P, P]
        lib.mc_estimate_counts.argtypes = [P, C.POINTER(EstimateParams), P, P,
                                           C.POINTER(EstimateStats), P]
        for f in ("mc_num_shapes", "mc_num_unrooted", "mc_num_classes"):
            getattr(lib, f).argtypes = [C.c_int]
        lib.mc_shape_info.argtypes = [C.c_int, P, P, P, P, P]
        lib.mc_class_codes.argtypes = [C.c_int, P]
        lib.mc_sigma.argtypes = [C.c_int, P, P]
        lib.mc_last_error.restype = C.c_char_p
        lib.mc_profile_enable.argtypes = [C.c_int]
        lib.mc_profile_read.argtypes = [P, C.c_size_t, P, P, P, C.c_int, C.POINTER(C.c_int)]
        lib.mc_launch_count.restype = C.c_int64
        lib.mc_estimate_uniform_noalloc.argtypes = [P, C.c_int, u64, u64, i64, P, P, P]
        lib.mc_server_create.argtypes = [P, C.c_int, C.c_int, C.c_size_t, C.POINTER(P)]
        lib.mc_server_submit.argtypes = [P, C.POINTER(Request), C.POINTER(i64)]
        lib.mc_server_wait.argtypes = [P, i64, P, P, P, P, C.POINTER(C.c_double),
                                       C.POINTER(C.c_double)]
        lib.mc_server_free.argtypes = [P]
        lib.mc_server_free.restype = None
        lib.mc_star_total.argtypes = [P, C.c_int, P, P]
        lib.mc_rebuild_tables.argtypes = [P, P, P]
        lib.mc_color_biased.argtypes = [P, C.c_int, u64, C.c_uint32, P, P]
        lib.mc_table_nonzeros.argtypes = [P, C.c_int, C.c_int, C.POINTER(i64), P]
        lib.mc_skip_round_info.argtypes = [C.c_int, P, P, P, P, P, P]
        lib.mc_tables_status.argtypes = [P, P]
        lib.mc_sample_stars.argtypes = [P, C.c_int, u64, u64, i64, P, P, P, P]
        lib.mc_autotune.argtypes = [C.c_int, C.c_char_p]
        lib.mc_table_bytes.argtypes = [P, C.POINTER(i64), C.POINTER(i64)]
        lib.mc_autotune_choice.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, i64, i64, i64]
        lib.mc_autotune_set.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, i64, i64, i64, C.c_int]
        _lib = lib
        return lib


def build(force: bool = False) -> str:
    """Compile libmotif for sm_103a in-tree."""
    return build_ext.build(force=force)


def _check(st: int):
    if st != MC_OK:
        msg = (load().mc_last_error() or b"").decode()
        if st == MC_E_OVERFLOW:
            raise MotifOverflow(st, msg)
        raise MotifError(st, msg)


# ---------------------------------------------------------------------------
# torch plumbing: device memory and streams
# ---------------------------------------------------------------------------

def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libmotif needs a CUDA device")
    return torch


def _stream_ptr(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class TorchAllocator:
    """Allocator callbacks backed by torch's caching allocator."""

    def __init__(self):
        torch = _torch()
        self.device = torch.cuda.current_device()
        dev = self.device

        @C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
        def _alloc(nbytes, ctx, stream):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))
            except Exception:
                return None

        @C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
        def _free(ptr, nbytes, ctx, stream):
            torch.cuda.caching_allocator_delete(int(ptr))

        self._keep = (_alloc, _free)
        self.struct = Allocator(_alloc, _free, None)


_allocator = None


def torch_allocator() -> TorchAllocator:
    global _allocator
    if _allocator is None:
        _allocator = TorchAllocator()
    return _allocator


def _ptr(x) -> int:
    return int(x.data_ptr()) if hasattr(x, "data_ptr") else int(x.ctypes.data)


def _u128(a) -> int:
    return int(a[0]) | (int(a[1]) << 64)


# ---------------------------------------------------------------------------
# handles
# ---------------------------------------------------------------------------

class Graph:
    """mc_load_graph: a CSR graph copied to the device."""

    def __init__(self, row_ptr, col, trusted: bool = False, stream=None):
        lib = load()
        torch = _torch()
        on_dev = hasattr(row_ptr, "is_cuda") and row_ptr.is_cuda
        if not hasattr(row_ptr, "data_ptr"):  # numpy input; torch CPU tensors (e.g. pinned) pass as is
            row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
            col = np.ascontiguousarray(col, dtype=np.uint32)
        n = int(row_ptr.shape[0]) - 1
        nnz = int(col.shape[0])
        flags = (MC_GRAPH_DEVICE_PTRS if on_dev else 0) | (MC_GRAPH_TRUSTED if trusted else 0)
        self._alloc = torch_allocator()
        h = C.c_void_p()
        _check(lib.mc_load_graph(n, nnz, _ptr(row_ptr), _ptr(col) if nnz else None, flags,
                                 C.byref(self._alloc.struct), _stream_ptr(stream), C.byref(h)))
        self.handle = h
        self.n, self.nnz = n, nnz
        self.device = torch.cuda.current_device()

    @classmethod
    def from_csr(cls, g, **kw) -> "Graph":
        return cls(g.row_ptr, g.col, **kw)

    def star_total(self, h: int, stream=None) -> int:
        """mc_star_total: the number of h-stars, sum_v C(d_v, h-1)."""
        out = (C.c_uint64 * 2)()
        _check(load().mc_star_total(self.handle, h, out, _stream_ptr(stream)))
        return int(out[0]) | (int(out[1]) << 64)

    def sample_stars(self, h: int, seed: int, first_index: int, count: int, stream=None):
        """mc_sample_stars: uncoloured uniform h-stars, device tensors
        (nodes [count, h], centres, classes)."""
        torch = _torch()
        t_nodes = torch.empty((max(count, 1), h), dtype=torch.int32, device="cuda")
        t_cen = torch.empty(max(count, 1), dtype=torch.int32, device="cuda")
        t_cls = torch.empty(max(count, 1), dtype=torch.int32, device="cuda")
        _check(load().mc_sample_stars(self.handle, h, seed, first_index, count, _ptr(t_nodes),
                                      _ptr(t_cen), _ptr(t_cls), _stream_ptr(stream)))
        return t_nodes[:count], t_cen[:count], t_cls[:count]

    def info(self) -> tuple[int, int, int]:
        n, nnz, md = C.c_int64(), C.c_int64(), C.c_int64()
        _check(load().mc_graph_info(self.handle, C.byref(n), C.byref(nnz), C.byref(md)))
        return n.value, nnz.value, md.value

    def free(self):
        if getattr(self, "handle", None):
            load().mc_free_graph(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def color(graph: Graph, k: int, seed: int, out=None, stream=None, bias_q32: int = 0):
    """mc_color (or mc_color_biased with bias_q32 = lambda * 2^32 > 0):
    counter-based colouring, a device uint8 tensor."""
    torch = _torch()
    if out is None:
        out = torch.empty(max(graph.n, 1), dtype=torch.uint8, device="cuda")
    if bias_q32:
        _check(load().mc_color_biased(graph.handle, k, seed, bias_q32, _ptr(out), _stream_ptr(stream)))
    else:
        _check(load().mc_color(graph.handle, k, seed, _ptr(out), _stream_ptr(stream)))
    return out[: graph.n]


class Tables:
    """mc_build_tables: the exact colourful treelet count tables."""

    def __init__(self, graph: Graph, colors, k: int, count_bits: int = 64, stream=None,
                 zero_root: bool = False, own_memory: bool = False, skip_round: bool = False,
                 succinct: bool = False, varlen: bool = False, _handle=None):
        torch = _torch()
        if _handle is not None:  # built by batch()
            self.graph, self.k, self.bits, self._alloc, self.handle = graph, k, count_bits, \
                torch_allocator(), _handle
            return
        if not (hasattr(colors, "is_cuda") and colors.is_cuda):
            colors = torch.as_tensor(np.ascontiguousarray(colors, dtype=np.uint8)).cuda()
        self.graph, self.k, self.bits = graph, k, count_bits
        self._alloc = torch_allocator()
        h = C.c_void_p()
        # own_memory: the library allocates (stream-ordered scratch, no
        # callbacks into Python), e.g. for tables served from worker threads
        flags = (MC_BUILD_ZERO_ROOT if zero_root else 0) | (MC_BUILD_SKIP_ROUND if skip_round else 0) | \
            (MC_BUILD_SUCCINCT if succinct else 0) | (MC_BUILD_VARLEN if varlen else 0)
        _check(load().mc_build_tables(graph.handle, _ptr(colors) if graph.n else None, k,
                                      count_bits, flags,
                                      None if own_memory else C.byref(self._alloc.struct),
                                      _stream_ptr(stream), C.byref(h)))
        self.handle = h

    def table_bytes(self) -> tuple[int, int]:
        """mc_table_bytes: (dense bytes, stored bytes) of the c and S levels."""
        d, st = C.c_int64(), C.c_int64()
        _check(load().mc_table_bytes(self.handle, C.byref(d), C.byref(st)))
        return d.value, st.value

    def nonzeros(self, h: int, which: int = 0, stream=None) -> int:
        """mc_table_nonzeros: non-zero entries of level h (0: c, 1: S)."""
        out = C.c_int64()
        _check(load().mc_table_nonzeros(self.handle, h, which, C.byref(out), _stream_ptr(stream)))
        return out.value

    def rebuild(self, colors, stream=None):
        """mc_rebuild_tables: the whole build again for a new colouring (device
        uint8 tensor), in place, without allocating or synchronising -- it
        can be captured into a CUDA graph."""
        _check(load().mc_rebuild_tables(self.handle, _ptr(colors) if self.graph.n else None,
                                        _stream_ptr(stream)))

    def status(self, stream=None):
        """mc_tables_status: checks of the last rebuild (synchronises)."""
        _check(load().mc_tables_status(self.handle, _stream_ptr(stream)))

    @classmethod
    def batch(cls, graphs, colors, k: int, count_bits: int = 64, zero_root: bool = False,
              stream=None):
        """mc_build_tables_batch: one build over the disjoint union of the
        instances; returns (tables, node offsets) -- instance i owns union
        nodes [offsets[i], offsets[i+1])."""
        torch = _torch()
        cols = [c if (hasattr(c, "is_cuda") and c.is_cuda) else
                torch.as_tensor(np.ascontiguousarray(c, dtype=np.uint8)).cuda() for c in colors]
        gh = (C.c_void_p * len(graphs))(*[g.handle.value for g in graphs])
        ch = (C.c_void_p * len(cols))(*[_ptr(c) for c in cols])
        offs = np.zeros(len(graphs) + 1, np.int64)
        alloc = torch_allocator()
        h = C.c_void_p()
        _check(load().mc_build_tables_batch(len(graphs), gh, ch, k, count_bits,
                                            MC_BUILD_ZERO_ROOT if zero_root else 0,
                                            C.byref(alloc.struct), _stream_ptr(stream), C.byref(h),
                                            _ptr(offs)))

        class _Union:  # the union graph is owned by the tables
            n = int(offs[-1])
        return cls(_Union(), None, k, count_bits, _handle=h), offs

    def free(self):
        if getattr(self, "handle", None):
            load().mc_free_tables(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def total(self, h: int, unrooted: int = -1, node_range=(0, 0), stream=None) -> tuple[int, int]:
        """mc_total_range: (rooted total, number of colourful h-treelet
        copies), over the roots in node_range ((0, 0): all nodes)."""
        r = np.zeros(2, np.uint64)
        u = np.zeros(2, np.uint64)
        _check(load().mc_total_range(self.handle, h, unrooted, node_range[0], node_range[1],
                                     _ptr(r), _ptr(u), _stream_ptr(stream)))
        return _u128(r), _u128(u)

    def layout(self, h: int, which: int = 0) -> tuple[int, int]:
        w, b = C.c_int64(), C.c_int()
        _check(load().mc_table_layout(self.handle, h, which, C.byref(w), C.byref(b)))
        return w.value, b.value

    def read(self, h: int, which: int = 0, stream=None) -> np.ndarray:
        """mc_read_table into host memory: uint64 array [n, W, words] (words
        = 1 for 64-bit counts, 2 for 128-bit ones, low word first)."""
        W, b = self.layout(h, which)
        words = b // 8
        out = np.zeros(max(self.graph.n * W * words, 1), np.uint64)
        _check(load().mc_read_table(self.handle, h, which, _ptr(out), out.nbytes, 0,
                                    _stream_ptr(stream)))
        return out[: self.graph.n * W * words].reshape(self.graph.n, W, words)

    def sample(self, h: int, seed: int, first_index: int, count: int, unrooted: int = -1,
               nodes=True, roots=True, shapes=True, classes=True, node_range=(0, 0), stream=None):
        """mc_sample: device tensors (nodes [count, h], roots, shapes, classes)."""
        torch = _torch()
        dev = "cuda"
        t_nodes = torch.empty((max(count, 1), h), dtype=torch.int32, device=dev) if nodes else None
        t_roots = torch.empty(max(count, 1), dtype=torch.int32, device=dev) if roots else None
        t_shapes = torch.empty(max(count, 1), dtype=torch.int32, device=dev) if shapes else None
        t_cls = torch.empty(max(count, 1), dtype=torch.int32, device=dev) if classes else None
        p = lambda t: _ptr(t) if t is not None else None
        _check(load().mc_sample_range(self.handle, h, unrooted, node_range[0], node_range[1], seed,
                                      first_index, count, p(t_nodes), p(t_roots), p(t_shapes),
                                      p(t_cls), _stream_ptr(stream)))
        cut = lambda t: t[:count] if t is not None else None
        return cut(t_nodes), cut(t_roots), cut(t_shapes), cut(t_cls)

    def estimate(self, h: int, seed: int, samples: int, mode: int = MC_EST_UNIFORM,
                 first_index: int = 0, cbar: int = 0, eps: float = 0.0, delta: float = 0.0,
                 batch: int = 0, node_range=(0, 0), star_samples: int = 0, colour_bias_q32: int = 0,
                 stream=None):
        """mc_estimate_counts: (estimates, hits, stats dict)."""
        ncls = num_classes(h)
        est = np.zeros(ncls, np.float64)
        hits = np.zeros(ncls, np.uint64)
        prm = EstimateParams(mode, h, seed, first_index, samples, cbar, eps, delta, batch,
                             node_range[0], node_range[1], colour_bias_q32, star_samples)
        st = EstimateStats()
        _check(load().mc_estimate_counts(self.handle, C.byref(prm), _ptr(est), _ptr(hits),
                                         C.byref(st), _stream_ptr(stream)))
        return est, hits, {"samples": st.samples, "switches": st.switches,
                           "covered": st.covered, "batches": st.batches,
                           "discarded": st.discarded}

    def estimate_noalloc(self, h: int, seed: int, samples: int, first_index: int = 0,
                         stream=None):
        """mc_estimate_uniform_noalloc: the uniform estimate without any
        device allocation (for callers that cannot allocate); the graphlet
        catalogue of size h must exist (sigma(h) creates it)."""
        ncls = num_classes(h)
        est = np.zeros(ncls, np.float64)
        hits = np.zeros(ncls, np.uint64)
        _check(load().mc_estimate_uniform_noalloc(self.handle, h, seed, first_index, samples,
                                                  _ptr(est), _ptr(hits), _stream_ptr(stream)))
        return est, hits


# ---------------------------------------------------------------------------
# catalogue
# ---------------------------------------------------------------------------

def num_shapes(h: int) -> int:
    return int(load().mc_num_shapes(h))


def num_unrooted(h: int) -> int:
    return int(load().mc_num_unrooted(h))


def num_classes(h: int) -> int:
    n = int(load().mc_num_classes(h))
    if n < 0:
        _check(MC_E_INTERNAL)
    return n


def shape_info(h: int) -> dict:
    r = num_shapes(h)
    code = np.zeros(r, np.uint32)
    arrs = [np.zeros(r, np.int32) for _ in range(4)]
    _check(load().mc_shape_info(h, _ptr(code), *[_ptr(a) for a in arrs]))
    return {"code": code, "unrooted": arrs[0], "beta": arrs[1], "left": arrs[2],
            "right": arrs[3]}


def skip_round_info(k: int) -> dict:
    """mc_skip_round_info: the balanced level-k decompositions of round
    skipping and the rooted copies a_j per unrooted k-shape."""
    r, nu = num_shapes(k), num_unrooted(k)
    arrs = [np.zeros(r, np.int32) for _ in range(5)]
    copies = np.zeros(nu, np.int32)
    _check(load().mc_skip_round_info(k, *[_ptr(a) for a in arrs], _ptr(copies)))
    return {"beta": arrs[0], "left_size": arrs[1], "left": arrs[2], "right_size": arrs[3],
            "right": arrs[4], "copies": copies}


def class_codes(h: int) -> np.ndarray:
    out = np.zeros(num_classes(h), np.uint32)
    _check(load().mc_class_codes(h, _ptr(out)))
    return out


def sigma(h: int) -> tuple[np.ndarray, np.ndarray]:
    nc, nu = num_classes(h), num_unrooted(h)
    si = np.zeros(nc, np.int64)
    sij = np.zeros(nc * nu, np.int64)
    _check(load().mc_sigma(h, _ptr(si), _ptr(sij)))
    return si, sij.reshape(nc, nu)


# ---------------------------------------------------------------------------
# tracing
# ---------------------------------------------------------------------------

def profile_enable(on: bool = True, count_bytes: bool = False):
    """mc_profile_enable: time every launch; count_bytes also has the
    sampler count its bytes (items and 32-byte sectors)."""
    _check(load().mc_profile_enable((3 if count_bytes else 1) if on else 0))


def profile_reset():
    _check(load().mc_profile_reset())


def profile_read(with_bytes: bool = False) -> dict:
    """{kernel name: (total ms, launches[, bytes])} of the library's own
    kernels; bytes are the counted data bytes of kernels that count them."""
    maxk = 256
    names = C.create_string_buffer(maxk * 32)
    ms = np.zeros(maxk, np.float64)
    launches = np.zeros(maxk, np.int64)
    nbytes = np.zeros(maxk, np.int64)
    cnt = C.c_int()
    _check(load().mc_profile_read(names, len(names), _ptr(ms), _ptr(launches), _ptr(nbytes), maxk,
                                  C.byref(cnt)))
    out = {}
    parts = names.raw.split(b"\0")
    for i in range(cnt.value):
        v = (float(ms[i]), int(launches[i]))
        out[parts[i].decode()] = v + (int(nbytes[i]),) if with_bytes else v
    return out


def autotune(mode: int = 1, cache_file: str | None = None):
    """mc_autotune: 0 never tune, 1 tune new keys (default), 2 tune every key
    once more; cache_file: load choices from it and append new ones ("" stops
    appending)."""
    _check(load().mc_autotune(mode, cache_file.encode() if cache_file is not None else None))


def autotune_choice(kind: int, k: int, count_bits: int, h: int, n: int, nnz: int,
                    max_degree: int) -> int:
    """mc_autotune_choice: the schedule chosen for (kernel kind, k, width,
    level h) on graphs of this size and degree bucket (-1: not tuned yet)."""
    return int(load().mc_autotune_choice(kind, k, count_bits, h, n, nnz, max_degree))


def autotune_set(kind: int, k: int, count_bits: int, h: int, n: int, nnz: int,
                 max_degree: int, choice: int):
    """mc_autotune_set: fix the schedule of one key."""
    _check(load().mc_autotune_set(kind, k, count_bits, h, n, nnz, max_degree, choice))


def launch_count() -> int:
    return int(load().mc_launch_count())


# ---------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------

class Server:
    """mc_server_*: continuous batching of sample / estimate requests over
    device-resident tables (which must outlive the server)."""

    def __init__(self, tables: list, slots: int = 4, memory_budget: int = 0):
        self.tables = list(tables)
        arr = (C.c_void_p * len(tables))(*[t.handle.value for t in tables])
        h = C.c_void_p()
        _check(load().mc_server_create(arr, len(tables), slots, memory_budget, C.byref(h)))
        self.handle = h
        self._req = {}

    def submit_sample(self, table: int, h: int, seed: int, count: int, first_index: int = 0,
                      unrooted: int = -1, node_range=(0, 0)) -> int:
        r = Request(MC_REQ_SAMPLE, table, h, unrooted, node_range[0], node_range[1], seed,
                    first_index, count, EstimateParams())
        i = C.c_int64()
        _check(load().mc_server_submit(self.handle, C.byref(r), C.byref(i)))
        self._req[i.value] = ("sample", h, count)
        return i.value

    def submit_estimate(self, table: int, h: int, seed: int, samples: int,
                        mode: int = MC_EST_UNIFORM, first_index: int = 0, cbar: int = 0,
                        eps: float = 0.0, delta: float = 0.0, batch: int = 0,
                        node_range=(0, 0), star_samples: int = 0, colour_bias_q32: int = 0) -> int:
        e = EstimateParams(mode, h, seed, first_index, samples, cbar, eps, delta, batch,
                           node_range[0], node_range[1], colour_bias_q32, star_samples)
        r = Request(MC_REQ_ESTIMATE, table, 0, -1, 0, 0, 0, 0, 0, e)
        i = C.c_int64()
        _check(load().mc_server_submit(self.handle, C.byref(r), C.byref(i)))
        self._req[i.value] = ("estimate", h, 0)
        return i.value

    def wait(self, rid: int) -> dict:
        kind, h, count = self._req.pop(rid)
        q, lat = C.c_double(), C.c_double()
        if kind == "sample":
            nodes = np.zeros(max(count * h, 1), np.uint32)
            cls = np.zeros(max(count, 1), np.int32)
            _check(load().mc_server_wait(self.handle, rid, _ptr(nodes), _ptr(cls), None, None,
                                         C.byref(q), C.byref(lat)))
            return {"nodes": nodes[: count * h].reshape(count, h), "classes": cls[:count],
                    "queue_us": q.value, "latency_us": lat.value}
        nc = num_classes(h)
        est = np.zeros(nc, np.float64)
        hits = np.zeros(nc, np.uint64)
        _check(load().mc_server_wait(self.handle, rid, None, None, _ptr(est), _ptr(hits),
                                     C.byref(q), C.byref(lat)))
        return {"est": est, "hits": hits, "queue_us": q.value, "latency_us": lat.value}

    def free(self):
        if getattr(self, "handle", None):
            load().mc_server_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
