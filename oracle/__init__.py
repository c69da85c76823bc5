"""CPU oracle for colour-coding treelet counting and graphlet sampling.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only users.  Nothing here is imported
by, or imports, the CUDA library ``paper_2009_03052_gb300``.

The exact-integer core is plain C (``motif_oracle.c``, built here with gcc);
the treelet catalogue is plain Python (``catalog.py``).  Each function cites
the part of the paper it writes out.

Parity status: every function is pinned by the ``-m "not gpu"`` tests
(brute force on tiny graphs, closed forms, the colouring-average
invariant, Philox known-answer vectors, published sequence counts, exact
sampler probabilities, estimator unbiasedness).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

from . import catalog as _cat

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libmotif_oracle.so")
_SRC = os.path.join(_HERE, "motif_oracle.c")
_lock = threading.Lock()
_lib = None

OK, INVALID, NOMEM, OVERFLOW, INTERNAL = 0, 1, 2, 3, 7


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        super().__init__(f"oracle status {status} {what}")
        self.status = status


class OracleOverflow(OracleError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle's C core with gcc (no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread",
                               "-ffp-contract=off", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        P = C.c_void_p
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C")
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C")
        u64p = np.ctypeslib.ndpointer(np.uint64, flags="C")
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
        lib.oc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.oc_color.argtypes = [C.c_int64, C.c_int, C.c_uint64, u8p]
        lib.oc_draw_below.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, u64p, u64p]
        lib.oc_build.restype = P
        lib.oc_build.argtypes = [C.c_int64, i64p, u32p, u8p, C.c_int, C.c_int, C.c_int,
                                 i32p, i32p, i32p, i32p, i32p, i32p, i32p, C.c_int, C.c_int,
                                 C.c_int, C.POINTER(C.c_int)]
        lib.oc_free.argtypes = [P]
        lib.oc_read_level.argtypes = [P, C.c_int, u64p]
        lib.oc_neighbor_sum.argtypes = [P, C.c_int, C.c_int64, u64p]
        lib.oc_total.argtypes = [P, C.c_int, C.c_int, u64p, u64p]
        lib.oc_sample.argtypes = [P, C.c_int, C.c_int, C.c_uint64, C.c_uint64, C.c_int64,
                                  u32p, u32p, i32p, i32p]
        lib.oc_canonical_code.restype = C.c_uint32
        lib.oc_canonical_code.argtypes = [C.c_int, C.c_uint32]
        lib.oc_num_classes.argtypes = [C.c_int]
        lib.oc_class_codes.argtypes = [C.c_int, u32p]
        lib.oc_class_of_word.argtypes = [C.c_int, C.c_uint32]
        lib.oc_spanning_trees.restype = C.c_int64
        lib.oc_spanning_trees.argtypes = [C.c_int, C.c_uint32]
        lib.oc_sigma_matrix.argtypes = [C.c_int, C.c_int, i32p, i32p, i32p, i32p, i32p, i32p,
                                        i32p, C.c_int, i64p, C.c_int]
        lib.oc_estimate_uniform.argtypes = [P, C.c_int, C.c_uint64, C.c_uint64, C.c_int64,
                                            i64p, C.c_int64, i64p, C.c_uint32, f64p, u64p]
        lib.oc_estimate_ags.argtypes = [P, C.c_int, C.c_uint64, C.c_uint64, C.c_int64, C.c_int64,
                                        i64p, C.c_int, C.c_int64, i64p, i64p, C.c_uint32, f64p, u64p,
                                        i64p, C.c_int64, P, P, P]
        lib.oc_color_biased.argtypes = [C.c_int64, C.c_int, C.c_uint64, C.c_uint32, u8p]
        lib.oc_inv_colorful_prob.restype = C.c_double
        lib.oc_inv_colorful_prob.argtypes = [C.c_int, C.c_int, C.c_uint32]
        lib.oc_star_total.argtypes = [P, C.c_int, u64p]
        lib.oc_sample_stars.argtypes = [P, C.c_int, C.c_uint64, C.c_uint64, C.c_int64,
                                        u32p, u32p, i32p]
        _lib = lib
        return lib


def _check(st: int, what: str = ""):
    if st == OVERFLOW:
        raise OracleOverflow(st, what)
    if st != OK:
        raise OracleError(st, what)


def _u128(lo_hi) -> int:
    return int(lo_hi[0]) | (int(lo_hi[1]) << 64)


# ---------------------------------------------------------------------------
# random numbers and colouring
# ---------------------------------------------------------------------------

def philox4x32_10(counter, key) -> tuple[int, int, int, int]:
    out = np.zeros(4, np.uint32)
    _load().oc_philox4x32_10(np.asarray(counter, np.uint32), np.asarray(key, np.uint32), out)
    return tuple(int(x) for x in out)


def draw_below(seed: int, index: int, step: int, W: int) -> int:
    """uniform(W) of sample ``index`` at descent step ``step``."""
    out = np.zeros(2, np.uint64)
    w = np.array([W & (2**64 - 1), W >> 64], np.uint64)
    _load().oc_draw_below(seed, index, step, w, out)
    return _u128(out)


def color(n: int, k: int, seed: int) -> np.ndarray:
    """c_v uniform in [k] (Section 2.1), counter-based."""
    out = np.zeros(max(n, 1), np.uint8)
    _load().oc_color(n, k, seed, out)
    return out[:n]


def color_biased(n: int, k: int, seed: int, bias_q32: int) -> np.ndarray:
    """Biased colouring (Section 3.5): colours 1..k-1 with probability
    lambda = bias_q32 / 2^32 each, colour 0 otherwise."""
    out = np.zeros(max(n, 1), np.uint8)
    _check(_load().oc_color_biased(n, k, seed, bias_q32, out))
    return out[:n]


def inv_colorful_prob_biased(k: int, h: int, bias_q32: int) -> float:
    return float(_load().oc_inv_colorful_prob(k, h, bias_q32))


# ---------------------------------------------------------------------------
# catalogue helpers
# ---------------------------------------------------------------------------

def _catalog_arrays(cat: "_cat.Catalog"):
    a = lambda x: np.ascontiguousarray(np.asarray(x, np.int32))
    copies = [c for h in range(1, cat.k + 1) for c in cat.copies_divisor(h)]
    return (len(cat.strings), a(cat.size), a(cat.local), a(cat.left), a(cat.right),
            a(cat.beta), a(cat.unrooted), a(copies))


def num_classes(h: int) -> int:
    return int(_load().oc_num_classes(h))


def class_codes(h: int) -> np.ndarray:
    """Canonical adjacency words of the connected h-node graphs, ascending
    (their positions are the class ids)."""
    out = np.zeros(num_classes(h), np.uint32)
    _check(_load().oc_class_codes(h, out))
    return out


def canonical_code(h: int, word: int) -> int:
    return int(_load().oc_canonical_code(h, word))


def class_of_word(h: int, word: int) -> int:
    return int(_load().oc_class_of_word(h, word))


def spanning_trees(h: int, word: int) -> int:
    """sigma by Kirchhoff's matrix-tree theorem (Section 4.4.3)."""
    return int(_load().oc_spanning_trees(h, word))


_sigma_cache: dict[int, tuple[np.ndarray, np.ndarray]] = {}


def sigma(h: int) -> tuple[np.ndarray, np.ndarray]:
    """(sigma_i [classes], sigma_ij [classes x unrooted shapes]) for h-node
    graphlets; sigma_i by Kirchhoff, sigma_ij by the distinct-colour build
    (Section 4.4.3)."""
    if h not in _sigma_cache:
        codes = class_codes(h)
        s_i = np.array([spanning_trees(h, int(w)) for w in codes], np.int64)
        cat = _cat.Catalog(h)
        nsh, *arrs = _catalog_arrays(cat)
        nu = cat.n_unrooted(h)
        s_ij = np.zeros((len(codes), nu), np.int64)
        _check(_load().oc_sigma_matrix(h, nsh, *arrs, nu, s_ij, min(16, os.cpu_count() or 1)),
               "sigma")
        _sigma_cache[h] = (s_i, s_ij)
    return _sigma_cache[h]


def inv_colorful_prob(k: int, h: int) -> float:
    return float(k ** h * math.factorial(k - h)) / float(math.factorial(k))


# ---------------------------------------------------------------------------
# tables
# ---------------------------------------------------------------------------

class Tables:
    """Exact count tables c(T_C, v) for |T| = 1..k (Section 2.1, Eq. 1)."""

    def __init__(self, graph, colors, k: int, width: int = 128, nthreads: int | None = None,
                 zero_root: bool = False, skip_round: bool = False):
        lib = _load()
        self.k, self.width, self.zero_root, self.skip_round = k, width, zero_root, skip_round
        self.n = int(graph.n)
        self.cat = _cat.Catalog(k, skip_round)
        nsh, *arrs = _catalog_arrays(self.cat)
        self._keep = arrs
        colors = np.ascontiguousarray(np.asarray(colors, np.uint8))
        self.colors = colors
        self.graph = graph
        st = C.c_int(0)
        nthreads = nthreads or min(16, os.cpu_count() or 1)
        self.nthreads = nthreads
        h = lib.oc_build(self.n, np.ascontiguousarray(graph.row_ptr, np.int64),
                         np.ascontiguousarray(graph.col, np.uint32), colors if self.n else
                         np.zeros(1, np.uint8), k, width, nsh, *arrs, nthreads,
                         1 if zero_root else 0, 1 if skip_round else 0, C.byref(st))
        _check(st.value, "build")
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None):
            _load().oc_free(self._h)
            self._h = None

    def level(self, h: int) -> np.ndarray:
        """uint64 array [n, r_h, C(k,h), 2] (low, high words); the colour-set
        axis is indexed by the rank of the mask among size-h masks, ascending."""
        r, q = self.cat.r(h), math.comb(self.k, h)
        out = np.zeros(max(self.n * r * q * 2, 1), np.uint64)
        _check(_load().oc_read_level(self._h, h, out))
        return out[: self.n * r * q * 2].reshape(self.n, r, q, 2)

    def level_int(self, h: int) -> list:
        """Same as level() as nested Python ints [v][shape][rank]."""
        a = self.level(h)
        lo = a[..., 0].astype(object)
        hi = a[..., 1].astype(object)
        return (lo + hi * (1 << 64)).tolist()

    def neighbor_sum(self, h: int, v: int) -> np.ndarray:
        r, q = self.cat.r(h), math.comb(self.k, h)
        out = np.zeros(r * q * 2, np.uint64)
        _check(_load().oc_neighbor_sum(self._h, h, v, out))
        return out.reshape(r, q, 2)

    def star_total(self, h: int) -> int:
        """S = sum_v C(d_v, h-1): the h-stars of the graph."""
        out = np.zeros(2, np.uint64)
        _check(_load().oc_star_total(self._h, h, out))
        return _u128(out)

    def sample_stars(self, h: int, seed: int, first_index: int, count: int):
        """Uncoloured h-stars: (nodes [count, h] ascending, centres, class ids)."""
        nodes = np.zeros(max(count * h, 1), np.uint32)
        centres = np.zeros(max(count, 1), np.uint32)
        classes = np.zeros(max(count, 1), np.int32)
        _check(_load().oc_sample_stars(self._h, h, seed, first_index, count, nodes, centres,
                                       classes), "stars")
        return nodes[: count * h].reshape(count, h), centres[:count], classes[:count]

    def total(self, h: int, unrooted: int = -1) -> tuple[int, int]:
        """(rooted total R, unrooted count: R_j / h per shape j, summed)."""
        R = np.zeros(2, np.uint64)
        U = np.zeros(2, np.uint64)
        _check(_load().oc_total(self._h, h, unrooted, R, U))
        return _u128(R), _u128(U)

    def sample(self, h: int, seed: int, first_index: int, count: int, unrooted: int = -1):
        """(nodes [count, h] ascending, roots, rooted shape ids, class ids)."""
        nodes = np.zeros(max(count * h, 1), np.uint32)
        roots = np.zeros(max(count, 1), np.uint32)
        shapes = np.zeros(max(count, 1), np.int32)
        classes = np.zeros(max(count, 1), np.int32)
        _check(_load().oc_sample(self._h, h, unrooted, seed, first_index, count,
                                 nodes, roots, shapes, classes), "sample")
        return (nodes[: count * h].reshape(count, h), roots[:count], shapes[:count],
                classes[:count])

    def _skip_sigmas(self, h: int):
        """(sigma'_i = sum_j sigma_ij a_j, sigma*_i = spanning stars of H_i) for a
        round-skipped level k; (sigma_i, zeros) otherwise."""
        s_i, s_ij = sigma(h)
        if not (self.skip_round and h == self.k):
            return s_i, np.zeros_like(s_i)
        a = np.asarray(self.cat.copies_divisor(h), np.int64)
        star = _cat.unrooted_id("10" * (h - 1))
        return (np.ascontiguousarray(s_ij @ a), np.ascontiguousarray(s_ij[:, star]))

    def estimate_uniform(self, h: int, seed: int, n_samples: int, first_index: int = 0,
                         star_samples: int = 0, bias_q32: int = 0):
        s_use, s_star = self._skip_sigmas(h)
        est = np.zeros(len(s_use), np.float64)
        hits = np.zeros(len(s_use), np.uint64)
        _check(_load().oc_estimate_uniform(self._h, h, seed, first_index, n_samples,
                                           s_use, star_samples, s_star, bias_q32, est, hits))
        return est, hits

    def estimate_ags(self, h: int, seed: int, max_samples: int, cbar: int = 1000,
                     first_index: int = 0, star_samples: int = 0, bias_q32: int = 0,
                     trace: bool = False):
        """(estimates, hits, stats).  The n-th sample drawn with treelet
        T_j has sample index first_index + j * 2^40 + n.  trace=True adds to stats the first
        treelet ("first") and, per switch, the treelet chosen ("trace_j"),
        the samples drawn by then ("trace_at") and the weights w it was
        chosen with ("trace_w", [switches, classes])."""
        _, s_ij = sigma(h)
        s_prime, s_star = self._skip_sigmas(h)
        ncls = s_ij.shape[0]
        est = np.zeros(ncls, np.float64)
        hits = np.zeros(ncls, np.uint64)
        stats = np.zeros(4, np.int64)
        cap = ncls if trace else 0
        tj = np.zeros(max(cap, 1), np.int32)
        tat = np.zeros(max(cap, 1), np.int64)
        tw = np.zeros(max(cap * ncls, 1), np.float64)
        _check(_load().oc_estimate_ags(self._h, h, seed, first_index, max_samples, cbar,
                                       np.ascontiguousarray(s_ij), s_ij.shape[1], star_samples,
                                       s_prime, s_star, bias_q32, est, hits, stats, cap,
                                       tj.ctypes.data, tat.ctypes.data, tw.ctypes.data))
        out = {"samples": int(stats[0]), "switches": int(stats[1]), "covered": int(stats[2])}
        if trace:
            ns = min(int(stats[1]), cap)
            out.update(first=int(stats[3]), trace_j=tj[:ns].copy(), trace_at=tat[:ns].copy(),
                       trace_w=tw[: ns * ncls].reshape(ns, ncls).copy())
        return est, hits, out


def ags_cbar(eps: float, delta: float, s: int) -> int:
    """Covering threshold ceil(4/eps^2 ln(2s/delta)) of Algorithm AGS."""
    return int(math.ceil(4.0 / (eps * eps) * math.log(2.0 * s / delta)))
