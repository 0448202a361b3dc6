"""CPU oracle for node2vec second-order random walks (GRAPE, Methods,
"Implementation of second-order RWs", eqs. alphaRW, alpha and beta).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_2110_06196_gb300``) neither imports it nor shares code with it.

The arithmetic lives in ``walk_oracle.c`` (plain C, single-threaded, built with
``gcc -O2 -ffp-contract=off``); this module compiles it on first use and wraps
it with ctypes.  ctypes drops the GIL for the duration of each call, so
``walks_parallel`` runs disjoint walk-id ranges on several host threads and
gets byte-identical output to a single-threaded call.

Pins (see ``tests/test_oracle_*.py``): Philox4x32-10 against the published
known-answer vectors; transition frequencies against the exact law computed from
graph distances d(t, x) (eq. alphaRW) by chi-square; closed forms on cycles,
complete graphs and stars; stationarity of p = q = 1 walks; the trial-cap
fallback against the same exact law; and the context windows against a worked
example, an independent sliding-window construction, a closed-form count and
their symmetry.

``elias_fano.py`` is the oracle of the Elias-Fano graph store (plain Python and
numpy): the edge encoding phi_k, the low/high split, the quantum indexes, and
rank and select, pinned in ``tests/test_oracle_ef.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "walk_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]

DEFAULT_TRIAL_CAP = 4096

_lock = threading.Lock()
_lib = None


class OracleStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("trials", ctypes.c_int64),
                ("fallbacks", ctypes.c_int64)]


def compile_oracle(src: str = _SRC, out: str = _LIB_PATH, extra_flags=()) -> str:
    """Compile ``src`` into the shared library ``out`` with gcc."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *CFLAGS, *extra_flags, src, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, out)
    return out


def _bind(lib):
    i64, i32, u64, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
    vp = ctypes.c_void_p
    lib.oracle_philox4x32_10.argtypes = [vp, vp, vp]
    lib.oracle_philox4x32_10.restype = None
    lib.oracle_thresholds.argtypes = [dbl, dbl, vp]
    lib.oracle_thresholds.restype = None
    lib.oracle_weighted_accept.argtypes = [ctypes.c_uint32, ctypes.c_float, u64, ctypes.c_float]
    lib.oracle_weighted_accept.restype = ctypes.c_int
    lib.oracle_node_wmax.argtypes = [vp, vp, i64, vp]
    lib.oracle_node_wmax.restype = None
    lib.oracle_next.argtypes = [vp, vp, vp, vp, i32, i32, dbl, dbl, u64, i64, i32, i64, i64, vp]
    lib.oracle_next.restype = i32
    lib.oracle_next_many.argtypes = [vp, vp, vp, vp, i32, i32, dbl, dbl, u64, i64, i64,
                                     i32, i64, i64, vp, vp]
    lib.oracle_next_many.restype = None
    lib.oracle_walks.argtypes = [vp, vp, vp, vp, i64, vp, i64, i32, dbl, dbl, u64, i64,
                                 i64, i64, i64, vp, vp]
    lib.oracle_suss_positions.argtypes = [i64, i64, u64, i64, i32, vp]
    lib.oracle_suss_positions.restype = None
    lib.oracle_walks.restype = ctypes.c_int
    lib.oracle_contexts.argtypes = [vp, i64, i32, i32, vp]
    lib.oracle_contexts.restype = None
    return lib


def load(path: str | None = None):
    """Load (building if needed) the oracle library.  ``path`` loads another
    build of the same source, e.g. one compiled with different flags."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            stale = (not os.path.exists(_LIB_PATH)
                     or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
            if stale:
                compile_oracle()
            _lib = _bind(ctypes.CDLL(_LIB_PATH))
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class Graph:
    """Host CSR graph as the oracle sees it: int64 offsets[n+1], int32 dsts[m]
    sorted ascending and duplicate-free within each row, optional fp32 weights."""

    def __init__(self, offsets, dsts, weights=None, lib=None):
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self.dsts = np.ascontiguousarray(dsts, dtype=np.int32)
        self.weights = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
        self.num_nodes = len(self.offsets) - 1
        self.lib = lib if lib is not None else load()
        self.wmax = None
        if self.weights is not None:
            self.wmax = np.zeros(self.num_nodes, dtype=np.float32)
            self.lib.oracle_node_wmax(_ptr(self.offsets), _ptr(self.weights),
                                      self.num_nodes, _ptr(self.wmax))

    def degree(self, v):
        return int(self.offsets[v + 1] - self.offsets[v])


def philox4x32_10(ctr, key, lib=None):
    """Philox4x32-10 of one counter block (4 x uint32) under key (2 x uint32)."""
    lib = lib or load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib.oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def weighted_accept(r2, wmax, T, w, lib=None):
    """The weighted acceptance test r2 * wmax < T * w (exact)."""
    lib = lib or load()
    return bool(lib.oracle_weighted_accept(int(r2), float(wmax), int(T), float(w)))


def thresholds(p, q, lib=None):
    """(T_return, T_in, T_out) as Python ints."""
    lib = lib or load()
    t = np.zeros(3, dtype=np.uint64)
    lib.oracle_thresholds(float(p), float(q), _ptr(t))
    return tuple(int(x) for x in t)


def next_many(g: Graph, t, v, p, q, seed, walk_begin, n, step, trial_cap=DEFAULT_TRIAL_CAP,
              stats=None, suss_k=0):
    """n independent draws of the transition out of v with previous node t
    (t = -1: first step), one per walk id in [walk_begin, walk_begin + n).
    suss_k > 0: approximated walks (SUSS sub-sample of k when deg(v) > k)."""
    out = np.empty(n, dtype=np.int32)
    st = stats if stats is not None else OracleStats()
    g.lib.oracle_next_many(_ptr(g.offsets), _ptr(g.dsts), _ptr(g.weights), _ptr(g.wmax),
                           int(t), int(v), float(p), float(q), int(seed), int(walk_begin),
                           int(n), int(step), int(trial_cap), int(suss_k), _ptr(out),
                           ctypes.byref(st))
    return out


def walks(g: Graph, starts, walk_len, walks_per_node, p, q, seed,
          trial_cap=DEFAULT_TRIAL_CAP, walk_ids=None, stats=None, suss_k=0):
    """Walk rows for all walk ids (default) or for the half-open id range
    ``walk_ids = (begin, end)``.  ``starts`` None means every node in order.
    suss_k > 0: approximated walks (GRAPE, "Approximated RWs").
    Returns (rows int32[count, walk_len], rc) with rc -1 on a bad start id."""
    num_starts = g.num_nodes if starts is None else len(starts)
    st_arr = None if starts is None else np.ascontiguousarray(starts, dtype=np.int32)
    total = num_starts * walks_per_node
    b, e = (0, total) if walk_ids is None else walk_ids
    out = np.empty((max(e - b, 0), walk_len), dtype=np.int32)
    st = stats if stats is not None else OracleStats()
    rc = g.lib.oracle_walks(_ptr(g.offsets), _ptr(g.dsts), _ptr(g.weights), _ptr(g.wmax),
                            g.num_nodes, _ptr(st_arr), num_starts, int(walk_len), float(p),
                            float(q), int(seed), int(trial_cap), int(suss_k), int(b), int(e),
                            _ptr(out), ctypes.byref(st))
    return out, rc


def suss_positions(deg, k, seed, walk_id, step, lib=None):
    """Row positions of the SUSS sub-sample of one step (k of them when deg > k,
    else all deg positions)."""
    lib = lib or load()
    m = k if 0 < k < deg else deg
    out = np.empty(m, dtype=np.int64)
    lib.oracle_suss_positions(int(deg), int(k), int(seed), int(walk_id), int(step), _ptr(out))
    return out


def walks_parallel(g: Graph, starts, walk_len, walks_per_node, p, q, seed, walk_ids=None,
                   threads=None, trial_cap=DEFAULT_TRIAL_CAP):
    """``walks`` split over host threads by contiguous walk-id ranges."""
    num_starts = g.num_nodes if starts is None else len(starts)
    total = num_starts * walks_per_node
    b, e = (0, total) if walk_ids is None else walk_ids
    threads = threads or os.cpu_count() or 1
    bounds = np.linspace(b, e, threads + 1).astype(np.int64)
    out = np.empty((e - b, walk_len), dtype=np.int32)

    def run(j):
        lo, hi = int(bounds[j]), int(bounds[j + 1])
        rows, _ = walks(g, starts, walk_len, walks_per_node, p, q, seed, trial_cap,
                        walk_ids=(lo, hi))
        out[lo - b:hi - b] = rows

    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(run, range(threads)))
    return out


def walk_rows(g: Graph, starts, walk_len, walks_per_node, p, q, seed, ids,
              trial_cap=DEFAULT_TRIAL_CAP):
    """Rows for an arbitrary list of walk ids (one oracle call per id)."""
    out = np.empty((len(ids), walk_len), dtype=np.int32)
    for j, w in enumerate(ids):
        rows, _ = walks(g, starts, walk_len, walks_per_node, p, q, seed, trial_cap,
                        walk_ids=(int(w), int(w) + 1))
        out[j] = rows[0]
    return out


def contexts(rows, window, lib=None):
    """Context windows of walk rows (``oracle_contexts``): int32
    [num_rows, walk_len, 2 * window], the ``window`` positions before each
    centre then the ``window`` after it, -1 outside the row, after a dead end,
    or around a -1 centre."""
    lib = lib or load()
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    n, L = rows.shape
    out = np.empty((n, L, 2 * window), dtype=np.int32)
    lib.oracle_contexts(_ptr(rows), int(n), int(L), int(window), _ptr(out))
    return out
