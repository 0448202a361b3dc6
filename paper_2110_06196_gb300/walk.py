"""Python face of libgrape_walk: the same calls as include/grape_walk.h, taking
torch tensors for device memory and torch streams for ordering.

PyTorch is plumbing here: it allocates device memory and supplies the stream.
Every walk step runs in the library's kernels.
"""
from __future__ import annotations

import atexit
import ctypes
import weakref

import numpy as np
import torch

from . import _lib
from ._lib import GrapeError, check


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dev_tensor(x, dtype, device):
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(x)
    if x.device.type != "cuda" or x.dtype != dtype or not x.is_contiguous():
        x = x.to(device=device, dtype=dtype).contiguous()
    return x


class Graph:
    """A CSR graph resident in device memory (grape_graph_create)."""

    def __init__(self, offsets, dsts, weights=None, undirected=True, validate=True,
                 device="cuda", stream=None):
        lib = _lib.load()
        offsets = _dev_tensor(offsets, torch.int64, device)
        dsts = _dev_tensor(dsts, torch.int32, device)
        weights = None if weights is None else _dev_tensor(weights, torch.float32, device)
        n = offsets.numel() - 1
        flags = (_lib.GRAPE_UNDIRECTED if undirected else 0) | (_lib.GRAPE_VALIDATE if validate else 0)
        h = ctypes.c_void_p()
        with torch.cuda.device(offsets.device):
            code = lib.grape_graph_create(_ptr(offsets), _ptr(dsts), _ptr(weights), n,
                                          dsts.numel(), flags, _stream_ptr(stream),
                                          ctypes.byref(h))
        check(code, "grape_graph_create")
        self._h = h
        self._lib = lib
        self.device = offsets.device
        self.num_nodes = n
        self.num_entries = dsts.numel()
        self.weighted = weights is not None

    @classmethod
    def from_csr(cls, csr, undirected=True, validate=True, device="cuda"):
        return cls(csr.offsets, csr.dsts, csr.weights, undirected, validate, device)

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("graph is closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.grape_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        i = _lib.GraphInfo()
        check(self._lib.grape_graph_info(self.handle, ctypes.byref(i)), "grape_graph_info")
        return {f: getattr(i, f) for f, _ in i._fields_ if f != "pad"}

    def get_tuning(self) -> _lib.Tuning:
        t = _lib.Tuning()
        check(self._lib.grape_graph_get_tuning(self.handle, ctypes.byref(t)))
        return t

    def set_tuning(self, **kw):
        t = self.get_tuning()
        for k, v in kw.items():
            setattr(t, k, v)
        check(self._lib.grape_graph_set_tuning(self.handle, ctypes.byref(t)), "set_tuning")
        return t

    def stream_status(self, stream=None):
        """Synchronise, read and clear the device status word (raises GRAPE_ERR_DEVICE)."""
        check(self._lib.grape_stream_status(self.handle, _stream_ptr(stream)), "stream_status")

    def counters(self, enable=None):
        if enable is not None:
            check(self._lib.grape_counters_enable(self.handle, 1 if enable else 0))
            return None
        c = _lib.Counters()
        check(self._lib.grape_counters_read(self.handle, ctypes.byref(c)))
        return c.as_dict()


def walks(graph: Graph, starts=None, walk_len=80, walks_per_node=1, p=1.0, q=1.0, seed=0,
          num_starts=None, out=None, stream=None) -> torch.Tensor:
    """grape_walks: rows [walks_per_node * num_starts, walk_len] int32 on the device."""
    lib = graph._lib
    if starts is not None:
        starts = _dev_tensor(starts, torch.int32, graph.device)
        ns = starts.numel()
    else:
        ns = graph.num_nodes if num_starts is None else int(num_starts)
    rows = ns * walks_per_node
    if out is None:
        out = torch.empty((rows, walk_len), dtype=torch.int32, device=graph.device)
    code = lib.grape_walks(graph.handle, _ptr(starts), ns, walk_len, walks_per_node, float(p),
                           float(q), int(seed) & (2**64 - 1), _ptr(out), _stream_ptr(stream))
    check(code, "grape_walks")
    return out


def walks_cumsum(graph: Graph, starts=None, walk_len=80, walks_per_node=1, p=1.0, q=1.0, seed=0,
                 num_starts=None, out=None, stream=None) -> torch.Tensor:
    """grape_walks_cumsum: the paper's cumulative-sum sampler at every step (the
    rows of walks() with trial_cap = 0)."""
    lib = graph._lib
    if starts is not None:
        starts = _dev_tensor(starts, torch.int32, graph.device)
        ns = starts.numel()
    else:
        ns = graph.num_nodes if num_starts is None else int(num_starts)
    if out is None:
        out = torch.empty((ns * walks_per_node, walk_len), dtype=torch.int32, device=graph.device)
    code = lib.grape_walks_cumsum(graph.handle, _ptr(starts), ns, walk_len, walks_per_node,
                                  float(p), float(q), int(seed) & (2**64 - 1), _ptr(out),
                                  _stream_ptr(stream))
    check(code, "grape_walks_cumsum")
    return out


def walks_approx(graph: Graph, starts=None, walk_len=80, walks_per_node=1, p=1.0, q=1.0, seed=0,
                 suss_k=10000, num_starts=None, out=None, stream=None) -> torch.Tensor:
    """grape_walks_approx: approximated walks (SUSS sub-samples of suss_k
    neighbours at nodes of degree above suss_k)."""
    lib = graph._lib
    if starts is not None:
        starts = _dev_tensor(starts, torch.int32, graph.device)
        ns = starts.numel()
    else:
        ns = graph.num_nodes if num_starts is None else int(num_starts)
    if out is None:
        out = torch.empty((ns * walks_per_node, walk_len), dtype=torch.int32, device=graph.device)
    code = lib.grape_walks_approx(graph.handle, _ptr(starts), ns, walk_len, walks_per_node,
                                  float(p), float(q), int(seed) & (2**64 - 1), int(suss_k),
                                  _ptr(out), _stream_ptr(stream))
    check(code, "grape_walks_approx")
    return out


def walks_host(graph: Graph, starts=None, walk_len=80, walks_per_node=1, p=1.0, q=1.0, seed=0,
               num_starts=None, out=None, stream=None) -> np.ndarray:
    """grape_walks_host: host starts in, host rows out (copies inside the call)."""
    lib = graph._lib
    st = None
    if starts is not None:
        st = np.ascontiguousarray(starts, dtype=np.int32)
        ns = st.size
    else:
        ns = graph.num_nodes if num_starts is None else int(num_starts)
    if out is None:
        out = np.empty((ns * walks_per_node, walk_len), dtype=np.int32)
    sp = None if st is None else ctypes.c_void_p(st.ctypes.data)
    op = ctypes.c_void_p(out.data_ptr()) if isinstance(out, torch.Tensor) else \
        ctypes.c_void_p(out.ctypes.data)
    code = lib.grape_walks_host(graph.handle, sp, ns, walk_len, walks_per_node, float(p),
                                float(q), int(seed) & (2**64 - 1), op, _stream_ptr(stream))
    check(code, "grape_walks_host")
    return out


def trim_scratch(keep_bytes: int = 0):
    """grape_trim_scratch: release the pooled device scratch of host-buffer calls."""
    check(_lib.load().grape_trim_scratch(int(keep_bytes)), "grape_trim_scratch")


def contexts_from_rows(rows: torch.Tensor, window: int, out=None, stream=None) -> torch.Tensor:
    """grape_contexts_from_rows: int32 [num_rows, walk_len, 2 * window] on the device."""
    lib = _lib.load()
    rows = rows.contiguous()
    n, L = rows.shape
    if out is None:
        out = torch.empty((n, L, 2 * window), dtype=torch.int32, device=rows.device)
    check(lib.grape_contexts_from_rows(_ptr(rows), n, L, int(window), _ptr(out),
                                       _stream_ptr(stream)), "grape_contexts_from_rows")
    return out


def contexts(graph: Graph, starts=None, walk_len=80, walks_per_node=1, p=1.0, q=1.0, seed=0,
             window=5, walk_begin=0, walk_count=None, num_starts=None, centres=False, out=None,
             stream=None):
    """grape_walk_contexts: (centre rows or None, contexts) on the device for walks
    [walk_begin, walk_begin + walk_count) of the job."""
    lib = graph._lib
    if starts is not None:
        starts = _dev_tensor(starts, torch.int32, graph.device)
        ns = starts.numel()
    else:
        ns = graph.num_nodes if num_starts is None else int(num_starts)
    total = ns * walks_per_node
    count = total - walk_begin if walk_count is None else int(walk_count)
    cen = None
    if centres:
        cen = torch.empty((count, walk_len), dtype=torch.int32, device=graph.device)
    if out is None:
        out = torch.empty((count, walk_len, 2 * window), dtype=torch.int32, device=graph.device)
    code = lib.grape_walk_contexts(graph.handle, _ptr(starts), ns, walk_len, walks_per_node,
                                   float(p), float(q), int(seed) & (2**64 - 1), int(window),
                                   int(walk_begin), count, _ptr(cen), _ptr(out),
                                   _stream_ptr(stream))
    check(code, "grape_walk_contexts")
    return cen, out


def _requests(reqs, graph):
    """list of dicts {starts (device tensor or None), num_starts, walk_len,
    walks_per_node, p, q, seed, out (device tensor)} -> ctypes array."""
    arr = (_lib.WalkRequest * len(reqs))()
    keep = []
    for j, r in enumerate(reqs):
        st = r.get("starts")
        if st is not None:
            st = _dev_tensor(st, torch.int32, graph.device)
            keep.append(st)
        ns = st.numel() if st is not None else int(r["num_starts"])
        wpn = int(r.get("walks_per_node", 1))
        out = r.get("out")
        if out is None:
            out = torch.empty((ns * wpn, int(r["walk_len"])), dtype=torch.int32,
                              device=graph.device)
            r["out"] = out
        keep.append(out)
        arr[j] = _lib.WalkRequest(None if st is None else st.data_ptr(), ns, int(r["walk_len"]),
                                  wpn, float(r["p"]), float(r["q"]),
                                  int(r["seed"]) & (2**64 - 1), out.data_ptr())
    return arr, keep


class BatchPlan:
    """grape_batch_plan_*: all requests in one persistent launch replayed from a CUDA graph."""

    def __init__(self, graph: Graph, reqs, stream=None):
        self.graph = graph
        self.reqs = reqs
        self._arr, self._keep = _requests(reqs, graph)
        h = ctypes.c_void_p()
        check(graph._lib.grape_batch_plan_create(graph.handle, self._arr, len(reqs),
                                                 _stream_ptr(stream), ctypes.byref(h)),
              "grape_batch_plan_create")
        self._h = h

    def launch(self, stream=None):
        check(self.graph._lib.grape_batch_plan_launch(self._h, _stream_ptr(stream)),
              "grape_batch_plan_launch")

    def outputs(self):
        return [r["out"] for r in self.reqs]

    def close(self):
        if getattr(self, "_h", None) is not None:
            self.graph._lib.grape_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def walks_batched(graph: Graph, reqs, stream=None):
    arr, keep = _requests(reqs, graph)
    check(graph._lib.grape_walks_batched(graph.handle, arr, len(reqs), _stream_ptr(stream)),
          "grape_walks_batched")
    return [r["out"] for r in reqs]


def autotune_batched(graph: Graph, reqs, stream=None) -> dict:
    arr, keep = _requests(reqs, graph)
    best = _lib.Tuning()
    check(graph._lib.grape_autotune_batched(graph.handle, arr, len(reqs), _stream_ptr(stream),
                                            ctypes.byref(best)), "grape_autotune_batched")
    return best.as_dict()


_live_servers = weakref.WeakSet()


@atexit.register
def _close_servers():
    # A process must not exit while a resident kernel may still write to the
    # server's mapped host memory: shut every live server down first.
    for s in list(_live_servers):
        try:
            s.close()
        except Exception:
            pass


class Server:
    """grape_walk_server_*: continuous batching with the graph resident."""

    def __init__(self, graph: Graph, output_cap_bytes=40 << 30, max_inflight=1024,
                 chunk_walks=0, max_chunks=1 << 22, idle_exit_us=2000, admit_timeout_ms=0,
                 kernel_wait_ms=0):
        self.graph = graph
        cfg = _lib.ServerConfig(output_cap_bytes, max_inflight, chunk_walks, max_chunks,
                                idle_exit_us, admit_timeout_ms, kernel_wait_ms)
        h = ctypes.c_void_p()
        check(graph._lib.grape_walk_server_create(graph.handle, ctypes.byref(cfg),
                                                  ctypes.byref(h)), "grape_walk_server_create")
        self._h = h
        self._lib = graph._lib
        self._outs = {}
        _live_servers.add(self)

    def submit(self, starts, walk_len, p, q, seed, walks_per_node=1, out=None, hold=False):
        """Host starts (copied at once); `out` a host int32 buffer (numpy or pinned
        torch) of [walks_per_node * len(starts), walk_len], allocated if None.
        hold=True: no buffer now; the rows wait in the server's device arena and
        wait() copies them into a buffer it allocates."""
        st = np.ascontiguousarray(starts, dtype=np.int32)
        shape = (st.size * walks_per_node, walk_len)
        if hold:
            op = None
        else:
            if out is None:
                out = np.empty(shape, dtype=np.int32)
            op = out.data_ptr() if isinstance(out, torch.Tensor) else out.ctypes.data
        req = _lib.WalkRequest(st.ctypes.data, st.size, walk_len, walks_per_node, float(p),
                               float(q), int(seed) & (2**64 - 1), op)
        t = ctypes.c_uint64()
        check(self._lib.grape_walk_server_submit(self._h, ctypes.byref(req), ctypes.byref(t)),
              "grape_walk_server_submit")
        self._outs[t.value] = ("held", shape) if hold else out
        return t.value

    def wait(self, ticket, timeout_ms=-1):
        held = self._outs.get(ticket)
        host = None
        if isinstance(held, tuple):
            host = np.empty(held[1], dtype=np.int32)
        code = self._lib.grape_walk_server_wait(self._h, ticket, int(timeout_ms),
                                                None if host is None else host.ctypes.data)
        out = self._outs.pop(ticket, None) if code != _lib.CODES["GRAPE_ERR_TIMEOUT"] else None
        check(code, "grape_walk_server_wait")
        return host if host is not None else out

    def wait_any(self, timeout_ms=-1):
        """(ticket, latency_s, rows) of the next finished request.  Held rows
        land in a buffer as large as the largest held request, returned as
        that request's view of it."""
        t = ctypes.c_uint64()
        lat = ctypes.c_int64()
        held = [v[1] for v in self._outs.values() if isinstance(v, tuple)]
        host = np.empty(max(a * b for a, b in held), dtype=np.int32) if held else None
        code = self._lib.grape_walk_server_wait_any(self._h, int(timeout_ms), ctypes.byref(t),
                                                    ctypes.byref(lat),
                                                    None if host is None else host.ctypes.data)
        if code == _lib.CODES["GRAPE_ERR_TIMEOUT"]:
            raise GrapeError(code, "grape_walk_server_wait_any")
        out = self._outs.pop(t.value, None)
        check(code, f"ticket {t.value}")
        if isinstance(out, tuple):
            out = host[:out[1][0] * out[1][1]].reshape(out[1])
        return t.value, lat.value * 1e-9, out

    def cancel(self, ticket):
        check(self._lib.grape_walk_server_cancel(self._h, ticket), "grape_walk_server_cancel")

    def inject_fault(self, no_heartbeat: bool):
        """grape_walk_server_inject_fault: stop (True) or restore (False) the host
        heartbeat that renews the resident kernel's bounded wait."""
        check(self._lib.grape_walk_server_inject_fault(
            self._h, _lib.GRAPE_FAULT_NO_HEARTBEAT if no_heartbeat else 0),
            "grape_walk_server_inject_fault")

    def stats(self) -> dict:
        s = _lib.ServerStats()
        check(self._lib.grape_walk_server_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.grape_walk_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def philox4x32_10(ctr_key: torch.Tensor, stream=None) -> torch.Tensor:
    """Device Philox4x32-10 on rows (c0 c1 c2 c3 k0 k1) of an int32 [n, 6] tensor
    holding uint32 bit patterns; returns int32 [n, 4] bit patterns."""
    lib = _lib.load()
    ck = ctr_key.contiguous()
    out = torch.empty((ck.shape[0], 4), dtype=torch.int32, device=ck.device)
    check(lib.grape_philox4x32_10(_ptr(ck), ck.shape[0], _ptr(out), _stream_ptr(stream)))
    return out


def sector_probe(buf: torch.Tensor, n_reads: int, seed: int, mode: int = 0, load_bytes: int = 32,
                 loads_in_flight: int = 8, blocks_per_sm: int = 0, stream=None) -> tuple:
    """grape_sector_probe: random 32-byte-sector reads over `buf` (mode: 0
    ld.global.nc, 1 .cg, 2 .cs; load_bytes 4/16/32, or 64 for both sectors of a
    64-byte block; loads_in_flight per thread; blocks_per_sm 0 = occupancy
    maximum).  Returns (32-byte sectors read, resident 256-thread blocks per SM)."""
    lib = _lib.load()
    sink = torch.zeros(1, dtype=torch.int32, device=buf.device)
    res = ctypes.c_int32()
    done = ctypes.c_int64()
    check(lib.grape_sector_probe(_ptr(buf), buf.numel() * buf.element_size(), int(n_reads),
                                 int(seed), int(mode), int(load_bytes), int(loads_in_flight),
                                 int(blocks_per_sm), _ptr(sink), ctypes.byref(res),
                                 ctypes.byref(done), _stream_ptr(stream)), "grape_sector_probe")
    return done.value, res.value
