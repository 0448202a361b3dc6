"""Python face of the Elias-Fano graph store of libgrape_walk (the grape_ef_*
calls of include/grape_walk.h): argument marshalling only.  The store is built,
queried and walked by the library's kernels.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import check
from .walk import _dev_tensor, _ptr, _stream_ptr

PAPER_QUANTUM = 1024
DEFAULT_TRIAL_CAP = 4096


class EFGraph:
    """A graph held as the Elias-Fano representation of its edge codes
    (grape_ef_graph_create)."""

    def __init__(self, offsets, dsts, weights=None, quantum=PAPER_QUANTUM, undirected=True,
                 validate=True, device="cuda", stream=None):
        lib = _lib.load()
        offsets = _dev_tensor(offsets, torch.int64, device)
        dsts = _dev_tensor(dsts, torch.int32, device)
        weights = None if weights is None else _dev_tensor(weights, torch.float32, device)
        n = offsets.numel() - 1
        h = ctypes.c_void_p()
        with torch.cuda.device(offsets.device):
            code = lib.grape_ef_graph_create(_ptr(offsets), _ptr(dsts), _ptr(weights), n,
                                             dsts.numel(), int(quantum),
                                             (_lib.GRAPE_UNDIRECTED if undirected else 0) |
                                             (_lib.GRAPE_VALIDATE if validate else 0),
                                             _stream_ptr(stream),
                                             ctypes.byref(h))
        check(code, "grape_ef_graph_create")
        self._h = h
        self._lib = lib
        self.device = offsets.device
        self.num_nodes = n
        self.num_entries = dsts.numel()
        self.weighted = weights is not None

    @classmethod
    def from_csr(cls, csr, quantum=PAPER_QUANTUM, undirected=True, validate=True, device="cuda"):
        return cls(csr.offsets, csr.dsts, csr.weights, quantum, undirected, validate, device)

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("store is closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.grape_ef_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        i = _lib.EFInfo()
        check(self._lib.grape_ef_graph_info(self.handle, ctypes.byref(i)), "grape_ef_graph_info")
        return i.as_dict()

    def export(self, stream=None) -> dict:
        """The store's arrays as int64 device tensors (the bit arrays' words
        reinterpreted as signed)."""
        i = self.info()
        t = {name: torch.empty(max(i[length], 0), dtype=torch.int64, device=self.device)
             for name, length in (("low", "low_words"), ("high", "high_words"),
                                  ("ones_index", "ones_index_len"),
                                  ("zeros_index", "zeros_index_len"))}
        check(self._lib.grape_ef_graph_export(self.handle, _ptr(t["low"]), _ptr(t["high"]),
                                              _ptr(t["ones_index"]), _ptr(t["zeros_index"]),
                                              _stream_ptr(stream)), "grape_ef_graph_export")
        return t

    def select(self, idx, stream=None) -> torch.Tensor:
        idx = _dev_tensor(idx, torch.int64, self.device)
        out = torch.empty_like(idx)
        check(self._lib.grape_ef_select(self.handle, _ptr(idx), idx.numel(), _ptr(out),
                                        _stream_ptr(stream)), "grape_ef_select")
        return out

    def rank(self, values, stream=None) -> torch.Tensor:
        values = _dev_tensor(values, torch.int64, self.device)
        out = torch.empty_like(values)
        check(self._lib.grape_ef_rank(self.handle, _ptr(values), values.numel(), _ptr(out),
                                      _stream_ptr(stream)), "grape_ef_rank")
        return out

    def stream_status(self, stream=None):
        check(self._lib.grape_ef_stream_status(self.handle, _stream_ptr(stream)),
              "grape_ef_stream_status")

    def counters(self, enable=None):
        if enable is not None:
            check(self._lib.grape_ef_counters_enable(self.handle, 1 if enable else 0))
            return None
        c = _lib.EFCounters()
        check(self._lib.grape_ef_counters_read(self.handle, ctypes.byref(c)))
        return c.as_dict()


def ef_walks(graph: EFGraph, starts=None, walk_len=80, walks_per_node=1, p=1.0, q=1.0, seed=0,
             trial_cap=DEFAULT_TRIAL_CAP, num_starts=None, out=None, stream=None) -> torch.Tensor:
    """grape_ef_walks: rows [walks_per_node * num_starts, walk_len] int32 on the device,
    byte-identical to walks() on the same CSR."""
    if starts is not None:
        starts = _dev_tensor(starts, torch.int32, graph.device)
        ns = starts.numel()
    else:
        ns = graph.num_nodes if num_starts is None else int(num_starts)
    if out is None:
        out = torch.empty((ns * walks_per_node, walk_len), dtype=torch.int32, device=graph.device)
    code = graph._lib.grape_ef_walks(graph.handle, _ptr(starts), ns, walk_len, walks_per_node,
                                     float(p), float(q), int(seed) & (2**64 - 1), int(trial_cap),
                                     _ptr(out), _stream_ptr(stream))
    check(code, "grape_ef_walks")
    return out
