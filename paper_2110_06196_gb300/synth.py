"""Seeded synthetic inputs: Erdos-Renyi and R-MAT graphs in sorted CSR form,
walk-request mixes and arrival processes.

This module holds none of the walk arithmetic.  It only builds inputs, and both
the CUDA path and the CPU oracle consume them.  Every random number here comes
from a counter-based hash (the SplitMix64 output function, Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014) of a (stream,
index) pair.  All arithmetic is int64 tensor algebra, so a graph built on the GPU
is bit-identical to the same graph built on the CPU, and its construction does
not depend on how the work is chunked.

The graphs stand in for the paper's biomedical and social graphs, which are not
available here: STRING, CTD, PheKnowLator, Wikipedia and sk-2005 (GRAPE, Results,
"Graph processing" and "Node2vec-based models at scale").  R-MAT (Chakrabarti,
Zhan, Faloutsos, SDM 2004) with a=0.57, b=0.19, c=0.19 gives them the same
heavy-tailed, hub-dominated degree law.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

_GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def _s64(x: int) -> int:
    """Reinterpret an unsigned 64-bit constant as a signed int64."""
    x &= (1 << 64) - 1
    return x - (1 << 64) if x >= (1 << 63) else x


def _lsr(z: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 lanes (torch's >> is arithmetic)."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def mix64(z: torch.Tensor) -> torch.Tensor:
    """SplitMix64 output function on int64 lanes (wrapping arithmetic)."""
    z = z ^ _lsr(z, 30)
    z = z * _s64(_M1)
    z = z ^ _lsr(z, 27)
    z = z * _s64(_M2)
    return z ^ _lsr(z, 31)


def stream_hash(stream: int, idx: torch.Tensor) -> torch.Tensor:
    """64 random bits for every index of a named stream."""
    base = mix64(torch.tensor([_s64(stream * _GAMMA + 0x632BE59BD9B4E019)], dtype=torch.int64))
    base = int(base.item())
    return mix64(idx.to(torch.int64) * _s64(_GAMMA) + base)


def _u32_hi(h: torch.Tensor) -> torch.Tensor:
    return _lsr(h, 32)


def _u32_lo(h: torch.Tensor) -> torch.Tensor:
    return h & 0xFFFFFFFF


# --------------------------------------------------------------------------
# Edge streams
# --------------------------------------------------------------------------

def rmat_pairs(scale: int, a: float, b: float, c: float, seed: int, begin: int, count: int,
               device) -> tuple[torch.Tensor, torch.Tensor]:
    """Candidate edges begin..begin+count-1 of an R-MAT stream: at each of the
    `scale` levels the quadrant (a | b | c | d) picks one bit of src and dst."""
    ta = int(math.floor(a * 2**32))
    tab = int(math.floor((a + b) * 2**32))
    tabc = int(math.floor((a + b + c) * 2**32))
    k = torch.arange(begin, begin + count, dtype=torch.int64, device=device)
    src = torch.zeros(count, dtype=torch.int64, device=device)
    dst = torch.zeros(count, dtype=torch.int64, device=device)
    levels_per_hash = 2
    nh = (scale + levels_per_hash - 1) // levels_per_hash
    for j in range(nh):
        h = stream_hash(seed * 64 + j, k)
        for half in range(levels_per_hash):
            lvl = j * levels_per_hash + half
            if lvl >= scale:
                break
            u = _u32_hi(h) if half == 0 else _u32_lo(h)
            sbit = (u >= tab).to(torch.int64)                       # quadrants c, d
            dbit = ((u >= ta) & (u < tab)) | (u >= tabc)            # quadrants b, d
            src = src | (sbit << lvl)
            dst = dst | (dbit.to(torch.int64) << lvl)
    return src, dst


def uniform_pairs(n: int, seed: int, begin: int, count: int, device):
    """Candidate edges of a uniform (Erdos-Renyi G(n, m)) stream."""
    k = torch.arange(begin, begin + count, dtype=torch.int64, device=device)
    h = stream_hash(seed * 64 + 1, k)
    src = (_u32_hi(h) * n) >> 32
    dst = (_u32_lo(h) * n) >> 32
    return src, dst


def first_unique_undirected(pair_fn, n: int, m: int, device, overshoot: float = 1.3):
    """The first m distinct unordered non-loop pairs of a candidate stream, in
    stream order.  Grows the prefix until m are found, so the result does not
    depend on the initial prefix length.  Keys are sorted in parts of disjoint
    key ranges so that no single sort exceeds torch's 2^31 - 1 element limit."""
    count = max(int(m * overshoot) + 1024, 16)
    while True:
        src, dst = pair_fn(0, count)
        lo = torch.minimum(src, dst)
        hi = torch.maximum(src, dst)
        ok = lo != hi
        key = torch.where(ok, lo * n + hi, torch.full_like(lo, -1))
        del src, dst, lo, hi, ok
        parts = 1
        while count // parts > (1 << 29):
            parts *= 2
        bounds = [n * n * j // parts for j in range(parts + 1)]
        firsts = []
        for a, b in zip(bounds[:-1], bounds[1:]):
            idx = torch.nonzero((key >= a) & (key < b)).squeeze(1)
            skey, order = torch.sort(key[idx], stable=True)
            first = torch.ones_like(skey, dtype=torch.bool)
            first[1:] = skey[1:] != skey[:-1]
            firsts.append(idx[order[first]])
            del idx, skey, order, first
        pos = torch.sort(torch.cat(firsts)).values
        del firsts
        if pos.numel() >= m:
            pos = pos[:m]
            keys = key[pos]
            return keys // n, keys % n, pos
        count = int(count * 1.6) + 1024


def relabel(n: int, seed: int, device) -> torch.Tensor:
    """A seeded random permutation new_id[old_id] of [0, n) (Graph500 practice)."""
    h = stream_hash(seed * 64 + 2, torch.arange(n, dtype=torch.int64, device=device))
    order = torch.sort(h, stable=True).indices
    new_id = torch.empty(n, dtype=torch.int64, device=device)
    new_id[order] = torch.arange(n, dtype=torch.int64, device=device)
    return new_id


@dataclass
class CSRGraph:
    """Sorted CSR: offsets int64[n+1], dsts int32[nnz], optional fp32 weights."""
    offsets: torch.Tensor
    dsts: torch.Tensor
    weights: torch.Tensor | None
    num_nodes: int
    name: str = ""

    @property
    def num_entries(self) -> int:
        return int(self.dsts.numel())

    def to(self, device) -> "CSRGraph":
        return CSRGraph(self.offsets.to(device), self.dsts.to(device),
                        None if self.weights is None else self.weights.to(device),
                        self.num_nodes, self.name)

    def numpy(self):
        return (self.offsets.cpu().numpy(), self.dsts.cpu().numpy(),
                None if self.weights is None else self.weights.cpu().numpy())

    def degrees(self) -> torch.Tensor:
        return self.offsets[1:] - self.offsets[:-1]


def symmetric_csr(n: int, u: torch.Tensor, v: torch.Tensor, w: torch.Tensor | None,
                  name: str = "") -> CSRGraph:
    """CSR holding both directions of every undirected pair, rows sorted.

    Rows are built in parts of consecutive node ranges, each sorted on its own,
    so that no single sort exceeds torch's 2^31 - 1 element limit."""
    dev = u.device
    counts = torch.bincount(u, minlength=n) + torch.bincount(v, minlength=n)
    offsets = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    offsets[1:] = torch.cumsum(counts, 0)
    del counts
    m2 = 2 * u.numel()
    dsts = torch.empty(m2, dtype=torch.int32, device=dev)
    ww = None if w is None else torch.empty(m2, dtype=torch.float32, device=dev)
    parts = 1
    while m2 // parts > (1 << 29):
        parts *= 2
    bounds = [n * j // parts for j in range(parts + 1)]
    for lo, hi in zip(bounds[:-1], bounds[1:]):
        sa = (u >= lo) & (u < hi)
        sb = (v >= lo) & (v < hi)
        src = torch.cat([u[sa], v[sb]])
        dst = torch.cat([v[sa], u[sb]])
        wp = None if w is None else torch.cat([w[sa], w[sb]])
        del sa, sb
        if src.numel() >= (1 << 31) - 1:
            raise RuntimeError("graph part too large for one sort")
        key = (src - lo) * n + dst
        del src
        key, order = torch.sort(key)
        a, b = int(offsets[lo]), int(offsets[hi])
        dsts[a:b] = (key % n).to(torch.int32)
        if ww is not None:
            ww[a:b] = wp[order]
        del key, order, dst, wp
    return CSRGraph(offsets, dsts, ww, n, name)


def pair_weights(seed: int, pos: torch.Tensor) -> torch.Tensor:
    """fp32 weights uniform in [0.1, 1.0] per undirected pair (keyed by the pair's
    index in the candidate stream, so symmetric by construction)."""
    h = stream_hash(seed * 64 + 3, pos)
    u = _lsr(h, 11).to(torch.float64) * (2.0 ** -53)
    return (0.1 + 0.9 * u).to(torch.float32)


def erdos_renyi(n: int, m: int, seed: int, weighted: bool = False, device="cpu") -> CSRGraph:
    """G(n, m): m distinct unordered non-loop pairs, stored in both directions."""
    u, v, pos = first_unique_undirected(
        lambda b, c: uniform_pairs(n, seed, b, c, device), n, m, device)
    w = pair_weights(seed, pos) if weighted else None
    return symmetric_csr(n, u, v, w, name=f"er_n{n}_m{m}_s{seed}")


def rmat(scale: int, m: int, seed: int, weighted: bool = False, a=0.57, b=0.19, c=0.19,
         device="cpu", relabel_nodes: bool = True) -> CSRGraph:
    """R-MAT graph with 2^scale nodes and m distinct undirected non-loop edges
    (stored both directions), node ids randomly relabelled."""
    n = 1 << scale
    u, v, pos = first_unique_undirected(
        lambda bb, cc: rmat_pairs(scale, a, b, c, seed, bb, cc, device), n, m, device)
    if relabel_nodes:
        perm = relabel(n, seed, device)
        u, v = perm[u], perm[v]
        del perm
    w = pair_weights(seed, pos) if weighted else None
    del pos
    return symmetric_csr(n, u, v, w, name=f"rmat_s{scale}_m{m}_seed{seed}")


# --------------------------------------------------------------------------
# The benchmark workloads (graph + walk job)
# --------------------------------------------------------------------------

@dataclass
class WalkJob:
    walk_len: int
    walks_per_node: int
    p: float
    q: float
    seed: int


WORKLOADS = {
    # Erdos-Renyi, 1,000 nodes, 10,000 undirected edges, unweighted.
    "er1k": dict(kind="er", n=1000, m=10_000, seed=1, weighted=False,
                 job=WalkJob(32, 1, 2.0, 0.5, 42)),
    # R-MAT scale 20, 16M undirected edges, fp32 weights U[0.1, 1].
    "rmat20w": dict(kind="rmat", scale=20, m=1 << 24, seed=2, weighted=True,
                    job=WalkJob(100, 10, 0.5, 2.0, 7)),
    # R-MAT scale 24, 256M undirected edges, unweighted, hub-heavy.
    "rmat24": dict(kind="rmat", scale=24, m=1 << 28, seed=3, weighted=False,
                   job=WalkJob(80, 10, 1.0, 0.25, 11)),
    # R-MAT scale 22, 64M undirected edges, unweighted: the scale-24 job on a
    # graph of a sixteenth of the size (about 6 GB on device with its rows).
    "rmat22": dict(kind="rmat", scale=22, m=1 << 26, seed=3, weighted=False,
                   job=WalkJob(80, 1, 1.0, 0.25, 11)),
    # R-MAT scale 21, 32M undirected edges, unweighted: the scale-24 job's
    # kernel at a size a full profiler capture holds (about 3 GB on device).
    "rmat21": dict(kind="rmat", scale=21, m=1 << 25, seed=3, weighted=False,
                   job=WalkJob(80, 1, 1.0, 0.25, 11)),
    # R-MAT scale 26, 1B undirected edges, unweighted: the serving graph, and a
    # walk job of the scale-24 kind with one walk per node.
    "rmat26": dict(kind="rmat", scale=26, m=1 << 30, seed=5, weighted=False,
                   job=WalkJob(80, 1, 1.0, 0.25, 13)),
}


def workload_graph(name: str, device="cpu") -> CSRGraph:
    spec = WORKLOADS[name]
    if spec["kind"] == "er":
        return erdos_renyi(spec["n"], spec["m"], spec["seed"], spec["weighted"], device)
    return rmat(spec["scale"], spec["m"], spec["seed"], spec["weighted"], device=device)


PQ_CHOICES = (0.25, 0.5, 1.0, 2.0, 4.0)


@dataclass
class Request:
    starts: np.ndarray      # int32 start node ids
    walk_len: int
    p: float
    q: float
    seed: int


def request_mix(num_nodes: int, count: int, gen_seed: int, max_starts: int,
                len_lo: int, len_hi: int, first_seed: int = 0) -> list[Request]:
    """Walk requests of uneven size: start count round(exp(U[0, ln max_starts])) >= 1
    (log-uniform), start ids uniform with replacement, length uniform in
    [len_lo, len_hi], p and q drawn from {0.25, 0.5, 1, 2, 4}, seeds
    first_seed, first_seed + 1, ..."""
    idx = torch.arange(count, dtype=torch.int64)
    h = stream_hash(gen_seed * 64 + 10, idx)
    u = _lsr(h, 11).to(torch.float64) * (2.0 ** -53)
    sizes = torch.clamp(torch.round(torch.exp(u * math.log(max_starts))), min=1).to(torch.int64)
    h2 = stream_hash(gen_seed * 64 + 11, idx)
    lens = len_lo + (_u32_hi(h2) * (len_hi - len_lo + 1) >> 32)
    pi = (_u32_lo(h2) * len(PQ_CHOICES)) >> 32
    h3 = stream_hash(gen_seed * 64 + 12, idx)
    qi = (_u32_hi(h3) * len(PQ_CHOICES)) >> 32
    total = int(sizes.sum())
    hs = stream_hash(gen_seed * 64 + 13, torch.arange(total, dtype=torch.int64))
    all_starts = ((_u32_hi(hs) * num_nodes) >> 32).to(torch.int32).numpy()
    out, pos = [], 0
    for j in range(count):
        s = int(sizes[j])
        out.append(Request(all_starts[pos:pos + s].copy(), int(lens[j]),
                           PQ_CHOICES[int(pi[j])], PQ_CHOICES[int(qi[j])], first_seed + j))
        pos += s
    return out


def poisson_arrivals(rate_per_s: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process: exponential gaps."""
    h = stream_hash(seed * 64 + 20, torch.arange(count, dtype=torch.int64))
    u = (_lsr(h, 11).to(torch.float64) + 0.5) * (2.0 ** -53)
    gaps = -torch.log(u) / rate_per_s
    return torch.cumsum(gaps, 0).numpy()
