"""Exact node2vec transition law on tiny graphs, computed from graph distances.

This is the pin for the oracle's sampler.  It uses the distance form of the bias
(GRAPE, Methods, eq. alphaRW): alpha = 1/p if d(t,x) = 0, 1 if d(t,x) = 1 and
1/q if d(t,x) = 2, with d the directed shortest-path length from a breadth-first
search.  It does not use the membership form x in N(t) that the oracle and the
kernels evaluate.  The first step is first-order: pi_vx = w_vx.
"""
from __future__ import annotations

from collections import deque

import numpy as np
from scipy import stats as sst


def csr_from_edges(n, edges, weights=None, undirected=True):
    """Sorted CSR from an edge list (both directions when undirected)."""
    pairs = {}
    for k, (a, b) in enumerate(edges):
        w = 1.0 if weights is None else weights[k]
        pairs[(a, b)] = w
        if undirected and a != b:
            pairs[(b, a)] = w
    rows = [[] for _ in range(n)]
    for (a, b), w in pairs.items():
        rows[a].append((b, w))
    offsets = [0]
    dsts, ws = [], []
    for r in rows:
        r.sort()
        dsts += [b for b, _ in r]
        ws += [w for _, w in r]
        offsets.append(len(dsts))
    return (np.array(offsets, np.int64), np.array(dsts, np.int32),
            None if weights is None else np.array(ws, np.float32))


def bfs_dist(offsets, dsts, src):
    n = len(offsets) - 1
    d = np.full(n, -1, np.int64)
    d[src] = 0
    dq = deque([src])
    while dq:
        a = dq.popleft()
        for e in range(offsets[a], offsets[a + 1]):
            b = dsts[e]
            if d[b] < 0:
                d[b] = d[a] + 1
                dq.append(b)
    return d


def exact_law(offsets, dsts, weights, t, v, p, q):
    """Normalised transition probabilities over the row of v (row order)."""
    lo, hi = offsets[v], offsets[v + 1]
    w = np.ones(hi - lo) if weights is None else weights[lo:hi].astype(np.float64)
    if t < 0:
        pi = w
    else:
        d = bfs_dist(offsets, dsts, t)
        alpha = []
        for x in dsts[lo:hi]:
            dx = d[x]
            assert dx in (0, 1, 2), "a neighbour of v is within two hops of t"
            alpha.append({0: 1.0 / p, 1: 1.0, 2: 1.0 / q}[int(dx)])
        pi = np.array(alpha) * w
    return pi / pi.sum()


def chi2_pvalue(samples, row, probs):
    """Chi-square goodness of fit of node samples against probabilities over row."""
    pos = {int(x): j for j, x in enumerate(row)}
    counts = np.zeros(len(row))
    for x, c in zip(*np.unique(samples, return_counts=True)):
        if int(x) not in pos:
            return 0.0          # a draw outside the row is an outright failure
        counts[pos[int(x)]] = c
    expected = probs * len(samples)
    keep = expected > 0
    if (counts[~keep] > 0).any():
        return 0.0
    if keep.sum() < 2:
        return 1.0
    return float(sst.chisquare(counts[keep], expected[keep]).pvalue)


# Tiny test graphs ---------------------------------------------------------------

def graph_house():
    """Undirected: a square 0-1-2-3 with roof 4 on 2-3, a chord 1-3, a tail 4-5-6,
    a pendant 7 on 0 and a self-loop on 5."""
    edges = [(0, 1), (1, 2), (2, 3), (3, 0), (1, 3), (2, 4), (3, 4), (4, 5), (5, 6),
             (0, 7), (5, 5)]
    return 8, edges


def graph_directed():
    """Directed, with a dead end at node 5 and a 2-cycle 0<->1."""
    edges = [(0, 1), (1, 0), (1, 2), (1, 3), (2, 3), (3, 0), (3, 4), (2, 4), (4, 1),
             (4, 5), (0, 2)]
    return 6, edges


def contexts(offsets, dsts):
    """Every (t, v) with an edge t -> v and deg(v) > 0, plus (-1, v) first steps."""
    n = len(offsets) - 1
    out = []
    for v in range(n):
        if offsets[v + 1] == offsets[v]:
            continue
        out.append((-1, v))
    for t in range(n):
        for e in range(offsets[t], offsets[t + 1]):
            v = int(dsts[e])
            if offsets[v + 1] > offsets[v]:
                out.append((t, v))
    return out


PQ_GRID = [(0.25, 4.0), (4.0, 0.25), (2.0, 0.5), (0.5, 2.0), (1.0, 1.0), (1.0, 0.25),
           (4.0, 1.0), (0.25, 0.25)]
