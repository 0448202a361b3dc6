"""Fuzzing of the library's input checks on the device (graph validation, walk
arguments), seeded.  Every case is decided first by a host predicate written
here from the header's contract; the library must agree case by case:

* random small CSRs, valid or corrupted in one way (offsets out of order or
  off the ends, ids out of range, rows unsorted or with a repeated id, weights
  zero, negative, NaN or infinite, a missing or unequal reverse entry) are
  accepted by grape_graph_create (with GRAPE_VALIDATE) and grape_ef_graph_create
  exactly when the predicate says they are valid;
* random walk arguments (start counts, lengths, walks per node, p and q among
  zero, negative, NaN, infinite, huge and tiny values) are refused with
  GRAPE_ERR_INVALID_ARG exactly when the predicate refuses them, and otherwise
  produce the oracle's rows.

Validation runs before anything is built from the CSR, so corrupted inputs are
never read out of bounds.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2110_06196_gb300 import EFGraph, Graph, GrapeError, synth, walks

pytestmark = pytest.mark.gpu


def valid_csr(off, dst, w, n, undirected):
    off = np.asarray(off, np.int64)
    dst = np.asarray(dst, np.int64)
    m = len(dst)
    if len(off) != n + 1 or off[0] != 0 or off[-1] != m or np.any(np.diff(off) < 0):
        return False
    if m and (dst.min() < 0 or dst.max() >= n):
        return False
    for a in range(n):
        row = dst[off[a]:off[a + 1]]
        if len(row) > 1 and np.any(np.diff(row) <= 0):
            return False
    if w is not None:
        w = np.asarray(w, np.float32)
        if not np.all(np.isfinite(w)) or np.any(w <= 0):
            return False
    if undirected:
        ent = {}
        for a in range(n):
            for e in range(off[a], off[a + 1]):
                ent[(a, int(dst[e]))] = None if w is None else float(w[e])
        for (a, b), wt in ent.items():
            if (b, a) not in ent or ent[(b, a)] != wt:
                return False
    return True


def random_case(rng):
    n = int(rng.integers(2, 12))
    m_pairs = min(int(rng.integers(0, 12)), n * (n - 1) // 2)
    csr = synth.erdos_renyi(n, m_pairs, seed=int(rng.integers(1 << 30)),
                            weighted=bool(rng.integers(2)))
    off, dst, w = csr.numpy()
    n = csr.num_nodes
    off, dst = off.copy(), dst.astype(np.int64).copy()
    w = None if w is None else w.copy()
    undirected = bool(rng.integers(2))
    kind = int(rng.integers(0, 9))
    m = len(dst)
    if kind == 1 and n > 1:                           # offsets out of order
        a = int(rng.integers(1, n))
        off[a] = off[-1] + 1 if rng.integers(2) else -1
    elif kind == 2:                                   # last offset wrong
        off[-1] = m + 1
    elif kind == 3 and m:                             # id out of range
        dst[int(rng.integers(m))] = n if rng.integers(2) else -1
    elif kind == 4 and m:                             # repeated id / unsorted row
        rows = [a for a in range(n) if off[a + 1] - off[a] >= 2]
        if rows:
            a = rows[int(rng.integers(len(rows)))]
            dst[off[a] + 1] = dst[off[a]] if rng.integers(2) else dst[off[a]] - 1
    elif kind == 5 and m and w is not None:           # bad weight
        w[int(rng.integers(m))] = [0.0, -1.0, np.nan, np.inf][int(rng.integers(4))]
    elif kind == 6 and m:                             # drop the last entry (asymmetric)
        a = int(np.searchsorted(off, m - 1, side="right") - 1)
        dst = dst[:-1]
        off[a + 1:] = np.minimum(off[a + 1:], m - 1)
        if w is not None:
            w = w[:-1]
    elif kind == 7 and m and w is not None:           # unequal reverse weight
        w[int(rng.integers(m))] *= 1.5
    return off, dst, w, n, undirected


def _tensors(off, dst, w):
    return (torch.from_numpy(np.asarray(off, np.int64)),
            torch.from_numpy(np.asarray(dst, np.int64).astype(np.int32)),
            None if w is None else torch.from_numpy(np.asarray(w, np.float32)))


def test_graph_validation_agrees_with_the_contract():
    rng = np.random.default_rng(2024)
    seen = {True: 0, False: 0}
    for case in range(240):
        off, dst, w, n, und = random_case(rng)
        ok = valid_csr(off, dst, w, n, und)
        seen[ok] += 1
        o, d, wt = _tensors(off, dst, w)
        for make in (lambda: Graph(o, d, wt, undirected=und, validate=True),
                     lambda: EFGraph(o, d, wt, quantum=int(2 ** rng.integers(0, 7)),
                                     undirected=und, validate=True)):
            try:
                g = make()
                accepted = True
                g.close()
            except GrapeError as e:
                assert e.name == "GRAPE_ERR_INVALID_GRAPH", (case, e.name)
                accepted = False
            assert accepted == ok, (case, ok, off.tolist(), dst.tolist(), w, und)
    assert seen[True] > 30 and seen[False] > 30


PQ = [0.0, -1.0, math.nan, math.inf, 1e-300, 1e300, 2.0 ** -33, 2.0 ** 31, 0.25, 1.0, 3.0]
GOOD = [0.25, 0.5, 1.0, 2.0, 4.0, 3.0, 0.7]


def valid_walk_args(num_starts, walk_len, wpn, p, q, n):
    def pq_ok(x):
        if not (math.isfinite(x) and x > 0):
            return False
        a = [1.0 / p, 1.0, 1.0 / q] if all(math.isfinite(v) and v > 0 for v in (p, q)) else None
        return a is not None and all(math.floor(c / max(a) * 2.0 ** 32) >= 1 for c in a)
    return (num_starts >= 1 and num_starts <= n and walk_len >= 1 and wpn >= 1
            and pq_ok(p) and pq_ok(q))


def test_walk_arguments_agree_with_the_contract():
    csr = synth.erdos_renyi(40, 120, seed=77)
    g = Graph.from_csr(csr)
    og = oracle.Graph(*csr.numpy())
    rng = np.random.default_rng(7)
    accepted = refused = 0
    for case in range(200):
        ns = int(rng.choice([-1, 0, 1, 7, 40, 40, 41]))
        L = int(rng.choice([-2, 0, 1, 2, 9, 9]))
        wpn = int(rng.choice([-1, 0, 1, 3, 3]))
        p = float(PQ[int(rng.integers(len(PQ)))]) if rng.integers(3) == 0 else float(rng.choice(GOOD))
        q = float(PQ[int(rng.integers(len(PQ)))]) if rng.integers(3) == 0 else float(rng.choice(GOOD))
        ok = valid_walk_args(ns, L, wpn, p, q, csr.num_nodes)
        out = torch.empty((max(ns, 1) * max(wpn, 1), max(L, 1)), dtype=torch.int32, device="cuda")
        try:
            walks(g, None, L, wpn, p, q, seed=case, num_starts=ns, out=out)
            torch.cuda.synchronize()
            got = True
        except GrapeError as e:
            assert e.name == "GRAPE_ERR_INVALID_ARG", (case, e.name)
            got = False
        assert got == ok, (case, ns, L, wpn, p, q)
        if ok:
            accepted += 1
            want, rc = oracle.walks(og, np.arange(ns, dtype=np.int32), L, wpn, p, q, case)
            assert rc == 0 and np.array_equal(out.cpu().numpy(), want), case
        else:
            refused += 1
    assert accepted > 10 and refused > 50
