"""The oracle's approximated walks (GRAPE, Methods, "Approximated RWs": SUSS,
Sorted Unique Sub-Sampling) pinned to things other than itself: the structure
of a sub-sample (one position per bucket, sorted, unique, inside its bucket),
the uniformity test the paper runs on SUSS, the exact transition law of the
approximated step computed by enumerating every sub-sample, and identity with
the exact walk when k >= deg.  Planted mistakes in a copy of the source fail
them."""
import itertools
import os

import numpy as np
import pytest
from scipy import stats as sst

import oracle
import _law

SRC = os.path.join(os.path.dirname(oracle.__file__), "walk_oracle.c")


def bucket_bounds(deg, k):
    return [((b * deg) // k, ((b + 1) * deg) // k) for b in range(k)]


def hub_graph(weighted):
    # node 0 has degree 7; 1 - 2 - 4 and 1 - 3 make the classes of x vary with t
    edges = [(0, x) for x in range(1, 8)] + [(1, 2), (1, 3), (2, 4), (5, 6)]
    w = [0.15 + 0.1 * k for k in range(len(edges))] if weighted else None
    return oracle.Graph(*_law.csr_from_edges(8, edges, w, True))


def suss_law(g, t, v, p, q, k):
    """Exact law of the approximated step: average, over every sub-sample, of
    the exact law restricted to the sub-sample."""
    lo, hi = g.offsets[v], g.offsets[v + 1]
    deg = int(hi - lo)
    full = _law.exact_law(g.offsets, g.dsts, g.weights, t, v, p, q)
    law = np.zeros(deg)
    buckets = [range(a, b) for a, b in bucket_bounds(deg, k)]
    for sub in itertools.product(*buckets):
        prob = np.prod([1.0 / len(b) for b in buckets])
        idx = np.array(sub)
        law[idx] += prob * full[idx] / full[idx].sum()
    return law


def pin_battery(lib):
    failed = []
    # structure of sub-samples
    rng = np.random.default_rng(0)
    for _ in range(300):
        deg = int(rng.integers(2, 5000))
        k = int(rng.integers(1, deg + 3))
        pos = oracle.suss_positions(deg, k, int(rng.integers(0, 2**63)), int(rng.integers(0, 10**9)),
                                    int(rng.integers(1, 100)), lib=lib)
        if k >= deg:
            ok = np.array_equal(pos, np.arange(deg))
        else:
            b = np.array(bucket_bounds(deg, k))
            ok = (len(pos) == k and np.all(np.diff(pos) > 0) and np.all(pos >= b[:, 0])
                  and np.all(pos < b[:, 1]))
        if not ok:
            failed.append("structure")
            break
    # the paper's uniformity check of SUSS: positions of [0, 10000) drawn with k = 100
    pos = np.concatenate([oracle.suss_positions(10000, 100, 77, w, 3, lib=lib)
                          for w in range(3000)])
    if pos.min() < 0 or pos.max() >= 10000 or \
            sst.chisquare(np.bincount(pos, minlength=10000)).pvalue < 1e-6:
        failed.append("uniformity")
    # exact law of the approximated step, by enumeration of sub-samples
    for weighted in (False, True):
        g = hub_graph(weighted)
        g.lib = lib
        row = g.dsts[g.offsets[0]:g.offsets[1]]
        for (t, p, q, k) in [(1, 0.5, 2.0, 3), (4, 2.0, 0.5, 3), (-1, 1.0, 1.0, 3), (1, 4.0, 0.25, 2)]:
            for cap in (oracle.DEFAULT_TRIAL_CAP, 0):
                d = oracle.next_many(g, t, 0, p, q, 5, 0, 30000, 2 if t >= 0 else 1, cap,
                                     suss_k=k)
                if _law.chi2_pvalue(d, row, suss_law(g, t, 0, p, q, k)) < 1e-6:
                    failed.append(f"law(w={weighted},t={t},k={k},cap={cap})")
    # k >= deg: the exact walk
    n, e = _law.graph_house()
    g = oracle.Graph(*_law.csr_from_edges(n, e, None, True), lib=lib)
    a, _ = oracle.walks(g, None, 20, 5, 0.5, 2.0, seed=9)
    b, _ = oracle.walks(g, None, 20, 5, 0.5, 2.0, seed=9, suss_k=16)
    if not np.array_equal(a, b):
        failed.append("k>=deg")
    return sorted(set(failed))


def test_oracle_suss_passes_its_pins():
    assert pin_battery(oracle.load()) == []


PLANTS = {
    "bucket_overlap": ("uint64_t hi = (uint64_t)(((unsigned __int128)(j + 1) * deg) / k);",
                       "uint64_t hi = (uint64_t)(((unsigned __int128)(j + 1) * deg) / k) + 1;"),
    "proposal_ignores_subsample": ("uint64_t idx = cand_pos(deg, suss_k, seed, walk_id, step, j);",
                                   "uint64_t idx = (uint64_t)(((unsigned __int128)r64 * deg) >> 64);"),
    "bucket_start_shifted": ("uint64_t lo = (uint64_t)(((unsigned __int128)j * deg) / k);",
                             "uint64_t lo = (uint64_t)(((unsigned __int128)j * deg) / k) + (j > 0);"),
}


@pytest.mark.parametrize("name", sorted(PLANTS))
def test_planted_suss_mistake_is_caught(name, tmp_path):
    old, new = PLANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    mutated = tmp_path / "walk_oracle_planted.c"
    mutated.write_text(src.replace(old, new))
    so = oracle.compile_oracle(str(mutated), str(tmp_path / "liboracle_planted.so"))
    assert pin_battery(oracle.load(so)), f"planted mistake {name} escaped every pin"
