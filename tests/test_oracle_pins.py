"""Pins of the CPU oracle against facts fixed outside it (CPU only).

* Philox4x32-10 against the published known-answer vectors.
* The sampler against the exact transition law computed from graph distances
  (GRAPE, Methods, eq. alphaRW), by chi-square over every (t, v) context of tiny
  graphs, for a grid of (p, q), weighted and unweighted, directed and undirected.
* The trial-cap fallback (the paper's cumulative-sum sampler, "Efficient sampling
  for Node2Vec RWs") against the same law.
* Closed forms: P(return) = q/(p+q) inside a cycle, (1/p)/(1/p + n-2) on K_n,
  and the star.
* Stationarity of p = q = 1 walks (degree- or strength-proportional).
* Invariants: every step follows an edge, -1 only as a suffix after a dead end.
"""
import math
import os

import numpy as np
import pytest

import oracle
import _law

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        vals = [int(x, 16) for x in r]
        ctr, key, want = vals[0:4], vals[4:6], vals[6:10]
        got = oracle.philox4x32_10(ctr, key)
        assert [int(x) for x in got] == want


@pytest.mark.parametrize("p,q", [(2.0, 0.5), (0.5, 2.0), (1.0, 0.25), (0.25, 4.0),
                                 (1.0, 1.0), (4.0, 4.0)])
def test_thresholds_powers_of_two(p, q):
    # alpha / max(alpha) is an exact binary fraction here, so T = ratio * 2^32 exactly.
    alphas = [1.0 / p, 1.0, 1.0 / q]
    amax = max(alphas)
    want = tuple(int(a / amax * 2**32) for a in alphas)
    assert oracle.thresholds(p, q) == want


def test_thresholds_general_are_floor_of_ratio():
    for p, q in [(3.0, 0.7), (0.3, 1.9), (1.7, 1.0)]:
        T = oracle.thresholds(p, q)
        alphas = [1.0 / p, 1.0, 1.0 / q]
        amax = max(alphas)
        for t, a in zip(T, alphas):
            assert abs(t - a / amax * 2**32) <= 1.0
            assert t <= 2**32


def _law_pvalues(g, pq_grid, n_draws, trial_cap=oracle.DEFAULT_TRIAL_CAP, step=2):
    pvals = []
    for (p, q) in pq_grid:
        for (t, v) in _law.contexts(g.offsets, g.dsts):
            s = step if t >= 0 else 1
            draws = oracle.next_many(g, t, v, p, q, seed=12345, walk_begin=1000 * v,
                                     n=n_draws, step=s, trial_cap=trial_cap)
            row = g.dsts[g.offsets[v]:g.offsets[v + 1]]
            probs = _law.exact_law(g.offsets, g.dsts, g.weights, t, v, p, q)
            pvals.append(_law.chi2_pvalue(draws, row, probs))
    return np.array(pvals)


def _house(weighted):
    n, edges = _law.graph_house()
    w = None
    if weighted:
        w = [0.1 + 0.9 * ((7 * k + 3) % 11) / 10 for k in range(len(edges))]
    return oracle.Graph(*_law.csr_from_edges(n, edges, w, undirected=True))


def _directed(weighted):
    n, edges = _law.graph_directed()
    w = None if not weighted else [0.2 + 0.15 * (k % 6) for k in range(len(edges))]
    return oracle.Graph(*_law.csr_from_edges(n, edges, w, undirected=False))


@pytest.mark.parametrize("make", [_house, _directed], ids=["undirected", "directed"])
@pytest.mark.parametrize("weighted", [False, True], ids=["unweighted", "weighted"])
def test_transition_law_chi_square(make, weighted):
    g = make(weighted)
    pv = _law_pvalues(g, _law.PQ_GRID, n_draws=20000)
    # Deterministic seeds: every p-value is a fixed number.  Hundreds of contexts
    # pass with a large margin; a wrong law drives p to ~0 with 20k draws.
    assert pv.min() > 1e-6, pv.min()
    # Under the true law p-values are spread over (0, 1).
    assert np.median(pv) > 0.1


@pytest.mark.parametrize("cap", [0, 1, 3])
def test_fallback_matches_law(cap):
    # cap = 0: every step is drawn by the cumulative-sum fallback; small caps mix.
    for weighted in (False, True):
        for g in (_house(weighted), _directed(weighted)):
            pv = _law_pvalues(g, [(0.25, 4.0), (2.0, 0.5), (1.0, 1.0)], 8000, trial_cap=cap)
            assert pv.min() > 1e-6


def _returns(rows):
    """Fraction of transitions s >= 2 with x_s == x_{s-2}."""
    a, c = rows[:, 2:], rows[:, :-2]
    valid = (a >= 0) & (c >= 0)
    return (a == c)[valid].mean(), valid.sum()


@pytest.mark.parametrize("p,q", [(2.0, 0.5), (0.5, 2.0), (1.0, 0.25), (4.0, 1.0)])
def test_cycle_return_probability(p, q):
    n = 9
    edges = [(i, (i + 1) % n) for i in range(n)]
    g = oracle.Graph(*_law.csr_from_edges(n, edges))
    rows, rc = oracle.walks(g, None, 40, 300, p, q, seed=5)
    assert rc == 0
    f, cnt = _returns(rows)
    want = q / (p + q)
    assert abs(f - want) < 5 * math.sqrt(want * (1 - want) / cnt), (f, want)


@pytest.mark.parametrize("p,q", [(2.0, 0.5), (0.25, 4.0), (1.0, 1.0)])
def test_complete_graph_return_probability(p, q):
    n = 7
    edges = [(i, j) for i in range(n) for j in range(i + 1, n)]
    g = oracle.Graph(*_law.csr_from_edges(n, edges))
    rows, _ = oracle.walks(g, None, 40, 400, p, q, seed=9)
    f, cnt = _returns(rows)
    want = (1 / p) / (1 / p + n - 2)
    assert abs(f - want) < 5 * math.sqrt(want * (1 - want) / cnt), (f, want)


def test_star():
    leaves = 6
    edges = [(0, i) for i in range(1, leaves + 1)]
    g = oracle.Graph(*_law.csr_from_edges(leaves + 1, edges))
    p, q = 0.5, 2.0
    rows, _ = oracle.walks(g, list(range(1, leaves + 1)), 21, 500, p, q, seed=3)
    # Leaf -> centre is forced: odd positions are the centre.
    assert (rows[:, 1::2] == 0).all()
    # Out of the centre (odd positions) the walk returns to the leaf it came from
    # (d = 0) or goes to one of the other leaves - 1 leaves (d = 2).
    a, c = rows[:, 2::2], rows[:, 0:-2:2]
    f, cnt = (a == c).mean(), a.size
    want = (1 / p) / (1 / p + (leaves - 1) / q)
    assert abs(f - want) < 5 * math.sqrt(want * (1 - want) / cnt), (f, want)


def _ring_with_chords(n, chords, seed):
    rng = np.random.default_rng(seed)
    edges = {(i, (i + 1) % n) for i in range(n)}
    while len(edges) < n + chords:
        a, b = rng.integers(0, n, 2)
        if a != b and (a, b) not in edges and (b, a) not in edges:
            edges.add((int(a), int(b)))
    return sorted(edges)


@pytest.mark.parametrize("weighted", [False, True])
def test_stationary_distribution_first_order(weighted):
    n = 40
    edges = _ring_with_chords(n, 50, seed=1)
    w = [0.1 + 0.9 * ((13 * k) % 17) / 16 for k in range(len(edges))] if weighted else None
    off, dst, ww = _law.csr_from_edges(n, edges, w)
    g = oracle.Graph(off, dst, ww)
    rows, _ = oracle.walks(g, None, 61, 2500, 1.0, 1.0, seed=77)
    last = rows[:, -1]
    strength = np.array([(ww[off[v]:off[v + 1]].astype(np.float64).sum() if weighted
                          else off[v + 1] - off[v]) for v in range(n)])
    probs = strength / strength.sum()
    assert _law.chi2_pvalue(last, np.arange(n), probs) > 1e-4


def _assert_invariants(g, starts, rows, num_starts):
    off, dst = g.offsets, g.dsts
    for w, row in enumerate(rows):
        i = w % num_starts
        v0 = i if starts is None else starts[i]
        assert row[0] == v0
        valid = row >= 0
        k = int(valid.sum())
        assert valid[:k].all() and not valid[k:].any(), "-1 only as a suffix"
        for s in range(1, k):
            a, b = row[s - 1], row[s]
            assert b in dst[off[a]:off[a + 1]], "every step follows an edge"
        if k < len(row):
            last = row[k - 1]
            assert off[last + 1] == off[last], "padding only after a dead end"


def test_invariants_er_and_directed():
    from paper_2110_06196_gb300 import synth
    cg = synth.erdos_renyi(300, 600, seed=4)
    g = oracle.Graph(*cg.numpy())
    rows, _ = oracle.walks(g, None, 30, 2, 2.0, 0.5, seed=42)
    _assert_invariants(g, None, rows, 300)
    gd = _directed(True)
    starts = [0, 1, 2, 3, 4, 5, 5]
    rows, _ = oracle.walks(gd, starts, 25, 30, 0.5, 2.0, seed=8)
    _assert_invariants(gd, starts, rows, len(starts))
    assert (rows[:, -1] == -1).any(), "node 5 is a dead end and is reached"


def test_bad_start_rows_are_minus_one():
    g = _house(False)
    rows, rc = oracle.walks(g, [0, 99, -1, 3], 6, 1, 1.0, 1.0, seed=1)
    assert rc == -1
    assert (rows[1] == -1).all() and (rows[2] == -1).all()
    assert rows[0, 0] == 0 and rows[3, 0] == 3


def test_parallel_equals_serial():
    from paper_2110_06196_gb300 import synth
    cg = synth.erdos_renyi(500, 2000, seed=6, weighted=True)
    g = oracle.Graph(*cg.numpy())
    a, _ = oracle.walks(g, None, 20, 3, 0.5, 2.0, seed=3)
    b = oracle.walks_parallel(g, None, 20, 3, 0.5, 2.0, seed=3, threads=4)
    assert np.array_equal(a, b)


def test_weighted_rule_is_exact_rational_comparison():
    # Pinned against Python's exact rationals: r2 * wmax < T * w over the reals.
    from fractions import Fraction
    rng = np.random.default_rng(11)
    f32 = np.float32
    cases = []
    for _ in range(20000):
        w1 = f32(rng.uniform(0.1, 1.0))
        w2 = f32(w1 * f32(rng.uniform(0.05, 1.0)))
        cases.append((int(rng.integers(0, 2**32)), w1, int(rng.integers(1, 2**32 + 1)), w2))
    # ties, zero r2, subnormal and far-apart exponents
    tiny = np.frombuffer(np.uint32(5).tobytes(), np.float32)[0]
    cases += [(2**31, f32(1.0), 2**31, f32(1.0)), (2**31 - 1, f32(1.0), 2**31, f32(1.0)),
              (0, f32(1.0), 1, tiny), (1, f32(1.0), 2**32, tiny), (3, f32(0.75), 2, f32(0.5)),
              (2, f32(0.75), 3, f32(0.5)), (1, f32(3e38), 2**32, f32(1e-30)),
              (2**32 - 1, tiny, 2**32, tiny), (2**32 - 1, f32(2.0) * tiny, 2**32, tiny)]
    for r2, wmax, T, w in cases:
        want = Fraction(r2) * Fraction(float(wmax)) < Fraction(T) * Fraction(float(w))
        assert oracle.weighted_accept(r2, wmax, T, w) == want, (r2, wmax, T, w)
