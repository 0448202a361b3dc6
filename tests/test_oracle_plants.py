"""The oracle's pins have teeth: each plausible mistake, planted in a copy of
the oracle source and compiled on the CPU, fails at least one pin.

Mistakes: p and q swapped; the return test dropped (open neighbourhood); the
range reduction one short; the weight left out of the acceptance test; the
membership operands transposed; alpha left out of the fallback; the previous node
updated after the current one; the wrong start index; acceptance inverted; the
weighted test accepting ties or shifting the wrong way.
"""
import os

import numpy as np
import pytest

import oracle
import _law

SRC = os.path.join(os.path.dirname(oracle.__file__), "walk_oracle.c")

PLANTS = {
    "swap_p_q": ("double a_ret = 1.0 / p, a_in = 1.0, a_out = 1.0 / q;",
                 "double a_ret = 1.0 / q, a_in = 1.0, a_out = 1.0 / p;"),
    "open_neighbourhood": ("    if (x == t) return CLS_RETURN;\n", ""),
    "range_one_short": ("(((unsigned __int128)r64 * m) >> 64)", "(((unsigned __int128)r64 * (m - 1)) >> 64)"),
    "weight_ignored": ("oracle_weighted_accept(r[2], wmax[v], thr, weights[off + (int64_t)idx])",
                       "oracle_weighted_accept(r[2], wmax[v], thr, wmax[v])"),
    "weighted_tie_accepted": ("return (lhs << d) < rhs;", "return (lhs << d) <= rhs;"),
    "weighted_exponent_gap_sign": ("int d = e1 - e2;", "int d = e2 - e1;"),
    "membership_transposed": ("in_row(offsets, dsts, t, x)", "in_row(offsets, dsts, x, t)"),
    "fallback_without_alpha": ("double a = (cls == CLS_FIRST) ? 1.0 : alpha[cls];",
                               "double a = 1.0;"),
    "prev_node_order": ("            t = v;\n            v = x;", "            v = x;\n            t = v;"),
    "start_index": ("int64_t i = w % num_starts;", "int64_t i = w / num_starts;"),
    "accept_inverted": ("accept = (uint64_t)r[2] < thr;", "accept = (uint64_t)r[2] >= thr;"),
}


def _graphs(lib):
    out = []
    for weighted in (False, True):
        n, e = _law.graph_house()
        w = [0.1 + 0.9 * ((7 * k + 3) % 11) / 10 for k in range(len(e))] if weighted else None
        out.append(oracle.Graph(*_law.csr_from_edges(n, e, w, True), lib=lib))
        n, e = _law.graph_directed()
        w = [0.2 + 0.15 * (k % 6) for k in range(len(e))] if weighted else None
        out.append(oracle.Graph(*_law.csr_from_edges(n, e, w, False), lib=lib))
    return out


def pin_battery(lib):
    """Names of the pins that fail for the oracle library `lib`."""
    failed = []
    for cap in (oracle.DEFAULT_TRIAL_CAP, 0):
        for g in _graphs(lib):
            pv = []
            for (p, q) in [(0.25, 4.0), (2.0, 0.5)]:
                for (t, v) in _law.contexts(g.offsets, g.dsts):
                    d = oracle.next_many(g, t, v, p, q, 99, 1000 * v, 4000,
                                         2 if t >= 0 else 1, cap)
                    row = g.dsts[g.offsets[v]:g.offsets[v + 1]]
                    pv.append(_law.chi2_pvalue(
                        d, row, _law.exact_law(g.offsets, g.dsts, g.weights, t, v, p, q)))
            if min(pv) < 1e-6:
                failed.append(f"law(cap={cap})")
                break
    # Closed form on a cycle through full walks.
    n = 9
    cyc = oracle.Graph(*_law.csr_from_edges(n, [(i, (i + 1) % n) for i in range(n)]), lib=lib)
    rows, _ = oracle.walks(cyc, None, 30, 200, 2.0, 0.5, seed=5)
    a, c = rows[:, 2:], rows[:, :-2]
    f = (a == c).mean()
    if abs(f - 0.5 / 2.5) > 0.02:
        failed.append("cycle")
    # Invariants: the first entry of every row is its start.
    starts = np.array([3, 1, 4, 1, 5], np.int32)
    g = _graphs(lib)[0]
    rows, _ = oracle.walks(g, starts, 8, 3, 1.0, 1.0, seed=2)
    if not all(rows[w, 0] == starts[w % len(starts)] for w in range(len(rows))):
        failed.append("starts")
    # The weighted rule against exact rationals (ties included).
    from fractions import Fraction
    f32 = np.float32
    for r2, wm, T, w in [(2**31, f32(1.0), 2**31, f32(1.0)), (3, f32(0.75), 2, f32(0.5)),
                         (5, f32(0.5), 4, f32(0.25)), (2**20, f32(0.9), 2**30, f32(0.001))]:
        want = Fraction(r2) * Fraction(float(wm)) < Fraction(T) * Fraction(float(w))
        if oracle.weighted_accept(r2, wm, T, w, lib=lib) != want:
            failed.append("weighted_rule")
            break
    # First-order unweighted walks accept every proposal: one trial per step.
    st = oracle.OracleStats()
    oracle.walks(g, None, 10, 5, 1.0, 1.0, seed=4, stats=st)
    if st.trials != st.steps or st.fallbacks != 0:
        failed.append("first_order_trials")
    return failed


def test_true_oracle_passes_battery():
    assert pin_battery(oracle.load()) == []


@pytest.mark.parametrize("name", sorted(PLANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = PLANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"plant site for {name} not found"
    mutated = tmp_path / "walk_oracle_planted.c"
    mutated.write_text(src.replace(old, new))
    so = oracle.compile_oracle(str(mutated), str(tmp_path / "liboracle_planted.so"))
    failed = pin_battery(oracle.load(so))
    assert failed, f"planted mistake {name} escaped every pin"
