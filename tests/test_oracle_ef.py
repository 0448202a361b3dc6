"""Pins of the Elias-Fano oracle (GRAPE, Methods, "Succinct data structures for
adjacency matrices") to facts that do not come from the oracle itself:

* the paper's own example of the inverted unary code (5 -> 000001);
* a worked example derived by hand from the definitions (the arithmetic is in
  the comments);
* brute force: select(i) is the i-th smallest value and rank(m) counts the
  values strictly below m, for every i and m, on random sequences with
  duplicates, for several quanta;
* the index entries: ones_index[j] is a one with exactly j*q ones before it,
  zeros_index[j] a zero with exactly j*q zeros before it;
* the paper's size bound EF(n, u) = 2n + n ceil(log2(u/n)) bits, the
  low/high split floor(log2(u/n)) minimising n*l + u/2^l, and the paper's two
  figures for quantum 1024 (3.125 % index overhead over the high bits, 16 words
  scanned per select on average);
* the graph encoding: phi_k and its inverse, the range property
  phi_k(a, 0) <= phi_k(a, b) < phi_k(a + 1, 0), degrees and rows equal to the
  CSR's, edge membership equal to a set lookup;
* planted mistakes in copies of the oracle source, each caught.
"""
import os
import random
import types
from fractions import Fraction

import numpy as np
import pytest

from oracle import elias_fano as EF
from paper_2110_06196_gb300 import synth

SRC = os.path.join(os.path.dirname(EF.__file__), "elias_fano.py")


def _bits_of_words(words, nbits):
    return [int((int(words[b // 64]) >> (b % 64)) & 1) for b in range(nbits)]


# ---------------------------------------------------------------------------
# examples
# ---------------------------------------------------------------------------
def check_paper_unary(mod):
    # Inverted unary code of a gap of 5: five zeros then a one ("000001").
    # Six copies of 5 below u = 6: n = 6 >= u, so l = 0 and every value is its
    # own high part.  The first one follows 5 zeros; the other five have gap 0;
    # one more zero closes bucket 5 = (u - 1) >> 0.
    e = mod.EliasFano([5] * 6, 6, quantum=1)
    assert e.l == 0
    assert "".join(map(str, e.high_bitarray)) == "000001" + "11111" + "0"
    assert int(e.high_words[0]) == 2016          # bits 5..10
    assert list(e.values()) == [5] * 6


def check_worked_example(mod):
    # y = 2 3 5 7 11 13 24, u = 32, quantum 2.
    # n = 7, u / n = 4.57 -> l = floor(log2 4.57) = 2.
    # low parts (y mod 4): 2 3 1 3 3 1 0, two bits each, LSB first:
    #   bits 0..13 = 01 11 10 11 11 10 00 -> set bits 1 2 3 4 6 7 8 9 10 -> word 2014
    # high parts (y >> 2): 0 0 1 1 2 3 6, gaps 0 0 1 0 1 1 3:
    #   1 1 01 1 01 01 0001, then ((32 - 1) >> 2) + 1 = 8 zeros in all, 6 used,
    #   2 more: 110110101000100 (15 bits) -> set bits 0 1 3 4 6 8 12 -> word 4443
    # ones at 0 1 3 4 6 8 12, zeros at 2 5 7 9 10 11 13 14;
    # every 2nd: ones_index = 0 3 6 12, zeros_index = 2 7 10 13.
    y = [2, 3, 5, 7, 11, 13, 24]
    e = mod.EliasFano(y, 32, quantum=2)
    assert e.l == 2
    assert e.n == 7 and e.num_zeros == 8 and e.high_len == 15
    assert [int(w) for w in e.low_words] == [2014]
    assert [int(w) for w in e.high_words] == [4443]
    assert "".join(map(str, e.high_bitarray)) == "110110101000100"
    assert list(e.ones_index) == [0, 3, 6, 12]
    assert list(e.zeros_index) == [2, 7, 10, 13]
    assert e.size_bits == 29
    assert [e.select(i) for i in range(7)] == y
    # rank(12): bucket 3, low 0; zero 2 (closing bucket 2) is at 7, so bucket 3
    # starts at 8 with value number 8 - 3 = 5 (13, low 1, not < 0): 5
    # rank(14): low 2; value 5 has low 1 < 2, position 9 is a zero: 6
    assert [e.rank(m) for m in (0, 2, 3, 5, 6, 12, 14, 24, 25, 31, 32, 40)] == \
        [0, 0, 1, 2, 3, 5, 6, 6, 7, 7, 7, 7]


def check_graph_example(mod):
    # |V| = 5 -> k = ceil(log2 5) = 3, u = 5 * 8 = 40.
    # rows: 0 -> 1 4; 1 -> 0; 2 -> (none); 3 -> 3 4; 4 -> 0 1 3
    # codes a*8 + b: 1 4 | 8 | | 27 28 | 32 33 35; n = 8, l = floor(log2 5) = 2
    offsets = [0, 2, 3, 3, 5, 8]
    dsts = [1, 4, 0, 3, 4, 0, 1, 3]
    g = mod.EFGraph(offsets, dsts, 5, quantum=2)
    assert g.k == 3 and g.ef.u == 40 and g.ef.l == 2
    assert list(g.ef.values()) == [1, 4, 8, 27, 28, 32, 33, 35]
    assert [g.degree(a) for a in range(5)] == [2, 1, 0, 2, 3]
    assert [list(g.neighbours(a)) for a in range(5)] == [[1, 4], [0], [], [3, 4], [0, 1, 3]]
    assert g.has_edge(3, 3) and g.has_edge(4, 1) and not g.has_edge(2, 0) and not g.has_edge(0, 0)
    assert mod.code_bits(4) == 2 and mod.code_bits(5) == 3 and mod.code_bits(1) == 0
    assert mod.code_bits(1 << 20) == 20 and mod.code_bits((1 << 20) + 1) == 21


# ---------------------------------------------------------------------------
# brute force and bounds
# ---------------------------------------------------------------------------
def _random_sequence(rng, n, u, distinct):
    if distinct:
        return sorted(rng.sample(range(u), n))
    return sorted(rng.randrange(u) for _ in range(n))


CASES = [(0, 1, 1), (0, 9, 4), (1, 1, 1), (1, 1000, 2), (5, 5, 1), (7, 3, 2), (50, 50, 4),
         (60, 5000, 8), (200, 1 << 20, 3), (300, 301, 1024), (400, 64, 16), (1000, 1 << 33, 64),
         (257, 4096, 256)]


def check_brute_force(mod, seed=5):
    rng = random.Random(seed)
    for (n, u, q) in CASES:
        for distinct in ((True, False) if n <= u else (False,)):
            y = _random_sequence(rng, n, u, distinct)
            e = mod.EliasFano(y, u, quantum=q)
            assert [e.select(i) for i in range(n)] == y, (n, u, q)
            ms = list(range(min(u + 3, 600))) + [rng.randrange(u + 5) for _ in range(200)]
            for m in ms:
                assert e.rank(m) == int(np.searchsorted(y, m, side="left")), (n, u, q, m)
            # contains() agrees with a set lookup
            s = set(y)
            for m in ms:
                assert e.contains(m) == (m in s)


def check_indexes(mod, seed=6):
    rng = random.Random(seed)
    for (n, u, q) in CASES:
        y = _random_sequence(rng, n, u, False)
        e = mod.EliasFano(y, u, quantum=q)
        H = [int(b) for b in e.high_bitarray]
        assert sum(H) == n and len(H) - n == ((u - 1) >> e.l) + 1
        assert _bits_of_words(e.high_words, len(H)) == H
        assert len(e.ones_index) == (n + q - 1) // q
        assert len(e.zeros_index) == (e.num_zeros + q - 1) // q
        for j, p in enumerate(e.ones_index):
            assert H[p] == 1 and sum(H[:p]) == j * q
        for j, p in enumerate(e.zeros_index):
            assert H[p] == 0 and (p - sum(H[:p])) == j * q
        # low words hold each value's low part, LSB first
        lb = _bits_of_words(e.low_words, n * e.l)
        for i, v in enumerate(y):
            assert sum(lb[i * e.l + j] << j for j in range(e.l)) == v % (1 << e.l)


def _ceil_log2_ratio(u, n):
    """ceil(log2(u / n)) for u >= n >= 1, exactly: the least c with n 2^c >= u."""
    c = 0
    while n << c < u:
        c += 1
    return c


def check_size_and_split(mod, seed=7):
    rng = random.Random(seed)
    for _ in range(150):
        u = rng.randrange(1, 1 << rng.randrange(1, 40))
        n = rng.randrange(1, min(u, 3000) + 1)
        l = mod.low_bits_count(n, u)
        # the paper's split: floor(log2(u / n)) exactly
        assert (n << l) <= u < (n << (l + 1)) or (u <= n and l == 0)
        # it minimises n*l + u/2^l (low bits plus the zeros of the high part)
        cost = [Fraction(n * j) + Fraction(u, 1 << j) for j in range(64)]
        assert cost[l] == min(cost)
        # the encoded size is within EF(n, u) = 2n + n ceil(log2(u/n)) (distinct values)
        if n <= 400:
            y = sorted(rng.sample(range(u), n))
            e = mod.EliasFano(y, u, quantum=8)
            assert e.size_bits <= 2 * n + n * _ceil_log2_ratio(u, n)


def check_graphs(mod):
    graphs = [synth.erdos_renyi(300, 1200, seed=3), synth.rmat(9, 3000, seed=4),
              synth.rmat(7, 300, seed=5)]
    for csr in graphs:
        offsets, dsts, _ = csr.numpy()
        n = csr.num_nodes
        for q in (1, 7, 64, 1024):
            g = mod.EFGraph(offsets, dsts, n, quantum=q)
            k = g.k
            assert (1 << k) >= n and (k == 0 or (1 << (k - 1)) < n)
            o2, d2 = g.to_csr()
            assert np.array_equal(o2, offsets) and np.array_equal(d2, dsts)
            for a in range(0, n, 17):
                assert g.row_begin(a) == offsets[a]
                row = dsts[offsets[a]:offsets[a + 1]]
                for b in row:
                    c = mod.phi(a, int(b), k)
                    assert mod.phi(a, 0, k) <= c < mod.phi(a + 1, 0, k)
                    assert mod.unphi(c, k) == (a, int(b))
                    assert c == (a << k) | int(b)
            rng = random.Random(q)
            edges = set(zip(np.repeat(np.arange(n), np.diff(offsets)).tolist(), dsts.tolist()))
            for _ in range(300):
                a, b = rng.randrange(n), rng.randrange(n)
                assert g.has_edge(a, b) == ((a, b) in edges)
    # a directed graph with a dead end and a self-loop
    offsets = np.array([0, 2, 2, 4], dtype=np.int64)
    dsts = np.array([1, 2, 0, 2], dtype=np.int32)
    g = mod.EFGraph(offsets, dsts, 3, quantum=1)
    assert [g.degree(a) for a in range(3)] == [2, 0, 2]
    assert g.has_edge(2, 2) and not g.has_edge(1, 0)


PINS = [check_paper_unary, check_worked_example, check_graph_example, check_brute_force,
        check_indexes, check_size_and_split, check_graphs]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(EF)


def test_paper_figures_for_quantum_1024():
    # "Efficient implementation of Elias-Fano": with q = 1024 the index costs
    # 3.125 % over the high bits, and a select scans 16 words on average.
    # Distinct values with u / n = 2^8: the high bits hold n ones and about n
    # zeros, so an index entry (64 bits) per 1024 ones is 64 / 2048 of them, and
    # the scan from an entry to a one covers half of a 2048-bit stretch.
    rng = np.random.default_rng(8)
    n, u = 1 << 17, (1 << 17) << 8
    y = np.sort(rng.choice(u, size=n, replace=False))
    e = EF.EliasFano(y, u, quantum=1024)
    assert e.l == 8
    overhead = 64 * len(e.ones_index) / e.high_len
    assert abs(overhead - 0.03125) < 0.0015, overhead
    idx = rng.integers(0, n, 3000)
    words = [(e.select1(int(i)) - int(e.ones_index[int(i) // 1024])) / 64 + 1 for i in idx]
    assert 15.0 < float(np.mean(words)) < 17.0, np.mean(words)


def test_rejects_bad_input():
    with pytest.raises(ValueError):
        EF.EliasFano([3, 2], 10)
    with pytest.raises(ValueError):
        EF.EliasFano([0, 10], 10)
    with pytest.raises(ValueError):
        EF.EFGraph([0, 2], [1, 1], 2)       # a multi-edge


# ---------------------------------------------------------------------------
# planted mistakes
# ---------------------------------------------------------------------------
PLANTS = {
    "rank_less_or_equal": ("and self.low(i) < lo:", "and self.low(i) <= lo:"),
    "split_one_too_many": ("return (u // n).bit_length() - 1", "return (u // n).bit_length()"),
    "unary_of_values": ("pos += int(high[i]) - prev", "pos += int(high[i])"),
    "bucket_start_off_by_one": ("i = p - h\n", "i = p - h + 1\n"),
    "select_skips_one": ("1, i % self.q)", "1, i % self.q + 1)"),
    "lows_msb_first": ("(lows[:, None] >> np.arange(l, dtype=np.int64))",
                       "(lows[:, None] >> np.arange(l - 1, -1, -1, dtype=np.int64))"),
    "k_one_too_many": ("return (num_nodes - 1).bit_length()", "return num_nodes.bit_length()"),
    "no_closing_zeros": ("self.num_zeros = ((self.u - 1) >> l) + 1",
                         "self.num_zeros = (int(high[-1]) if self.n else 0) + 1"),
    "zeros_index_of_ones": ("self.zeros_index = zeros[::self.q]", "self.zeros_index = ones[::self.q]"),
}


def _planted(name):
    src = open(SRC).read()
    old, new = PLANTS[name]
    assert src.count(old) == 1, name
    mod = types.ModuleType(f"ef_plant_{name}")
    exec(compile(src.replace(old, new), f"<plant {name}>", "exec"), mod.__dict__)
    return mod


def _failing_pins(mod):
    failed = []
    for pin in PINS:
        try:
            pin(mod)
        except Exception:       # an assertion, or the mistake breaking the code itself
            failed.append(pin.__name__)
    return failed


@pytest.mark.parametrize("name", sorted(PLANTS))
def test_planted_mistake_is_caught(name):
    assert _failing_pins(_planted(name)), f"no pin caught the planted mistake {name}"
