"""CPU oracle for the Elias-Fano graph store (GRAPE, Methods, "Succinct data
structures for adjacency matrices": "Memory Complexity", "Edge Encoding",
"Operations on Elias-Fano", "Efficient implementation of Elias-Fano").

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this module.  The product library
neither imports it nor shares code with it.

Plain Python and numpy, written for clarity, not speed: bit arrays are numpy
arrays of 0/1, every select and rank starts at an index entry and scans one bit
at a time.

The store, as the paper defines it:

* **Edge encoding.**  With k = ceil(log2 |V|), the edge (a, b) becomes
  phi_k(a, b) = a * 2^k + b, so the encodings of N(a) are the sorted run of
  codes in [phi_k(a, 0), phi_k(a + 1, 0)).  All codes lie below
  u = |V| * 2^k.
* **Elias-Fano** of a non-decreasing sequence y_0 .. y_{n-1} below u:
  l = floor(log2(u / n)) low bits per element (0 when u <= n), stored
  consecutively in a low-bits array; the high parts h_i = y_i >> l stored as
  the inverted unary codes of their gaps (h_i - h_{i-1} zeros, then a one).
* **Indexes.**  With quantum q, the position of every q-th one and of every
  q-th zero of the high-bits array.
* **select(S, i)** is the i-th smallest value (0-based here) and
  **rank(S, m)** is the number of values strictly below m (the paper's
  deviation from Jacobson's "less or equal").
* **Degree and neighbours:** d(a) = rank(phi_k(a + 1, 0)) - rank(phi_k(a, 0)),
  N(a) = { select(i) & (2^k - 1) : rank(phi_k(a, 0)) <= i < rank(phi_k(a + 1, 0)) }.

Readings where the paper leaves the layout open (the supplementary section
with the full layout is not available):

1. Bit order: bit b of a bit array is bit (b mod 64) of 64-bit word b div 64
   (little-endian within the word); element i's low part occupies bits
   [i * l, (i + 1) * l), least significant bit first.
2. The high-bits array ends with the zeros that close every bucket up to
   (u - 1) >> l, so it holds n ones and ((u - 1) >> l) + 1 zeros.  Zero
   number j then closes bucket j: it sits after the ones of every value with
   high part <= j.  The paper's gap code alone stops at the last one; the
   closing zeros let rank run to the end of the universe without a special
   case, and keep the size within the paper's bound 2n + n ceil(log2(u/n)).
3. Index entries: ones_index[j] is the position of one number j * q, for
   j = 0 .. ceil(n / q) - 1; zeros_index[j] the position of zero number j * q,
   for j = 0 .. ceil(Z / q) - 1 (Z the number of zeros).
4. u = |V| * 2^k (every code is below it); k = 0 when |V| = 1.
"""
from __future__ import annotations

import numpy as np


def low_bits_count(n: int, u: int) -> int:
    """l = floor(log2(u / n)), the paper's optimal split; 0 when u <= n or n = 0."""
    if n <= 0 or u <= n:
        return 0
    # floor(log2(u / n)) == floor(log2(floor(u / n))) for integers u, n
    return (u // n).bit_length() - 1


def _pack_words(bits: np.ndarray) -> np.ndarray:
    """0/1 array -> uint64 words, bit b in bit (b mod 64) of word b // 64."""
    nwords = (len(bits) + 63) // 64
    padded = np.zeros(nwords * 64, dtype=np.uint8)
    padded[:len(bits)] = bits
    by = np.packbits(padded, bitorder="little")
    return by.view("<u8").astype(np.uint64) if nwords else np.zeros(0, dtype=np.uint64)


class EliasFano:
    """Elias-Fano representation of a non-decreasing integer sequence below u."""

    def __init__(self, values, u: int, quantum: int = 1024):
        y = np.asarray(values, dtype=np.int64)
        if y.ndim != 1:
            raise ValueError("values must be one-dimensional")
        if u < 1 or quantum < 1:
            raise ValueError("u and quantum must be >= 1")
        if len(y) and (y[0] < 0 or y[-1] >= u or np.any(np.diff(y) < 0)):
            raise ValueError("values must be non-decreasing and in [0, u)")
        self.n = int(len(y))
        self.u = int(u)
        self.q = int(quantum)
        self.l = low_bits_count(self.n, self.u)
        l = self.l
        # low part: element i's l low bits at bit positions [i*l, (i+1)*l), LSB first
        if l > 0 and self.n:
            lows = y & ((1 << l) - 1)
            self.low_bitarray = ((lows[:, None] >> np.arange(l, dtype=np.int64)) & 1) \
                .astype(np.uint8).reshape(-1)
        else:
            self.low_bitarray = np.zeros(0, dtype=np.uint8)
        # high part: inverted unary codes of the gaps between high parts, then the
        # zeros closing the remaining buckets (reading 2)
        high = y >> l
        self.num_zeros = ((self.u - 1) >> l) + 1
        self.high_len = self.n + self.num_zeros
        H = np.zeros(self.high_len, dtype=np.uint8)
        prev = 0
        pos = 0
        for i in range(self.n):
            pos += int(high[i]) - prev          # h_i - h_{i-1} zeros ...
            H[pos] = 1                          # ... then a one
            pos += 1
            prev = int(high[i])
        self.high_bitarray = H
        self._H = H.tolist()                    # plain list: the scans index it bit by bit
        self._low_list = self.low_bitarray.tolist()
        self.low_words = _pack_words(self.low_bitarray)
        self.high_words = _pack_words(self.high_bitarray)
        ones = np.flatnonzero(H == 1)
        zeros = np.flatnonzero(H == 0)
        assert len(ones) == self.n and len(zeros) == self.num_zeros
        self.ones_index = ones[::self.q].astype(np.int64)      # every q-th one
        self.zeros_index = zeros[::self.q].astype(np.int64)    # every q-th zero

    # --- size --------------------------------------------------------------
    @property
    def size_bits(self) -> int:
        """Bits of the low and high arrays (the indexes excluded)."""
        return self.n * self.l + self.high_len

    # --- primitives -------------------------------------------------------
    def low(self, i: int) -> int:
        v = 0
        for j in range(self.l):
            v |= self._low_list[i * self.l + j] << j
        return v

    def _scan(self, start: int, bit: int, count: int) -> int:
        """Position of the count-th (0-based) `bit` at or after `start`."""
        p = start
        seen = -1
        H = self._H
        while True:
            if H[p] == bit:
                seen += 1
                if seen == count:
                    return p
            p += 1

    def select1(self, i: int) -> int:
        """Position of one number i in the high bits: start at the index entry of
        one number (i // q) * q and scan forward."""
        if not 0 <= i < self.n:
            raise IndexError(i)
        return self._scan(int(self.ones_index[i // self.q]), 1, i % self.q)

    def select0(self, z: int) -> int:
        """Position of zero number z in the high bits, from the zeros index."""
        if not 0 <= z < self.num_zeros:
            raise IndexError(z)
        return self._scan(int(self.zeros_index[z // self.q]), 0, z % self.q)

    # --- the paper's operations --------------------------------------------
    def select(self, i: int) -> int:
        """The i-th smallest value (0-based): high part = position of its one
        minus the ones before it, joined to its low part."""
        h = self.select1(i) - i
        return (h << self.l) | self.low(i)

    def rank(self, m: int) -> int:
        """Number of values strictly below m."""
        if m <= 0:
            return 0
        if m >= self.u:
            return self.n
        h = m >> self.l
        lo = m & ((1 << self.l) - 1)
        # the ones of bucket h start after the zero closing bucket h - 1; every
        # one before that position belongs to a value with high part < h
        p = 0 if h == 0 else self.select0(h - 1) + 1
        i = p - h
        H = self._H
        while H[p] == 1 and self.low(i) < lo:   # bucket h ends at its closing zero
            i += 1
            p += 1
        return i

    def contains(self, m: int) -> bool:
        i = self.rank(m)
        return i < self.n and self.select(i) == m

    def values(self) -> np.ndarray:
        return np.array([self.select(i) for i in range(self.n)], dtype=np.int64)


# ---------------------------------------------------------------------------
# Graphs
# ---------------------------------------------------------------------------
def code_bits(num_nodes: int) -> int:
    """k = ceil(log2 |V|)."""
    if num_nodes < 1:
        raise ValueError("num_nodes must be >= 1")
    return (num_nodes - 1).bit_length()


def phi(a: int, b: int, k: int) -> int:
    """phi_k(a, b) = a * 2^k + b (Edge Encoding)."""
    return a * (1 << k) + b


def unphi(c: int, k: int):
    """(a, b) = (c >> k, c & (2^k - 1))."""
    return c >> k, c & ((1 << k) - 1)


def edge_codes(offsets, dsts, k: int) -> np.ndarray:
    """phi_k(a, b) for every CSR entry, in CSR order."""
    offsets = np.asarray(offsets, dtype=np.int64)
    dsts = np.asarray(dsts, dtype=np.int64)
    rows = np.repeat(np.arange(len(offsets) - 1, dtype=np.int64), np.diff(offsets))
    return rows * (1 << k) + dsts


class EFGraph:
    """A CSR graph stored as the Elias-Fano representation of its edge codes."""

    def __init__(self, offsets, dsts, num_nodes: int, quantum: int = 1024):
        self.num_nodes = int(num_nodes)
        self.k = code_bits(self.num_nodes)
        codes = edge_codes(offsets, dsts, self.k)
        if len(codes) > 1 and np.any(np.diff(codes) <= 0):
            raise ValueError("rows must be strictly increasing")
        self.ef = EliasFano(codes, self.num_nodes << self.k, quantum)

    def row_begin(self, a: int) -> int:
        return self.ef.rank(phi(a, 0, self.k))

    def degree(self, a: int) -> int:
        return self.ef.rank(phi(a + 1, 0, self.k)) - self.ef.rank(phi(a, 0, self.k))

    def neighbours(self, a: int) -> np.ndarray:
        lo, hi = self.ef.rank(phi(a, 0, self.k)), self.ef.rank(phi(a + 1, 0, self.k))
        mask = (1 << self.k) - 1
        return np.array([self.ef.select(i) & mask for i in range(lo, hi)], dtype=np.int64)

    def has_edge(self, a: int, b: int) -> bool:
        return self.ef.contains(phi(a, b, self.k))

    def to_csr(self):
        deg = np.array([self.degree(a) for a in range(self.num_nodes)], dtype=np.int64)
        offsets = np.zeros(self.num_nodes + 1, dtype=np.int64)
        np.cumsum(deg, out=offsets[1:])
        mask = (1 << self.k) - 1
        dsts = np.array([self.ef.select(i) & mask for i in range(self.ef.n)], dtype=np.int32)
        return offsets, dsts
