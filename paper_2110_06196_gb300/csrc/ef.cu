// ef.cu -- the Elias-Fano graph store and node2vec walks over it.
//
// GRAPE, Methods, "Succinct data structures for adjacency matrices":
//   * Edge Encoding: the edge (a, b) becomes phi_k(a, b) = a * 2^k + b with
//     k = ceil(log2 |V|), so the codes of N(a) are the sorted run in
//     [phi_k(a, 0), phi_k(a + 1, 0)); every code is below u = |V| * 2^k.
//   * Efficient implementation of Elias-Fano: l = floor(log2(u / m)) low bits
//     of each code in a packed array; the high parts as the inverted unary
//     codes of their gaps; the positions of every q-th one and every q-th zero
//     of the high bits as indexes, from which a select scans forward.
//   * Operations on Elias-Fano: rank(c) = number of codes below c, select(i)
//     = the i-th smallest code; deg(a) = rank(phi(a + 1, 0)) - rank(phi(a, 0))
//     and N(a) = select(i) & (2^k - 1) over that range.
//
// Layout (64-bit words; bit b of an array is bit b mod 64 of word b / 64):
//   low[]         code i's l low bits at bits [i l, (i + 1) l), least significant first
//   high[]        code i's one at bit (code_i >> l) + i; Z = ((u - 1) >> l) + 1 zeros,
//                 zero j closing bucket j (it follows every code whose high part is <= j)
//   ones_index[]  position of one number j q,   j < ceil(m / q)
//   zeros_index[] position of zero number j q,  j < ceil(Z / q)
// Both bit arrays carry four words of zero padding.  Beside the paper's layout
// the store keeps the row pointers (rank(phi(a, 0)) of every node, with a
// directory slot in the high bits) and bucket directories for hub rows, so a
// walk reads a degree in one access and never scans the dense high bits of a
// hub's row.
//
// Walks over the store follow the same rule as the CSR engine (rejection
// against max(1/p, 1, 1/q) * wmax_v with Philox blocks keyed by (seed, walk,
// step, trial), then the cumulative-sum fallback), so their rows are
// byte-identical to grape_walks' rows for the same graph.  One thread owns one
// walk; every neighbour is a select and every membership test a bucket search
// on the compressed store.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "internal.h"

using namespace grape;

struct grape_ef_graph {
    int64_t n = 0, m = 0, u = 0;
    int32_t k = 0, l = 0, quantum = 0, qlog = 0;
    int64_t num_zeros = 0, high_bits = 0;
    int64_t low_words = 0, high_words = 0, ones_len = 0, zeros_len = 0;
    int32_t max_degree = 0;
    bool weighted = false;
    int device = 0, num_sms = 0;
    unsigned long long* low = nullptr;
    unsigned long long* high = nullptr;
    long long* ones_idx = nullptr;
    long long* zeros_idx = nullptr;
    float* weights = nullptr;
    float* wmax = nullptr;
    long long* rowptr = nullptr;              // [n + 1] first code of every row (CSR offsets),
                                              // a bucket directory slot in bits 40-62
    unsigned* dir = nullptr;                  // bucket directories of long rows
    int32_t dir_rows = 0;
    bool undirected = false;
    int* status = nullptr;                    // [0] device status word, [1] bad flags, [2] max degree
    unsigned long long* counters = nullptr;   // [C_COUNT]
    bool counting = false;
    int64_t device_bytes = 0, structure_bytes = 0;
};

namespace {

constexpr int kEFThreads = 256;
constexpr int kPadWords = 4;
// Row pointers hold the row's first code index in bits 0-39 and, for a row with
// a bucket directory, 1 + the directory's index in bits 40-62.
constexpr int kRowPtrBits = 40;
constexpr long long kRowPtrMask = (1LL << kRowPtrBits) - 1;
constexpr int kMaxDirRows = (1 << 23) - 1;

struct EFDev {
    const unsigned long long* low;
    const unsigned long long* high;
    const long long* ones_idx;
    const long long* zeros_idx;
    const float* weights;
    const float* wmax;
    const long long* rowptr;
    const unsigned* dir;
    long long m, n, u;
    long long hwords;           // high-bit words, padding included
    int k, l, qlog;
    int undirected;
    int* status;                // bit 0: a start id out of range; bit 1: an inconsistent store
    unsigned long long* counters;
};

EFDev dev_view(const grape_ef_graph* g) {
    EFDev d;
    d.low = g->low;
    d.high = g->high;
    d.ones_idx = g->ones_idx;
    d.zeros_idx = g->zeros_idx;
    d.weights = g->weights;
    d.wmax = g->wmax;
    d.rowptr = g->rowptr;
    d.dir = g->dir;
    d.undirected = g->undirected ? 1 : 0;
    d.m = g->m;
    d.n = g->n;
    d.u = g->u;
    d.hwords = g->high_words + kPadWords;
    d.k = g->k;
    d.l = g->l;
    d.qlog = g->qlog;
    d.status = g->status;
    d.counters = g->counting ? g->counters : nullptr;
    return d;
}

int ef_grid(int num_sms, long long items, int per_block) {
    const long long b = (items + per_block - 1) / per_block;
    return (int)std::max(1LL, std::min(b, (long long)num_sms * 32));
}

// ---------------------------------------------------------------------------
// Building the store from a device CSR
// ---------------------------------------------------------------------------
__global__ void ef_check_offsets_kernel(const int64_t* __restrict__ offsets, long long n,
                                        long long m, int* bad) {
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a <= n;
         a += (long long)gridDim.x * blockDim.x) {
        const long long o = offsets[a];
        bool ok = o >= 0 && o <= m;
        if (a == 0) ok = ok && o == 0;
        if (a == n) ok = ok && o == m;
        if (a < n) ok = ok && offsets[a + 1] >= o;
        if (!ok) atomicOr(bad, 1);
    }
}

// One warp per row: ids in range, rows strictly increasing, weights finite and
// > 0; the largest degree and each row's largest weight.
__global__ void ef_check_rows_kernel(const int64_t* __restrict__ offsets,
                                     const int32_t* __restrict__ dsts,
                                     const float* __restrict__ weights, long long n,
                                     float* __restrict__ wmax, int* bad, int* max_deg) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long a = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; a < n; a += warps) {
        const long long lo = offsets[a], hi = offsets[a + 1];
        bool ok = true;
        float wm = 0.0f;
        for (long long e = lo + lane; e < hi; e += 32) {
            const int x = dsts[e];
            ok = ok && x >= 0 && x < n;
            if (e + 1 < hi) ok = ok && dsts[e + 1] > x;
            if (weights) {
                const float w = weights[e];
                ok = ok && isfinite(w) && w > 0.0f;
                wm = fmaxf(wm, w);
            }
        }
        if (!__all_sync(FULL, ok) && lane == 0) atomicOr(bad, 1);
        if (weights) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) wm = fmaxf(wm, __shfl_xor_sync(FULL, wm, o));
            if (lane == 0) wmax[a] = wm;
        }
        if (lane == 0) {
            const long long d = hi - lo;
            atomicMax(max_deg, (int)(d < INT32_MAX ? d : INT32_MAX));
        }
    }
}

// GRAPE_UNDIRECTED with GRAPE_VALIDATE: every entry (a, b) has its reverse
// entry (b, a), with the same weight.  One warp per row, one binary search per
// entry (ids are known in range and rows sorted by now).
__global__ void ef_check_symmetry_kernel(const int64_t* __restrict__ offsets,
                                         const int32_t* __restrict__ dsts,
                                         const float* __restrict__ weights, long long n,
                                         int* bad) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long a = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; a < n; a += warps) {
        bool ok = true;
        for (long long e = offsets[a] + lane; e < offsets[a + 1]; e += 32) {
            const int b = dsts[e];
            long long lo = offsets[b], hi = offsets[b + 1];
            while (lo < hi) {
                const long long mid = lo + ((hi - lo) >> 1);
                if (dsts[mid] < a) lo = mid + 1;
                else hi = mid;
            }
            const bool has = lo < offsets[b + 1] && dsts[lo] == a;
            ok = ok && has && (!weights || weights[lo] == weights[e]);
        }
        if (!__all_sync(FULL, ok) && lane == 0) atomicOr(bad, 1);
    }
}

// One warp per row: OR each code's low bits and its high-part one into the
// zeroed arrays.  Codes and positions depend only on the CSR, so the words do
// not depend on the order of the ORs.
__global__ void ef_fill_kernel(const int64_t* __restrict__ offsets,
                               const int32_t* __restrict__ dsts, long long n, int k, int l,
                               unsigned long long* __restrict__ low,
                               unsigned long long* __restrict__ high) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const unsigned long long lmask = l ? ((1ull << l) - 1) : 0ull;
    for (long long a = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; a < n; a += warps) {
        const long long lo = offsets[a], hi = offsets[a + 1];
        for (long long e = lo + lane; e < hi; e += 32) {
            const unsigned long long c = ((unsigned long long)a << k) | (unsigned)dsts[e];
            const unsigned long long pos = (c >> l) + (unsigned long long)e;
            atomicOr(high + (pos >> 6), 1ull << (pos & 63));
            if (l) {
                const unsigned long long bits = c & lmask;
                const unsigned long long b = (unsigned long long)e * (unsigned)l;
                const int s = (int)(b & 63);
                if (bits) {
                    atomicOr(low + (b >> 6), bits << s);
                    if (s + l > 64) atomicOr(low + (b >> 6) + 1, bits >> (64 - s));
                }
            }
        }
    }
}

// Bucket directories.  A long row (deg + nb > 448 and deg >= 8 nb, nb = 2^(k-l)
// buckets per row) gets nb + 1 entries: entry j is the bit offset, from the
// row's region start, where bucket j's ones begin (j + the row's codes in
// buckets below j), entry nb the region's end (deg + nb).  A membership test in
// such a row then reads two entries instead of scanning the dense high bits.
__device__ __forceinline__ bool long_row(long long deg, long long nb) {
    return deg + nb > 448 && deg >= 8 * nb;
}

__global__ void ef_count_long_rows_kernel(const int64_t* __restrict__ offsets, long long n,
                                          long long nb, unsigned long long* count) {
    unsigned long long c = 0;
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < n;
         a += (long long)gridDim.x * blockDim.x)
        c += long_row(offsets[a + 1] - offsets[a], nb) ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// One warp per long row: take a slot (their order is arbitrary and changes no
// result), mark it in the row pointer and fill the directory from the CSR.
__global__ void ef_fill_dirs_kernel(const int64_t* __restrict__ offsets,
                                    const int32_t* __restrict__ dsts, long long n, long long nb,
                                    int l, long long* __restrict__ rowptr,
                                    unsigned* __restrict__ dir, unsigned long long* next) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long a = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; a < n; a += warps) {
        const long long lo = offsets[a], hi = offsets[a + 1];
        if (!long_row(hi - lo, nb)) continue;
        unsigned long long slot = 0;
        if (lane == 0) slot = atomicAdd(next, 1ull);
        slot = __shfl_sync(FULL, slot, 0);
        if (lane == 0) rowptr[a] = lo | (long long)((slot + 1) << kRowPtrBits);
        unsigned* d = dir + slot * (unsigned long long)(nb + 1);
        for (long long j = lane; j <= nb; j += 32) {
            const long long lim = j << l;          // codes of bucket < j: dsts below j 2^l
            long long a0 = lo, a1 = hi;
            while (a0 < a1) {
                const long long mid = a0 + ((a1 - a0) >> 1);
                if ((long long)dsts[mid] < lim) a0 = mid + 1;
                else a1 = mid;
            }
            d[j] = (unsigned)(j + (a0 - lo));
        }
    }
}

// Number of codes below c, from the CSR (c < u): offsets[a] plus the position
// of b in the sorted row a.
__device__ long long csr_rank(const int64_t* __restrict__ offsets, const int32_t* __restrict__ dsts,
                              long long n, int k, unsigned long long c) {
    const long long a = (long long)(c >> k);
    if (a >= n) return offsets[n];
    const int b = (int)(c & ((1ull << k) - 1));
    long long lo = offsets[a], hi = offsets[a + 1];
    while (lo < hi) {                          // first entry >= b
        const long long mid = lo + ((hi - lo) >> 1);
        if (dsts[mid] < b) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Index entries.  One number j q (code e = j q of row a) sits at
// (code >> l) + e.  Zero number z closes bucket z: it follows the codes whose
// high part is <= z, that is the codes below (z + 1) 2^l, so it sits at
// z + rank((z + 1) 2^l).
__global__ void ef_index_kernel(const int64_t* __restrict__ offsets,
                                const int32_t* __restrict__ dsts, long long n, int k, int l,
                                int qlog, long long ones_len, long long zeros_len,
                                unsigned long long u, long long* __restrict__ ones_idx,
                                long long* __restrict__ zeros_idx) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < ones_len + zeros_len;
         j += (long long)gridDim.x * blockDim.x) {
        if (j < ones_len) {
            const long long e = j << qlog;
            long long lo = 0, hi = n;                // row of entry e: last a with offsets[a] <= e
            while (hi - lo > 1) {
                const long long mid = lo + ((hi - lo) >> 1);
                if (offsets[mid] <= e) lo = mid;
                else hi = mid;
            }
            const unsigned long long c = ((unsigned long long)lo << k) | (unsigned)dsts[e];
            ones_idx[j] = (long long)((c >> l) + (unsigned long long)e);
        } else {
            const long long z = (j - ones_len) << qlog;
            const unsigned long long lim = (unsigned long long)(z + 1) << l;
            const long long r = lim >= u ? offsets[n] : csr_rank(offsets, dsts, n, k, lim);
            zeros_idx[j - ones_len] = z + r;
        }
    }
}

// ---------------------------------------------------------------------------
// select and rank on the device
// ---------------------------------------------------------------------------

// Distinct 32-byte sectors read (counting kernels only): a touch counts unless
// its sector is among the last kRecent sectors touched since begin(); a walk
// calls begin() once per step, so a sector read twice within a step (a row
// pointer, a high-bits word) counts once.
template <bool ON>
struct Tally {
    static constexpr int kRecent = 4;
    unsigned long long recent[kRecent];
    unsigned next = 0;
    unsigned sectors = 0;
    __device__ __forceinline__ void begin() {
#pragma unroll
        for (int i = 0; i < kRecent; ++i) recent[i] = ~0ull;
    }
    __device__ __forceinline__ void touch(const void* p) {
        const unsigned long long s = reinterpret_cast<uintptr_t>(p) >> 5;
#pragma unroll
        for (int i = 0; i < kRecent; ++i)
            if (recent[i] == s) return;
        recent[next++ % kRecent] = s;
        ++sectors;
    }
};
template <>
struct Tally<false> {
    __device__ __forceinline__ void begin() {}
    __device__ __forceinline__ void touch(const void*) {}
};

// Position of the r-th (0-based) set bit of x; x has more than r set bits.
__device__ __forceinline__ int nth_set_bit(unsigned long long x, int r) {
    int pos = 0;
    unsigned w = (unsigned)x;
    int c = __popc(w);
    if (r >= c) {
        r -= c;
        w = (unsigned)(x >> 32);
        pos = 32;
    }
    c = __popc(w & 0xffffu);
    if (r >= c) { r -= c; w >>= 16; pos += 16; }
    c = __popc(w & 0xffu);
    if (r >= c) { r -= c; w >>= 8; pos += 8; }
    c = __popc(w & 0xfu);
    if (r >= c) { r -= c; w >>= 4; pos += 4; }
    c = __popc(w & 0x3u);
    if (r >= c) { r -= c; w >>= 2; pos += 2; }
    if (r >= (int)(w & 1u)) pos += 1;
    return pos;
}

// Position of the r-th one (ONES) or zero at or after bit p of the high bits.
// A scan that would leave the array (an inconsistent store) stops, sets
// status bit 1 and returns the array's end.
template <bool ONES, bool C>
__device__ __forceinline__ long long scan_high(const EFDev& g, long long p, long long r,
                                               Tally<C>& ty) {
    long long w = p >> 6;
    if (p < 0 || w >= g.hwords) {
        atomicOr(g.status, 2);
        return g.hwords << 6;
    }
    ty.touch(g.high + w);
    unsigned long long x = __ldg(g.high + w);
    if (!ONES) x = ~x;
    x &= ~0ull << (p & 63);
    while (true) {
        const int c = __popcll(x);
        if (r < c) return (w << 6) + nth_set_bit(x, (int)r);
        r -= c;
        if (++w >= g.hwords) {
            atomicOr(g.status, 2);
            return g.hwords << 6;
        }
        ty.touch(g.high + w);
        x = __ldg(g.high + w);
        if (!ONES) x = ~x;
    }
}

template <bool C>
__device__ __forceinline__ long long select1(const EFDev& g, long long i, Tally<C>& ty) {
    ty.touch(g.ones_idx + (i >> g.qlog));
    const long long p = __ldg(g.ones_idx + (i >> g.qlog));
    return scan_high<true>(g, p, i & ((1LL << g.qlog) - 1), ty);
}

template <bool C>
__device__ __forceinline__ long long select0(const EFDev& g, long long z, Tally<C>& ty) {
    ty.touch(g.zeros_idx + (z >> g.qlog));
    const long long p = __ldg(g.zeros_idx + (z >> g.qlog));
    return scan_high<false>(g, p, z & ((1LL << g.qlog) - 1), ty);
}

template <bool C>
__device__ __forceinline__ unsigned long long low_of(const EFDev& g, long long i, Tally<C>& ty) {
    if (g.l == 0) return 0;
    const unsigned long long b = (unsigned long long)i * (unsigned)g.l;
    const long long w = (long long)(b >> 6);
    const int s = (int)(b & 63);
    ty.touch(g.low + w);
    unsigned long long v = __ldg(g.low + w) >> s;
    if (s + g.l > 64) {
        ty.touch(g.low + w + 1);
        v |= __ldg(g.low + w + 1) << (64 - s);
    }
    return v & ((1ull << g.l) - 1);
}

// The i-th smallest code.
template <bool C>
__device__ __forceinline__ unsigned long long select_code(const EFDev& g, long long i, Tally<C>& ty) {
    const unsigned long long h = (unsigned long long)(select1(g, i, ty) - i);
    return (h << g.l) | low_of(g, i, ty);
}

// Bit position where bucket h's ones begin (just after the zero closing
// bucket h - 1); the first code of the bucket is number (position - h).
template <bool C>
__device__ __forceinline__ long long bucket_begin(const EFDev& g, long long h, Tally<C>& ty) {
    return h == 0 ? 0 : select0(g, h - 1, ty) + 1;
}

// The first of the len codes from i0 (one bucket: their low parts increase)
// whose low part is >= lo, and whether one equals lo.
template <bool C>
__device__ __forceinline__ long long lows_search(const EFDev& g, long long i0, long long len,
                                                 unsigned long long lo, bool& found,
                                                 Tally<C>& ty) {
    found = false;
    if (len <= 0) return i0;
    if (lo == 0) {
        found = (low_of(g, i0, ty) == 0);
        return i0;
    }
    long long a = i0, b = i0 + len;
    while (a < b) {
        const long long mid = a + ((b - a) >> 1);
        if (low_of(g, mid, ty) < lo) a = mid + 1;
        else b = mid;
    }
    found = (a < i0 + len) && low_of(g, a, ty) == lo;
    return a;
}

// Search bucket h, whose ones begin at bit p, for the low part lo: the index
// of its first code whose low part is >= lo, and whether one equals lo.
template <bool C>
__device__ long long bucket_search(const EFDev& g, long long p, long long h, unsigned long long lo,
                                   bool& found, Tally<C>& ty) {
    found = false;
    const long long i0 = p - h;
    // length of bucket h: the run of ones from p (the word at p, then the
    // zeros index when the run reaches the end of that word)
    const long long w = p >> 6;
    if (w >= g.hwords) {                        // an inconsistent store (scan_high flagged it)
        atomicOr(g.status, 2);
        return g.m;
    }
    ty.touch(g.high + w);
    const unsigned long long x = __ldg(g.high + w) >> (p & 63);
    const int room = 64 - (int)(p & 63);
    int run = (~x == 0ull) ? 64 : __ffsll((long long)~x) - 1;
    long long len;
    if (run < room) len = run;
    else len = select0(g, h, ty) - p;          // the zero closing bucket h
    if (i0 < 0 || len < 0 || i0 + len > g.m) {
        atomicOr(g.status, 2);
        return g.m;
    }
    return lows_search(g, i0, len, lo, found, ty);
}

// Codes below c (0 <= c), and whether c itself is stored.
template <bool C>
__device__ long long rank_code(const EFDev& g, unsigned long long c, bool& found, Tally<C>& ty) {
    found = false;
    if ((long long)c >= g.u) return g.m;
    const long long h = (long long)(c >> g.l);
    const unsigned long long lo = g.l ? (c & ((1ull << g.l) - 1)) : 0ull;
    return bucket_search(g, bucket_begin(g, h, ty), h, lo, found, ty);
}

__global__ void ef_select_kernel(EFDev g, const long long* __restrict__ idx, long long n,
                                 long long* __restrict__ out) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        const long long i = idx[j];
        Tally<false> ty;
        if (i < 0 || i >= g.m) {
            out[j] = -1;
            atomicOr(g.status, 1);
        } else {
            out[j] = (long long)select_code(g, i, ty);
        }
    }
}

__global__ void ef_rank_kernel(EFDev g, const long long* __restrict__ vals, long long n,
                               long long* __restrict__ out) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        const long long c = vals[j];
        Tally<false> ty;
        bool f;
        out[j] = c <= 0 ? 0 : rank_code(g, (unsigned long long)c, f, ty);
    }
}

// ---------------------------------------------------------------------------
// Walks
// ---------------------------------------------------------------------------

// Is x in N(t)?
template <bool C>
__device__ __forceinline__ bool ef_has_edge(const EFDev& g, int t, int x, Tally<C>& ty) {
    bool found;
    rank_code(g, ((unsigned long long)t << g.k) | (unsigned)x, found, ty);
    return found;
}

__device__ __forceinline__ int ef_target(const EFDev& g, unsigned long long code) {
    return (int)(code & ((1ull << g.k) - 1));
}

// Words a scan near a known position looks at before it turns to an index.
constexpr int kNearWords = 8;

// The r-th (0-based) one (ONES) or zero at or after bit p, when it lies in the
// kNearWords words from p's word; -1 otherwise.
template <bool ONES, bool C>
__device__ __forceinline__ long long scan_near(const EFDev& g, long long p, long long r,
                                               Tally<C>& ty) {
    long long w = p >> 6;
    const long long wend = w + kNearWords < g.hwords ? w + kNearWords : g.hwords;
    if (p < 0 || w >= wend) return -1;
    ty.touch(g.high + w);
    unsigned long long x = __ldg(g.high + w);
    if (!ONES) x = ~x;
    x &= ~0ull << (p & 63);
    while (true) {
        const int c = __popcll(x);
        if (r < c) return (w << 6) + nth_set_bit(x, (int)r);
        r -= c;
        if (++w >= wend) return -1;
        ty.touch(g.high + w);
        x = __ldg(g.high + w);
        if (!ONES) x = ~x;
    }
}

// A row's place in the store: its first code, degree, the bit position P
// where its region of the high bits begins (-1 when l > k) and its bucket
// directory slot (0: none).
struct Row {
    long long P;
    long long off;
    int deg;
    int slot;
};

// Row a from the row pointers (one 16-byte read).  With l <= k every row
// starts a bucket, h0 = a 2^(k-l), so its region begins at P = off + h0 (off
// ones and h0 zeros before it) and spans deg ones and nb = 2^(k-l) zeros.
template <bool C>
__device__ __forceinline__ Row region_of(const EFDev& g, long long a, Tally<C>& ty) {
    ty.touch(g.rowptr + a);
    const long long w0 = __ldg(g.rowptr + a);
    ty.touch(g.rowptr + a + 1);
    const long long w1 = __ldg(g.rowptr + a + 1);
    Row r;
    r.off = w0 & kRowPtrMask;
    r.deg = (int)((w1 & kRowPtrMask) - r.off);
    r.slot = (int)(w0 >> kRowPtrBits);
    r.P = g.l <= g.k ? r.off + (a << (g.k - g.l)) : -1;
    return r;
}

// Is row r short enough for scans near its start to find every position in it?
__device__ __forceinline__ bool region_near(const EFDev& g, const Row& r) {
    return r.P >= 0 && (r.P & 63) + (long long)r.deg + (1LL << (g.k - g.l)) <= 64LL * kNearWords;
}

// Code number e, the idx-th code of row r (near: region_near(r)).
template <bool C>
__device__ __forceinline__ unsigned long long row_code(const EFDev& g, const Row& r, bool near,
                                                       long long e, long long idx, Tally<C>& ty) {
    long long pos = near ? scan_near<true>(g, r.P, idx, ty) : -1;
    if (pos < 0) pos = select1(g, e, ty);
    return ((unsigned long long)(pos - e) << g.l) | low_of(g, e, ty);
}

// Index of the first code of row a (r) at or above phi(a, b), and whether b is
// in N(a): the bucket of b from the row's directory, or a scan of the zeros
// near the row's start, or the zeros index; then its low parts.
template <bool C>
__device__ __forceinline__ long long find_in_row(const EFDev& g, const Row& r, bool near,
                                                 long long a, int b, bool& found, Tally<C>& ty) {
    if (r.P < 0) return rank_code(g, ((unsigned long long)a << g.k) | (unsigned)b, found, ty);
    const long long j = (long long)((unsigned)b >> g.l);      // bucket within the row
    const long long h = (a << (g.k - g.l)) + j;
    const unsigned long long lo = g.l ? ((unsigned)b & ((1ull << g.l) - 1)) : 0ull;
    if (r.slot > 0) {
        const long long nb = 1LL << (g.k - g.l);
        const unsigned* d = g.dir + (long long)(r.slot - 1) * (nb + 1) + j;
        ty.touch(d);
        const unsigned s0 = __ldg(d);
        ty.touch(d + 1);
        const unsigned s1 = __ldg(d + 1);
        return lows_search(g, r.P + s0 - h, (long long)s1 - s0 - 1, lo, found, ty);
    }
    long long B = r.P;
    if (j > 0) {
        long long z = near ? scan_near<false>(g, r.P, j - 1, ty) : -1;
        if (z < 0) z = select0(g, h - 1, ty);
        B = z + 1;
    }
    return bucket_search(g, B, h, lo, found, ty);
}

// The exact fallback after trial_cap rejections: inverse transform over the
// cumulative sum of pi in row order (GRAPE, "Efficient sampling for Node2Vec
// RWs"), every fp64 product and sum rounded separately; the uniform comes from
// the Philox block of trial index trial_cap.  Returns a position in N(v).
template <bool WEIGHTED, bool C>
__device__ int ef_fallback(const EFDev& g, long long w, int s, unsigned long long seed, int t,
                           long long off_v, int deg_v, double a_ret, double a_out,
                           unsigned trial_cap, Tally<C>& ty) {
    const uint4 r = trial_block(seed, w, s, trial_cap);
    double total = 0.0;
    for (int j = 0; j < deg_v; ++j) {
        const int x = ef_target(g, select_code(g, off_v + j, ty));
        double a = 1.0;
        if (t >= 0) a = (x == t) ? a_ret : (ef_has_edge(g, t, x, ty) ? 1.0 : a_out);
        const double wv = WEIGHTED ? (double)__ldg(g.weights + off_v + j) : 1.0;
        total = __dadd_rn(total, __dmul_rn(a, wv));
    }
    const unsigned long long r64 = (unsigned long long)r.x | ((unsigned long long)r.y << 32);
    const double u = __dmul_rn(__dmul_rn((double)(r64 >> 11), 0x1p-53), total);
    double run = 0.0;
    for (int j = 0; j < deg_v; ++j) {
        const int x = ef_target(g, select_code(g, off_v + j, ty));
        double a = 1.0;
        if (t >= 0) a = (x == t) ? a_ret : (ef_has_edge(g, t, x, ty) ? 1.0 : a_out);
        const double wv = WEIGHTED ? (double)__ldg(g.weights + off_v + j) : 1.0;
        run = __dadd_rn(run, __dmul_rn(a, wv));
        if (run > u) return j;
    }
    return deg_v - 1;
}

// One thread per walk (grid-stride over the launch's rows).  Rows are staged
// per thread in a 32-byte slot of shared memory and leave as whole sectors
// (put / fill_dead of the CSR engine).
//
// A lane keeps the region (region_of) of its current node v and of the
// previous node t, so proposals and membership tests in a short row scan the
// high bits near a known position instead of going through an index.  On
// undirected graphs a test against a long N(t) searches N(x) for t when that
// row is shorter.  With know_ret set (the in and out thresholds are both below
// 2^32: the return class has the largest bias), a lane whose current row is
// short also finds rt, the position of t in N(v), once per step: a proposal
// idx == rt is then the return and is decided without reading the store, and
// any other proposal whose r2 exceeds both the in and out thresholds is
// rejected without a read (w <= wmax_v).  Every decision is the same function
// of (r2, class, weight) as the oracle's, so the rows do not change.
template <bool WEIGHTED, bool COUNT>
__global__ void __launch_bounds__(kEFThreads)
ef_walk_kernel(EFDev g, WalkConst wc, unsigned trial_cap, int know_ret) {
    Counts<COUNT> cnt;
    cnt.clear();
    Tally<COUNT> ty;
    const unsigned tm1_io = wc.tm1_in > wc.tm1_out ? wc.tm1_in : wc.tm1_out;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x; row < wc.num_walks;
         row += stride) {
        const long long w = wc.walk_base + row;
        int* const rowp = wc.out + row * (long long)wc.walk_len;
        const int len = wc.walk_len;
        Lane L;
        L.flags = (wc.out_vec ? F_VEC : 0u) |
                  ((unsigned)((row * (long long)len) & 7) << F_PHASE_SHIFT);
        const long long i = w % wc.num_starts;
        const long long v0 = wc.starts ? (long long)__ldg(wc.starts + i) : i;
        if (v0 < 0 || v0 >= g.n) {
            atomicOr(g.status, 1);
            fill_dead(L, rowp, 0, len);
            continue;
        }
        cnt.add(C_WALKS);
        put(L, rowp, 0, (int)v0, len);
        int v = (int)v0, t = -1;
        ty.begin();
        Row rv = region_of(g, v, ty);
        Row row_t;                // the previous node's row
        row_t.P = -1;
        row_t.off = 0;
        row_t.deg = 0;
        row_t.slot = 0;
        float wmax_v = 0.0f;
        if (WEIGHTED) {
            ty.touch(g.wmax + v);
            wmax_v = __ldg(g.wmax + v);
        }
        int rt = -1;               // position of t in N(v) when ret_known, -1 when absent
        float w_rt = 0.0f;         // weighted: the weight there
        bool ret_known = false;
        int s = 1;
        for (; s < len && rv.deg > 0; ++s) {
            const bool near_v = region_near(g, rv);
            const bool near_t = region_near(g, row_t);
            int x = -1;
            for (unsigned k = 0; k < trial_cap; ++k) {
                const uint4 r = trial_block(wc.seed, w, s, k);
                cnt.add(C_TRIALS);
                const int idx = scale_index(r.x, r.y, rv.deg);
                if (t >= 0 && ret_known) {
                    if (idx == rt) {                        // the return, decided in registers
                        if (accept_test<WEIGHTED>(r.z, wmax_v, wc.tm1_ret, w_rt)) {
                            x = t;
                            break;
                        }
                        continue;
                    }
                    if (r.z > tm1_io) continue;             // rejected whatever its class
                }
                const long long e = rv.off + idx;
                const int cand = ef_target(g, row_code(g, rv, near_v, e, idx, ty));
                cnt.add(C_GATHERS);
                float wv = 1.0f;
                if (WEIGHTED) {
                    ty.touch(g.weights + e);
                    wv = __ldg(g.weights + e);
                }
                bool acc;
                if (t < 0) {
                    acc = accept_test<WEIGHTED>(r.z, wmax_v, 0xffffffffu, wv);
                } else if (cand == t) {
                    acc = accept_test<WEIGHTED>(r.z, wmax_v, wc.tm1_ret, wv);
                } else {
                    bool acc_in, acc_out;
                    if (WEIGHTED) {
                        weighted_accept2(r.z, wmax_v, wc.tm1_in, wc.tm1_out, wv, acc_in, acc_out);
                    } else {
                        acc_in = r.z <= wc.tm1_in;
                        acc_out = r.z <= wc.tm1_out;
                    }
                    acc = acc_in;
                    if (acc_in != acc_out) {      // only then does the class decide
                        cnt.add(C_SEARCHES);
                        bool in_t;
                        if (near_t || row_t.slot > 0 || !g.undirected) {
                            find_in_row(g, row_t, near_t, t, cand, in_t, ty);
                        } else {
                            // a long N(t) without a directory on an undirected
                            // graph: search the shorter of N(t) and N(x)
                            // (t in N(x) <=> x in N(t))
                            const Row rx = region_of(g, cand, ty);
                            if (rx.deg < row_t.deg)
                                find_in_row(g, rx, region_near(g, rx), cand, t, in_t, ty);
                            else
                                find_in_row(g, row_t, near_t, t, cand, in_t, ty);
                        }
                        acc = in_t ? acc_in : acc_out;
                    }
                }
                if (acc) {
                    x = cand;
                    break;
                }
            }
            if (x < 0) {
                cnt.add(C_FALLBACKS);
                const int j = ef_fallback<WEIGHTED>(g, w, s, wc.seed, t, rv.off, rv.deg, wc.a_ret,
                                                    wc.a_out, trial_cap, ty);
                x = ef_target(g, row_code(g, rv, near_v, rv.off + j, j, ty));
            }
            put(L, rowp, s, x, len);
            cnt.add(C_STEPS);
            t = v;
            row_t = rv;
            v = x;
            ty.begin();
            rv = region_of(g, v, ty);
            if (WEIGHTED) {
                ty.touch(g.wmax + v);
                wmax_v = __ldg(g.wmax + v);
            }
            // locate the return in a short row or one with a directory (a long
            // scan costs more than the reads it would save)
            const bool near_new = region_near(g, rv);
            ret_known = know_ret && rv.deg > 0 && (near_new || rv.slot > 0);
            if (ret_known) {
                bool found;
                const long long at = find_in_row(g, rv, near_new, v, t, found, ty);
                rt = found ? (int)(at - rv.off) : -1;
                if (WEIGHTED && found) {
                    ty.touch(g.weights + at);
                    w_rt = __ldg(g.weights + at);
                }
            }
        }
        if (s < len) fill_dead(L, rowp, s, len);
    }
    if constexpr (COUNT) {
        if (g.counters) {
            cnt.c[C_PROBES] = ty.sectors;        // sectors read, in the probes slot
#pragma unroll
            for (int c = 0; c < C_COUNT; ++c) {
                unsigned long long v = cnt.c[c];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
                if ((threadIdx.x & 31) == 0 && v) atomicAdd(g.counters + c, v);
            }
        }
    }
}

template <bool W, bool C>
cudaError_t launch_walks(const grape_ef_graph* g, const WalkConst& wc, unsigned trial_cap,
                         cudaStream_t stream) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, ef_walk_kernel<W, C>, kEFThreads, 32 * kEFThreads);
    if (e != cudaSuccess) return e;
    per_sm = std::max(per_sm, 1);
    const long long need = (wc.num_walks + kEFThreads - 1) / kEFThreads;
    const int blocks = (int)std::max(1LL, std::min(need, (long long)g->num_sms * per_sm));
    // the return is worth locating when it has the largest bias (both other
    // thresholds below 2^32): other proposals can then be rejected unread
    const int know_ret = (wc.tm1_in < 0xffffffffu && wc.tm1_out < 0xffffffffu) ? 1 : 0;
    ef_walk_kernel<W, C><<<blocks, kEFThreads, 32 * kEFThreads, stream>>>(dev_view(g), wc,
                                                                           trial_cap, know_ret);
    return cudaGetLastError();
}

void free_ef(grape_ef_graph* g) {
    if (!g) return;
    cudaFree(g->low);
    cudaFree(g->high);
    cudaFree(g->ones_idx);
    cudaFree(g->zeros_idx);
    cudaFree(g->weights);
    cudaFree(g->wmax);
    cudaFree(g->rowptr);
    cudaFree(g->dir);
    cudaFree(g->status);
    cudaFree(g->counters);
    delete g;
}

}  // namespace

extern "C" {

grape_status_t grape_ef_graph_create(const int64_t* offsets, const int32_t* dsts,
                                     const float* weights, int64_t num_nodes, int64_t num_entries,
                                     int32_t quantum, uint32_t flags, grape_stream_t stream_,
                                     grape_ef_graph_t** out) {
    if (!out) return GRAPE_ERR_INVALID_ARG;
    *out = nullptr;
    if (!offsets || num_nodes < 1 || num_nodes > 0x7fffffffLL || num_entries < 0 ||
        num_entries >= (1LL << kRowPtrBits) || (num_entries > 0 && !dsts) ||
        quantum < 1 || quantum > (1 << 16) || (quantum & (quantum - 1)) ||
        (flags & ~(GRAPE_UNDIRECTED | GRAPE_VALIDATE)))
        return GRAPE_ERR_INVALID_ARG;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    grape_ef_graph* g = new (std::nothrow) grape_ef_graph();
    if (!g) return GRAPE_ERR_NOMEM;
    g->n = num_nodes;
    g->m = num_entries;
    g->weighted = weights != nullptr;
    g->undirected = (flags & GRAPE_UNDIRECTED) != 0;
    g->quantum = quantum;
    while ((1 << g->qlog) < quantum) ++g->qlog;
    // k = ceil(log2 |V|); u = |V| 2^k; l = floor(log2(u / m)) (0 when u <= m)
    while ((1LL << g->k) < num_nodes) ++g->k;
    g->u = num_nodes << g->k;
    if (num_entries > 0 && g->u > num_entries) {
        const long long ratio = g->u / num_entries;     // floor(log2(u/m)) = floor(log2(floor(u/m)))
        while ((2LL << g->l) <= ratio) ++g->l;
    }
    g->num_zeros = ((g->u - 1) >> g->l) + 1;
    g->high_bits = num_entries + g->num_zeros;
    g->low_words = (num_entries * g->l + 63) / 64;
    g->high_words = (g->high_bits + 63) / 64;
    g->ones_len = (num_entries + quantum - 1) / quantum;
    g->zeros_len = (g->num_zeros + quantum - 1) / quantum;

    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    const size_t low_bytes = 8 * (size_t)(g->low_words + kPadWords);
    const size_t high_bytes = 8 * (size_t)(g->high_words + kPadWords);
    if (e == cudaSuccess) e = cudaMalloc(&g->low, low_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&g->high, high_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&g->ones_idx, 8 * (size_t)std::max<int64_t>(g->ones_len, 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->zeros_idx, 8 * (size_t)g->zeros_len);
    if (e == cudaSuccess && weights) {
        e = cudaMalloc(&g->weights, sizeof(float) * (size_t)std::max<int64_t>(num_entries, 1));
        if (e == cudaSuccess) e = cudaMalloc(&g->wmax, sizeof(float) * (size_t)num_nodes);
    }
    if (e == cudaSuccess) e = cudaMalloc(&g->rowptr, sizeof(long long) * (size_t)(num_nodes + 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->status, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&g->counters, sizeof(unsigned long long) * C_COUNT);
    if (e != cudaSuccess) {
        free_ef(g);
        return cuda_status(e);
    }
    g->structure_bytes = (int64_t)(low_bytes + high_bytes + 8 * (g->ones_len + g->zeros_len) +
                                   8 * (num_nodes + 1));
    g->device_bytes = g->structure_bytes +
                      (weights ? (int64_t)(4 * num_entries + 4 * num_nodes) : 0);
    int host[4] = {0, 0, 0, 0};
    e = cudaMemsetAsync(g->status, 0, sizeof(int) * 4, stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(g->counters, 0, sizeof(unsigned long long) * C_COUNT, stream);
    // 1. offsets, then the rows: the store's layout is computed from the ids,
    //    so the CSR is always checked before anything is written from it
    if (e == cudaSuccess) {
        ef_check_offsets_kernel<<<ef_grid(g->num_sms, num_nodes + 1, 256), 256, 0, stream>>>(
            offsets, num_nodes, num_entries, g->status + 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, g->status, sizeof(int) * 4, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess || host[1] != 0) {
        free_ef(g);
        return e != cudaSuccess ? cuda_status(e) : GRAPE_ERR_INVALID_GRAPH;
    }
    if (e == cudaSuccess) {
        ef_check_rows_kernel<<<ef_grid(g->num_sms, num_nodes * 32, 256), 256, 0, stream>>>(
            offsets, dsts, weights, num_nodes, g->wmax, g->status + 1, g->status + 2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, g->status, sizeof(int) * 4, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess || host[1] != 0) {
        free_ef(g);
        return e != cudaSuccess ? cuda_status(e) : GRAPE_ERR_INVALID_GRAPH;
    }
    g->max_degree = host[2];
    if (g->undirected && (flags & GRAPE_VALIDATE)) {
        ef_check_symmetry_kernel<<<ef_grid(g->num_sms, num_nodes * 32, 256), 256, 0, stream>>>(
            offsets, dsts, weights, num_nodes, g->status + 1);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(host, g->status, sizeof(int) * 4, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess || host[1] != 0) {
            free_ef(g);
            return e != cudaSuccess ? cuda_status(e) : GRAPE_ERR_INVALID_GRAPH;
        }
    }
    // 2. the bit arrays and their indexes
    if (e == cudaSuccess) e = cudaMemsetAsync(g->low, 0, low_bytes, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->high, 0, high_bytes, stream);
    if (e == cudaSuccess && weights && num_entries > 0)
        e = cudaMemcpyAsync(g->weights, weights, sizeof(float) * (size_t)num_entries,
                            cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->rowptr, offsets, sizeof(long long) * (size_t)(num_nodes + 1),
                            cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess) {
        ef_fill_kernel<<<ef_grid(g->num_sms, num_nodes * 32, 256), 256, 0, stream>>>(
            offsets, dsts, num_nodes, g->k, g->l, g->low, g->high);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        ef_index_kernel<<<ef_grid(g->num_sms, g->ones_len + g->zeros_len, 256), 256, 0, stream>>>(
            offsets, dsts, num_nodes, g->k, g->l, g->qlog, g->ones_len, g->zeros_len,
            (unsigned long long)g->u, g->ones_idx, g->zeros_idx);
        e = cudaGetLastError();
    }
    // 3. bucket directories of long rows (counted first, then filled; the
    //    counters double as the two scratch counts and are cleared after)
    if (e == cudaSuccess && g->l <= g->k && num_entries > 0) {
        const long long nb = 1LL << (g->k - g->l);
        unsigned long long count = 0;
        ef_count_long_rows_kernel<<<ef_grid(g->num_sms, num_nodes, 256), 256, 0, stream>>>(
            offsets, num_nodes, nb, g->counters);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&count, g->counters, sizeof(count), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e == cudaSuccess && count > 0 && count <= (unsigned long long)kMaxDirRows) {
            const size_t dir_bytes = sizeof(unsigned) * (size_t)count * (size_t)(nb + 1);
            e = cudaMalloc(&g->dir, dir_bytes);
            if (e == cudaSuccess) {
                ef_fill_dirs_kernel<<<ef_grid(g->num_sms, num_nodes * 32, 256), 256, 0, stream>>>(
                    offsets, dsts, num_nodes, nb, g->l, g->rowptr, g->dir, g->counters + 1);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) {
                g->dir_rows = (int32_t)count;
                g->structure_bytes += (int64_t)dir_bytes;
                g->device_bytes += (int64_t)dir_bytes;
            }
        }
        if (e == cudaSuccess)
            e = cudaMemsetAsync(g->counters, 0, sizeof(unsigned long long) * C_COUNT, stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(g->status, 0, sizeof(int) * 4, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        free_ef(g);
        return cuda_status(e);
    }
    *out = g;
    return GRAPE_OK;
}

void grape_ef_graph_destroy(grape_ef_graph_t* g) {
    if (!g) return;
    cudaSetDevice(g->device);
    cudaDeviceSynchronize();
    free_ef(g);
}

grape_status_t grape_ef_graph_info(const grape_ef_graph_t* g, grape_ef_info_t* info) {
    if (!g || !info) return GRAPE_ERR_INVALID_ARG;
    std::memset(info, 0, sizeof(*info));
    info->num_nodes = g->n;
    info->num_entries = g->m;
    info->universe = g->u;
    info->num_zeros = g->num_zeros;
    info->high_bits = g->high_bits;
    info->low_words = g->low_words;
    info->high_words = g->high_words;
    info->ones_index_len = g->ones_len;
    info->zeros_index_len = g->zeros_len;
    info->structure_bytes = g->structure_bytes;
    info->device_bytes = g->device_bytes;
    info->code_bits = g->k;
    info->low_bits = g->l;
    info->quantum = g->quantum;
    info->weighted = g->weighted ? 1 : 0;
    info->max_degree = g->max_degree;
    info->directory_rows = g->dir_rows;
    return GRAPE_OK;
}

grape_status_t grape_ef_graph_export(const grape_ef_graph_t* g, uint64_t* low, uint64_t* high,
                                     int64_t* ones_index, int64_t* zeros_index,
                                     grape_stream_t stream_) {
    if (!g) return GRAPE_ERR_INVALID_ARG;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    cudaError_t e = cudaSuccess;
    if (low && g->low_words)
        e = cudaMemcpyAsync(low, g->low, 8 * (size_t)g->low_words, cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess && high && g->high_words)
        e = cudaMemcpyAsync(high, g->high, 8 * (size_t)g->high_words, cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess && ones_index && g->ones_len)
        e = cudaMemcpyAsync(ones_index, g->ones_idx, 8 * (size_t)g->ones_len,
                            cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess && zeros_index && g->zeros_len)
        e = cudaMemcpyAsync(zeros_index, g->zeros_idx, 8 * (size_t)g->zeros_len,
                            cudaMemcpyDeviceToDevice, stream);
    return cuda_status(e);
}

grape_status_t grape_ef_select(const grape_ef_graph_t* g, const int64_t* idx, int64_t n,
                               int64_t* out, grape_stream_t stream_) {
    if (!g || n < 0 || (n > 0 && (!idx || !out))) return GRAPE_ERR_INVALID_ARG;
    if (n == 0) return GRAPE_OK;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    ef_select_kernel<<<ef_grid(g->num_sms, n, 256), 256, 0, stream>>>(
        dev_view(g), reinterpret_cast<const long long*>(idx), n, reinterpret_cast<long long*>(out));
    return cuda_status(cudaGetLastError());
}

grape_status_t grape_ef_rank(const grape_ef_graph_t* g, const int64_t* values, int64_t n,
                             int64_t* out, grape_stream_t stream_) {
    if (!g || n < 0 || (n > 0 && (!values || !out))) return GRAPE_ERR_INVALID_ARG;
    if (n == 0) return GRAPE_OK;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    ef_rank_kernel<<<ef_grid(g->num_sms, n, 256), 256, 0, stream>>>(
        dev_view(g), reinterpret_cast<const long long*>(values), n,
        reinterpret_cast<long long*>(out));
    return cuda_status(cudaGetLastError());
}

grape_status_t grape_ef_walks(const grape_ef_graph_t* g, const int32_t* starts,
                              int64_t num_starts, int32_t walk_len, int32_t walks_per_node,
                              double p, double q, uint64_t seed, int64_t trial_cap,
                              int32_t* out, grape_stream_t stream_) {
    if (!g || trial_cap < 0 || trial_cap > 0x7fffffffLL) return GRAPE_ERR_INVALID_ARG;
    WalkConst wc;
    grape_status_t st = make_walk_const_n(g->n, starts, num_starts, walk_len, walks_per_node, p,
                                          q, seed, out, &wc);
    if (st != GRAPE_OK) return st;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    cudaError_t e;
    const unsigned cap = (unsigned)trial_cap;
    if (g->counting) {
        e = g->weighted ? launch_walks<true, true>(g, wc, cap, stream)
                        : launch_walks<false, true>(g, wc, cap, stream);
    } else {
        e = g->weighted ? launch_walks<true, false>(g, wc, cap, stream)
                        : launch_walks<false, false>(g, wc, cap, stream);
    }
    return cuda_status(e);
}

grape_status_t grape_ef_stream_status(const grape_ef_graph_t* g, grape_stream_t stream_) {
    if (!g) return GRAPE_ERR_INVALID_ARG;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    int word = 0;
    cudaError_t e = cudaMemcpyAsync(&word, g->status, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->status, 0, sizeof(int), stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_status(e);
    return word ? GRAPE_ERR_DEVICE : GRAPE_OK;
}

grape_status_t grape_ef_counters_enable(grape_ef_graph_t* g, int32_t enable) {
    if (!g) return GRAPE_ERR_INVALID_ARG;
    g->counting = enable != 0;
    return cuda_status(cudaMemset(g->counters, 0, sizeof(unsigned long long) * C_COUNT));
}

grape_status_t grape_ef_counters_read(grape_ef_graph_t* g, grape_ef_counters_t* out) {
    if (!g || !out) return GRAPE_ERR_INVALID_ARG;
    unsigned long long c[C_COUNT];
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(c, g->counters, sizeof(c), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(g->counters, 0, sizeof(c));
    if (e != cudaSuccess) return cuda_status(e);
    out->steps = (int64_t)c[C_STEPS];
    out->trials = (int64_t)c[C_TRIALS];
    out->codes_read = (int64_t)c[C_GATHERS];
    out->membership_tests = (int64_t)c[C_SEARCHES];
    out->sectors = (int64_t)c[C_PROBES];
    out->fallbacks = (int64_t)c[C_FALLBACKS];
    out->walks = (int64_t)c[C_WALKS];
    return GRAPE_OK;
}

}  // extern "C"
