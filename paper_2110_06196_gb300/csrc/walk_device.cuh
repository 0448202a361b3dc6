// walk_device.cuh -- device side of the node2vec walk engine (sm_103a).
//
// One lane owns one walk at a time.  All three launch shapes share the engine
// `walk_loop`: per call (grid-stride over walk ids), batched (a queue of
// (request, walk range) entries), and served (the same queue, fed while the
// kernel runs).
//
// The engine is a per-lane state machine that issues at most one dependent
// gather per lane per loop iteration (one 32-byte sector at most) and
// consumes it in the next iteration.
// A lane deep in a membership search on a hub list therefore does not hold up
// the other 31 lanes of its warp.  Proposal entries carry the proposed node's
// degree and row offset ("edge-inlined records", see GraphDev::fat), so an
// accepted proposal needs no second gather.  Two kinds of proposal need no
// gather at all: the return (the lane knows the position of t in N(v) and the
// weight of that entry) and, once the return is ruled out, a proposal whose
// acceptance uniform is at or above every other class's threshold (rejected
// whatever its target and weight, since w <= wmax).  A step is therefore
// (read proposals + probes) dependent gathers.  Phases:
//   CAND    a proposal entry arrived: classify and decide, or start a search
//   SEARCH  a probe arrived (the aligned 32-byte sector of the list around the
//           interpolated position or the midpoint): narrow or finish
//
// Per trial (GRAPE, Methods, eq. alphaRW with the beta/gamma split of eqs. alpha, beta):
//   Philox4x32-10(key = seed, ctr = (w, s, k)) -> r0..r3
//   e = off_v + mulhi64(r1:r0, deg_v); x = dsts[e] (+ w_vx)
//   class: x == t -> return (1/p); x in N(t) -> in (1); else out (1/q)
//   accept iff r2 < T_class  (weighted: r2 * wmax_v < T_class * w_vx, exactly)
// The membership search runs only when the in and out thresholds give different
// answers for this r2.  The decision is the same function of (r2, class) as
// always, so the bytes written do not change.
#pragma once
#include <cstdint>
#include <cuda/atomic>
#include <cuda_runtime.h>

namespace grape {

constexpr unsigned FULL = 0xffffffffu;

// Node record: row offset, degree, largest row weight (fp32 bits), 16 bytes.
// One aligned 16-byte load per visited node.
struct __align__(16) NodeRec {
    long long off;
    int deg;
    float wmax;
};

enum Counter : int {
    C_STEPS = 0, C_TRIALS, C_GATHERS, C_SEARCHES, C_PROBES, C_FALLBACKS, C_WALKS, C_FILTERED,
    C_PIVOT_PROBES, C_HASH_PROBES, C_COUNT
};

// Neighbour filters (unweighted graphs): a 96-bit one-hash Bloom filter of each
// row, bit filter_bit(y) set for every y in the row.  A clear bit proves that y
// is not in the row.  Built once with the graph; the proposal entry of x
// carries the filter of N(x), and a lane keeps the filters of N(v) and N(t).
__host__ __device__ __forceinline__ int filter_bit(int y) {
    const unsigned h = (unsigned)y * 0x9E3779B1u;
    return (int)(((unsigned long long)h * 96ull) >> 32);
}

// Weighted entries have room for one 32-bit pair filter (undirected graphs).
__host__ __device__ __forceinline__ int filter_bit32(int y) {
    return (int)(((unsigned)y * 0x9E3779B1u) >> 27);
}

__host__ __device__ __forceinline__ bool filter_has(unsigned f0, unsigned f1, unsigned f2, int b) {
    const unsigned word = b < 32 ? f0 : (b < 64 ? f1 : f2);
    return (word >> (b & 31)) & 1u;
}

// Edge hash: membership of a pair in the graph by one 32-byte read.
// The key of a pair (a, b) is a * 2^k + b over K = 2k bits, with k bits per node
// id and (undirected graphs) a <= b.  A bijection of the K-bit keys (xor-shifts
// and multiplications by odd constants, modulo 2^K) spreads them; its top B
// bits pick a bucket of eight 32-bit slots, and its low K - B bits, plus one,
// are what the bucket stores (0 marks an empty slot).  Because the map is a
// bijection, (bucket, remainder) identifies the pair exactly.  A bucket that
// received more than eight pairs holds kHashOverflow in its last slot: a pair
// not found there must be searched in the sorted rows.
constexpr unsigned kHashOverflow = 0xffffffffu;

__host__ __device__ __forceinline__ unsigned long long edge_hash_mix(unsigned long long x, int K) {
    const unsigned long long mask = (K >= 64) ? ~0ull : ((1ull << K) - 1ull);
    const int r = K / 2 + 1;
    x &= mask;
    x ^= x >> r;
    x = (x * 0x9E3779B97F4A7C15ull) & mask;
    x ^= x >> (K / 3 + 1);
    x = (x * 0xD6E8FEB86659FD93ull) & mask;
    x ^= x >> r;
    return x;
}

struct GraphDev {
    const int4* rec;            // [n] NodeRec viewed as int4
    const int* dsts;            // [m + 8] sorted rows (membership search, fallback)
    // proposal entries, one 32-byte sector per CSR entry e (row v, target x):
    //   fat[2e]     = {x, deg_x, off_x lo, off_x hi}
    //   fat[2e + 1] = weighted:   {w_vx bits, wmax_x bits, rev, w_xv bits}
    //                 unweighted: {filter of N(x) bits 0-31, bits 32-63, rev, bits 64-95}
    // rev = position of v in N(x) (-1 when absent), w_xv the weight there
    const int4* fat;
    // sector pivots: piv[j] = dsts[8 j], the first id of each aligned 32-byte
    // sector of dsts ([ceil(m / 8) + 8], padded), or nullptr
    const int* piv;
    // edge hash: [2^eh_b buckets][8] slots, or nullptr; eh_k bits per node id
    const unsigned* eh;
    int eh_k, eh_b;
    // 1 (undirected graphs with an edge hash): an entry (v -> x) holds a filter
    // of N(v) n N(x), 96 bits in an unweighted entry, 32 bits in the last word
    // of a weighted one (in place of the reverse weight, equal to w_vx on an
    // undirected graph); 0: an unweighted entry holds a filter of N(x) and a
    // weighted one none
    int pair_filters;
    long long n;
    int* status;                // device status word (1 = bad start id)
    unsigned long long* counters;  // [C_COUNT] or nullptr
    int undirected;
};

// Per-request constants.  Thresholds are stored as T - 1 (T in [1, 2^32]):
// r2 < T  <=>  r2 <= T - 1.
struct __align__(16) WalkConst {
    const int* starts;          // nullptr: start i is node i
    int* out;                   // rows [num_walks][walk_len]
    long long num_starts;
    long long num_walks;        // rows of this launch
    long long walk_base;        // walk id of row 0 (a shard of a larger job), else 0
    unsigned long long seed;
    unsigned tm1_ret, tm1_in, tm1_out;
    int walk_len;
    double a_ret, a_out;        // 1/p and 1/q for the exact fallback
    int out_vec;                // 1 when out is 32-byte aligned (whole-sector row stores)
    int suss_k;                 // approximated walks: SUSS sub-sample size (0: exact walks)
};
static_assert(sizeof(WalkConst) % 16 == 0, "WalkConst is loaded as int4 words");

// Queue entry for batched and served launches: walks [walk_lo, walk_lo + count)
// of request `req`.
struct __align__(16) Chunk {
    long long walk_lo;
    int count;
    int req;
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): ten rounds of two
// 32x32->64 products with multipliers 0xD2511F53 / 0xCD9E8D57; the key is
// bumped by 0x9E3779B9 / 0xBB67AE85 between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        if (i > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        // one 32x32 -> 64 product each (high and low words from one multiply)
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((unsigned)(p1 >> 32) ^ c.y ^ k.x, (unsigned)p1,
                       (unsigned)(p0 >> 32) ^ c.w ^ k.y, (unsigned)p0);
    }
    return c;
}

// The round keys of one seed: round i uses (seed lo + i 0x9E3779B9,
// seed hi + i 0xBB67AE85).  A per-call launch passes them as a kernel parameter,
// so the rounds read them from the constant bank instead of adding them up.
struct RoundKeys {
    unsigned k[20];
};

__host__ __device__ inline RoundKeys round_keys(unsigned long long seed) {
    RoundKeys rk;
    unsigned a = (unsigned)seed, b = (unsigned)(seed >> 32);
    for (int i = 0; i < 10; ++i) {
        rk.k[2 * i] = a;
        rk.k[2 * i + 1] = b;
        a += 0x9E3779B9u;
        b += 0xBB67AE85u;
    }
    return rk;
}

// philox4x32_10 with the round keys given.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const RoundKeys& rk) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((unsigned)(p1 >> 32) ^ c.y ^ rk.k[2 * i], (unsigned)p1,
                       (unsigned)(p0 >> 32) ^ c.w ^ rk.k[2 * i + 1], (unsigned)p0);
    }
    return c;
}

__device__ __forceinline__ uint4 trial_block(unsigned long long seed, long long w, int s,
                                             unsigned k) {
    const unsigned long long uw = (unsigned long long)w;
    return philox4x32_10(make_uint4((unsigned)uw, (unsigned)(uw >> 32), (unsigned)s, k),
                         make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
}

// floor((hi:lo) * n / 2^64) for n < 2^31: the high word of a 64 x 32-bit
// product, from two 32 x 32 -> 64 products (exact: the sum stays below 2^64).
__device__ __forceinline__ int scale_index(unsigned lo, unsigned hi, int n) {
    const unsigned long long a = (unsigned long long)lo * (unsigned)n;
    const unsigned long long b = (unsigned long long)hi * (unsigned)n + (a >> 32);
    return (int)(b >> 32);
}

// Approximated walks (GRAPE, Methods, "Approximated RWs"): at a node of degree
// deg > k a step draws among k candidates, one per bucket of row positions
// [floor(b deg / k), floor((b + 1) deg / k)), the member of bucket b taken
// from the step's Philox block of trial index 2^31 + b (fixed for the step).
constexpr unsigned kSussTrialBase = 0x80000000u;

__device__ __forceinline__ int suss_pos(unsigned long long seed, long long w, int s, int b,
                                        int deg, int k) {
    const long long lo = (long long)b * deg / k;
    const long long hi = (long long)(b + 1) * deg / k;
    const uint4 u = trial_block(seed, w, s, kSussTrialBase | (unsigned)b);
    return (int)lo + scale_index(u.x, u.y, (int)(hi - lo));
}

// One 32-byte sector in a single 256-bit read-only load (sm_100 and later):
// the first 16 bytes to a, the last 16 to b.  p must be 32-byte aligned.
__device__ __forceinline__ void ld_sector(const void* p, int4& a, int4& b) {
    asm volatile("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z),
                   "=r"(b.w)
                 : "l"(p));
}

// Is key in the sorted list a[0, n)?  Lane-local binary search (used by the
// exact fallback, which runs outside the pipelined state machine).
__device__ __forceinline__ bool lane_search(const int* __restrict__ a, int n, int key) {
    if (n <= 0) return false;
    const int* b = a;
    while (n > 1) {
        const int half = n >> 1;
        b = (__ldg(b + half) <= key) ? b + half : b;
        n -= half;
    }
    return __ldg(b) == key;
}

// ---------------------------------------------------------------------------
// Lane state
// ---------------------------------------------------------------------------
//   PH_DRAW  nothing arrived: draw the next proposal
//   PH_RET   the return was drawn and accepted (no read): move back to t
enum Phase : int { PH_START = 0, PH_CAND = 1, PH_SEARCH = 2, PH_DRAW = 3, PH_RET = 4 };

// Proposals a lane may draw in one iteration.  Those decided without a read
// (returns, certain rejections) let the lane go on to the next one; the bound
// keeps the lanes of a warp in step.
constexpr int kDrawsPerIter = 2;

struct Lane {
    long long w;          // walk id (Philox counter words 0-1)
    long long off_v;
    unsigned k;           // trial index within the step
    int s;                // index of the entry being produced (1 .. len-1)
    int v, t;             // current and previous node (t < 0 on the first step)
    int deg_v;
    float wmax_v;
    int rt;               // position of t in N(v); -1 when t is not in N(v) or there is no t
    float wr;             // weighted: the weight of that entry (v -> t)
    int pidx;             // position in N(v) of the proposal in flight or under search
    // the rest of t's state lives in shared memory (TRec)
    int req;              // request index (batched / served), -1 for per-call
    int phase;
    unsigned r2;          // acceptance uniform of the proposal in flight
    unsigned flags;       // F_* bits below
    // the proposal under a membership search (its entry waits in shared memory)
    int x;
    // membership search over dsts[sb, sb + sn) for x (or for t, with F_KEY_T);
    // sd = (start of the probe block in flight) - sb; every value before the
    // range is <= vlo and every value after it >= vhi (vlo < key < vhi)
    long long sb;
    int sn;
    int sd;
    int vlo, vhi;
};

enum : unsigned {
    F_ACC_IN = 1u,        // accept if x is in N(t)
    F_ACC_OUT = 2u,       // accept if x is not in N(t)
    F_VEC = 8u,           // output rows may be written in whole 32-byte sectors
    F_KEY_T = 16u,        // the search looks for t in N(x) (else for x in N(t))
    F_BISECT = 32u,       // the next probe bisects (the last interpolated one did not halve)
    F_PIV = 64u,          // the search runs over the list's sector pivots, not the list
    F_WARPQ = 128u,       // a new search waits for the warp to narrow its list (no probe yet)
    F_HASH = 4u,          // the probe in flight is the pair's edge-hash bucket
    // bits 8-10: offset of the row's first entry inside its 32-byte sector
};
constexpr int F_PHASE_SHIFT = 8;
static_assert(((F_ACC_IN | F_ACC_OUT | F_HASH | F_VEC | F_KEY_T | F_BISECT | F_PIV | F_WARPQ) &
               (7u << F_PHASE_SHIFT)) == 0,
              "lane flags must leave the output phase bits (8-10) alone");

// Work counters, kept only by the counting instantiation of the kernels.
template <bool ON>
struct Counts {
    unsigned c[C_COUNT];
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int i = 0; i < C_COUNT; ++i) c[i] = 0;
    }
    __device__ __forceinline__ void add(int i) { c[i]++; }
    __device__ __forceinline__ void add_n(int i, unsigned n) { c[i] += n; }
};
template <>
struct Counts<false> {
    __device__ __forceinline__ void clear() {}
    __device__ __forceinline__ void add(int) {}
    __device__ __forceinline__ void add_n(int, unsigned) {}
};

// The previous node's record and the entry the walk arrived by.  Read only
// by membership searches, returns and the fallback, so it waits in shared
// memory instead of registers.
struct __align__(16) TRec {
    long long off_t;
    int deg_t;
    float wmax_t;
    int jv;               // position of v in N(t)
    float wj;             // weighted: the weight there (t -> v)
    unsigned long long ticket;   // lane 0 only: the warp's served-queue ticket (QueueFeed)
};

// The constants of the request a lane's walk belongs to (batched and served
// launches, where lanes of one warp may serve different requests).  Kept in
// shared memory instead of registers.
struct __align__(16) WRec {
    unsigned long long seed;
    int* row;             // this walk's output row
    unsigned tm1_ret, tm1_in, tm1_out;
    int len;
};

// Unweighted graphs: the neighbour filters of the current and previous node.
struct __align__(16) FRec {
    unsigned fv[3];       // filter of N(v) (all ones when unknown: the walk's start)
    unsigned pad0;
    unsigned ft[3];       // filter of N(t)
    unsigned pad1;
};

// Dynamic shared memory per lane: a 32-byte output staging slot, the 32-byte
// entry of the proposal under a membership search, the lane's TRec, its WRec
// and its FRec.
constexpr int kLaneSharedBytes = 160;

// Row writer.  Each lane stages its row's entries in its own 32-byte slot of
// shared memory; when an entry completes a 32-byte sector that lies inside the
// row, the sector leaves as two 16-byte stores, so DRAM sees whole sectors.
// Entries in the (at most two) sectors a row shares with its neighbours are
// stored singly.
__device__ __forceinline__ int* out_stage() {
    extern __shared__ int4 stage_words[];
    return reinterpret_cast<int*>(stage_words) + 8 * threadIdx.x;
}

__device__ __forceinline__ int4* parked_entry() {
    extern __shared__ int4 stage_words[];
    return stage_words + 2 * blockDim.x + 2 * threadIdx.x;
}

__device__ __forceinline__ TRec* trec() {
    extern __shared__ int4 stage_words[];
    return reinterpret_cast<TRec*>(stage_words + 4 * blockDim.x) + threadIdx.x;
}

constexpr unsigned long long kNoTicket = ~0ull;

// The warp's pending served-queue ticket, kept by lane 0 in its TRec.
__device__ __forceinline__ unsigned long long* warp_ticket() {
    extern __shared__ int4 stage_words[];
    return &(reinterpret_cast<TRec*>(stage_words + 4 * blockDim.x) + (threadIdx.x & ~31u))->ticket;
}

__device__ __forceinline__ WRec* wrec() {
    extern __shared__ int4 stage_words[];
    return reinterpret_cast<WRec*>(stage_words + 6 * blockDim.x) + threadIdx.x;
}

__device__ __forceinline__ FRec* frec() {
    extern __shared__ int4 stage_words[];
    return reinterpret_cast<FRec*>(stage_words + 8 * blockDim.x) + threadIdx.x;
}

__device__ __forceinline__ void put(const Lane& L, int* row, int s, int val, int len) {
    const int j = (int)(((L.flags >> F_PHASE_SHIFT) + (unsigned)s) & 7u);  // slot in the sector
    const int sec0 = s - j;                                                 // sector's first entry
    if (!(L.flags & F_VEC) || sec0 < 0 || sec0 + 8 > len) {
        row[s] = val;                       // a sector shared with a neighbouring row
        return;
    }
    int* st = out_stage();
    st[j] = val;
    if (j == 7) {
        const int4* s4 = reinterpret_cast<const int4*>(st);
        int4* g4 = reinterpret_cast<int4*>(row + sec0);
        g4[0] = s4[0];
        g4[1] = s4[1];
    }
}

// Entries from..len-1 are -1: staged up to the next sector boundary, then whole
// sectors as two 16-byte stores each, then the ragged end singly.
__device__ __forceinline__ void fill_dead(const Lane& L, int* row, int from, int len) {
    int s = from;
    while (s < len && (((L.flags >> F_PHASE_SHIFT) + (unsigned)s) & 7u) != 0) put(L, row, s++, -1, len);
    if (L.flags & F_VEC) {
        const int4 m1 = make_int4(-1, -1, -1, -1);
        for (; s + 8 <= len; s += 8) {
            int4* g4 = reinterpret_cast<int4*>(row + s);
            g4[0] = m1;
            g4[1] = m1;
        }
    }
    for (; s < len; ++s) row[s] = -1;
}

__device__ __forceinline__ NodeRec decode_rec(int4 r) {
    NodeRec n;
    n.off = (long long)(((unsigned long long)(unsigned)r.y << 32) | (unsigned)r.x);
    n.deg = r.z;
    n.wmax = __int_as_float(r.w);
    return n;
}

__device__ __forceinline__ NodeRec load_rec(const GraphDev& g, int x) {
    return decode_rec(__ldg(g.rec + x));
}

// Weighted acceptance, exact: r2 * wmax < T * w in real arithmetic, with
// T = tm1 + 1 <= 2^32, r2 < 2^32 and 0 < w <= wmax finite fp32.  Writing an fp32
// value as M * 2^E (M < 2^24 an integer) turns the test into
// (r2 * M_wmax) << (E_wmax - E_w) < T * M_w, evaluated in integers.
__device__ __forceinline__ bool weighted_accept(unsigned r2, float wmax, unsigned tm1, float w) {
    const unsigned b1 = __float_as_uint(wmax), b2 = __float_as_uint(w);
    const unsigned e1 = (b1 >> 23) & 0xffu, e2 = (b2 >> 23) & 0xffu;
    const unsigned long long m1 = (b1 & 0x7fffffu) | (e1 ? 0x800000u : 0u);
    const unsigned long long m2 = (b2 & 0x7fffffu) | (e2 ? 0x800000u : 0u);
    const int d = (int)(e1 ? e1 : 1u) - (int)(e2 ? e2 : 1u);   // >= 0 since w <= wmax
    const unsigned long long lhs = (unsigned long long)r2 * m1;        // < 2^56
    const unsigned long long rhs = (unsigned long long)tm1 * m2 + m2;      // (tm1 + 1) m2 <= 2^56
    if (lhs == 0) return rhs != 0;
    if (d >= 64) return false;
    if (d > 0 && (lhs >> (64 - d)) != 0) return false;
    return (lhs << d) < rhs;
}

// The same test against two thresholds at once (the in and out classes):
// r2 * wmax is split and shifted once.
__device__ __forceinline__ void weighted_accept2(unsigned r2, float wmax, unsigned tm1_a,
                                                 unsigned tm1_b, float w, bool& acc_a,
                                                 bool& acc_b) {
    const unsigned b1 = __float_as_uint(wmax), b2 = __float_as_uint(w);
    const unsigned e1 = (b1 >> 23) & 0xffu, e2 = (b2 >> 23) & 0xffu;
    const unsigned long long m1 = (b1 & 0x7fffffu) | (e1 ? 0x800000u : 0u);
    const unsigned long long m2 = (b2 & 0x7fffffu) | (e2 ? 0x800000u : 0u);
    const int d = (int)(e1 ? e1 : 1u) - (int)(e2 ? e2 : 1u);
    const unsigned long long lhs = (unsigned long long)r2 * m1;
    const unsigned long long rhs_a = (unsigned long long)tm1_a * m2 + m2;
    const unsigned long long rhs_b = (unsigned long long)tm1_b * m2 + m2;
    if (lhs == 0) {
        acc_a = rhs_a != 0;
        acc_b = rhs_b != 0;
        return;
    }
    if (d >= 64 || (d > 0 && (lhs >> (64 - d)) != 0)) {
        acc_a = acc_b = false;
        return;
    }
    const unsigned long long l = lhs << d;
    acc_a = l < rhs_a;
    acc_b = l < rhs_b;
}

template <bool WEIGHTED>
__device__ __forceinline__ bool accept_test(unsigned r2, float wmax, unsigned tm1, float w) {
    if (WEIGHTED) return weighted_accept(r2, wmax, tm1, w);
    return r2 <= tm1;
}

// Exact fallback after trial_cap rejections: inverse transform over the
// cumulative sum of pi in row order (GRAPE, "Efficient sampling for Node2Vec
// RWs"), in fp64 with every product and sum rounded separately.
// Returns the position of the drawn node in N(v).  Under SUSS (suss_k > 0
// and deg_v > suss_k) the cumulative sum runs over the k candidates of the
// step's sub-sample, in bucket order.
template <bool WEIGHTED>
__device__ __forceinline__ int exact_fallback(const GraphDev& g, const Lane& L, unsigned long long seed,
                              double a_ret, double a_out, unsigned trial_cap, int suss_k) {
    const uint4 r = trial_block(seed, L.w, L.s, trial_cap);
    const bool first = (L.t < 0);
    const TRec* tr = trec();
    const int* const nt = first ? g.dsts : g.dsts + tr->off_t;
    const int deg_t = first ? 0 : tr->deg_t;
    const bool suss = suss_k > 0 && L.deg_v > suss_k;
    const int m = suss ? suss_k : L.deg_v;
    double total = 0.0;
    for (int j = 0; j < m; ++j) {
        const int pos = suss ? suss_pos(seed, L.w, L.s, j, L.deg_v, suss_k) : j;
        const long long e = L.off_v + pos;
        const int x = __ldg(g.dsts + e);
        double a = 1.0;
        if (!first) {
            if (x == L.t) a = a_ret;
            else if (!lane_search(nt, deg_t, x)) a = a_out;
        }
        const double w = WEIGHTED ? (double)__int_as_float(__ldg(&g.fat[2 * e + 1].x)) : 1.0;
        total = __dadd_rn(total, __dmul_rn(a, w));
    }
    const unsigned long long r64 = (unsigned long long)r.x | ((unsigned long long)r.y << 32);
    const double u = __dmul_rn(__dmul_rn((double)(r64 >> 11), 0x1p-53), total);
    double run = 0.0;
    for (int j = 0; j < m; ++j) {
        const int pos = suss ? suss_pos(seed, L.w, L.s, j, L.deg_v, suss_k) : j;
        const long long e = L.off_v + pos;
        const int x = __ldg(g.dsts + e);
        double a = 1.0;
        if (!first) {
            if (x == L.t) a = a_ret;
            else if (!lane_search(nt, deg_t, x)) a = a_out;
        }
        const double w = WEIGHTED ? (double)__int_as_float(__ldg(&g.fat[2 * e + 1].x)) : 1.0;
        run = __dadd_rn(run, __dmul_rn(a, w));
        if (run > u) return pos;
    }
    return suss ? suss_pos(seed, L.w, L.s, m - 1, L.deg_v, suss_k) : L.deg_v - 1;
}

// Start the walk of row `row` (walk id walk_base + row) of request wc on this
// lane.  Returns true when the walk needs transitions (phase PH_START); false
// when it is already complete (length 1, dead start, or a start id out of
// range, whose row is all -1 and which sets the status word).
__device__ __forceinline__ bool begin_walk(const GraphDev& g, const WalkConst& wc, int req,
                                           long long row, Lane& L) {
    const long long w = wc.walk_base + row;
    int* const rowp = wc.out + row * (long long)wc.walk_len;
    L.w = w;
    L.req = req;
    L.flags = (wc.out_vec ? F_VEC : 0u) |
              ((unsigned)((row * (long long)wc.walk_len) & 7) << F_PHASE_SHIFT);
    const long long i = w % wc.num_starts;
    const long long v0 = wc.starts ? (long long)__ldg(wc.starts + i) : i;
    if (v0 < 0 || v0 >= g.n) {
        atomicOr(g.status, 1);
        fill_dead(L, rowp, 0, wc.walk_len);
        return false;
    }
    put(L, rowp, 0, (int)v0, wc.walk_len);
    {
        FRec* fr = frec();                 // the start's filter is not at hand: all ones
        fr->fv[0] = fr->fv[1] = fr->fv[2] = ~0u;
    }
    const NodeRec r = load_rec(g, (int)v0);
    L.v = (int)v0;
    L.t = -1;
    L.rt = -1;
    L.off_v = r.off;
    L.deg_v = r.deg;
    L.wmax_v = r.wmax;
    L.s = 1;
    L.k = 0;
    L.phase = PH_START;
    L.flags &= ~(F_KEY_T | F_ACC_IN | F_ACC_OUT | F_BISECT | F_PIV | F_WARPQ);
    if (wc.walk_len <= 1) return false;
    if (r.deg == 0) {
        fill_dead(L, rowp, 1, wc.walk_len);
        return false;
    }
    return true;
}

__device__ __forceinline__ void flush_counts(const GraphDev&, Counts<false>&) {}

__device__ __forceinline__ void flush_counts(const GraphDev& g, Counts<true>& c) {
    if (g.counters == nullptr) return;
#pragma unroll
    for (int i = 0; i < C_COUNT; ++i) {
        unsigned long long x = c.c[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd(g.counters + i, x);
    }
}

// ---------------------------------------------------------------------------
// Walk sources
// ---------------------------------------------------------------------------

// Completion signal of a per-call launch cut into slices of walk rows: every
// slice has a device counter of finished walks and a flag in mapped host
// memory, raised when its last walk is written, so the host can copy a
// slice out while the launch goes on.  walks_per_slice = 0: no slices.
struct SliceSink {
    unsigned long long* done;    // [slices] finished walks (device)
    unsigned* flags;             // [slices] host-mapped: 1 once the slice's rows are written
    long long walks_per_slice;
    long long num_walks;         // rows of the launch
};

// A lane's running count of finished walks in one slice (per-call launches do
// not use the WRec slot, so the tally lives there).
struct __align__(16) SliceTally {
    long long slice;
    unsigned count;
};

__device__ __forceinline__ SliceTally* slice_tally() {
    extern __shared__ int4 stage_words[];
    return reinterpret_cast<SliceTally*>(stage_words + 6 * blockDim.x) + threadIdx.x;
}

// Add the lane's tally to its slice's counter.  The add is a release, so this
// lane's rows are visible before they count; the add that completes the slice
// is followed by an acquire fence (every other lane's rows are then visible)
// and a system fence before the host-visible flag goes up.
__device__ __forceinline__ void flush_slice(const SliceSink& sk, SliceTally* st) {
    if (st->count == 0 || st->slice < 0) return;
    const long long sl = st->slice;
    const long long left = sk.num_walks - sl * sk.walks_per_slice;
    const unsigned long long size =
        (unsigned long long)(left < sk.walks_per_slice ? left : sk.walks_per_slice);
    cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> c(sk.done[sl]);
    const unsigned long long prev = c.fetch_add(st->count, cuda::memory_order_release);
    if (prev + st->count == size) {
        cuda::atomic_thread_fence(cuda::memory_order_acquire, cuda::thread_scope_device);
        __threadfence_system();
        *(volatile unsigned*)(sk.flags + sl) = 1u;
    }
    st->count = 0;
}

// Record the request constants of row `row` of wc for this lane (queue feeds).
__device__ __forceinline__ void set_wrec(const WalkConst& wc, long long row) {
    WRec r;
    r.seed = wc.seed;
    r.row = wc.out + row * (long long)wc.walk_len;
    r.tm1_ret = wc.tm1_ret;
    r.tm1_in = wc.tm1_in;
    r.tm1_out = wc.tm1_out;
    r.len = wc.walk_len;
    *wrec() = r;
}

// Per call: lane j of the grid takes walks j, j + stride, j + 2 * stride, ...
// SUSS: the approximated-walk instantiation (exact walks compile it out).
template <bool SUSS>
struct GridFeed {
    const WalkConst* wc;     // kernel-parameter copy
    const RoundKeys* rk;     // kernel-parameter copy: the Philox round keys of wc->seed
    const SliceSink* sink;   // kernel-parameter copy: slice completion (walks_per_slice 0: none)
    long long next;
    long long stride;

    // The Philox block of trial k of the lane's current step.
    __device__ __forceinline__ uint4 trial(const Lane& L, unsigned k) const {
        const unsigned long long uw = (unsigned long long)L.w;
        return philox4x32_10_rk(make_uint4((unsigned)uw, (unsigned)(uw >> 32), (unsigned)L.s, k),
                                *rk);
    }

    // Per-call constants are uniform: read them from the kernel parameters
    // (constant bank) instead of holding them in every lane's registers.
    __device__ __forceinline__ unsigned long long seed(const Lane&) const { return wc->seed; }
    __device__ __forceinline__ int len(const Lane&) const { return wc->walk_len; }
    __device__ __forceinline__ unsigned tm1_ret(const Lane&) const { return wc->tm1_ret; }
    __device__ __forceinline__ unsigned tm1_in(const Lane&) const { return wc->tm1_in; }
    __device__ __forceinline__ unsigned tm1_out(const Lane&) const { return wc->tm1_out; }
    __device__ __forceinline__ int suss_k(const Lane&) const { return SUSS ? wc->suss_k : 0; }
    // the row of walk id w is row w - walk_base of this call's output
    __device__ __forceinline__ int* row(const Lane& L) const {
        return wc->out + (L.w - wc->walk_base) * (long long)wc->walk_len;
    }

    // Rows of one lane finish in increasing walk-id order (grid stride), so a
    // lane's tally moves through the slices in order and is added to a
    // slice's counter when the lane moves past it.
    template <class C>
    __device__ __forceinline__ void finish(const Lane& L, C& cnt, int) {
        cnt.add(C_WALKS);
        if (sink->walks_per_slice <= 0) return;
        const long long sl = (L.w - wc->walk_base) / sink->walks_per_slice;
        SliceTally* st = slice_tally();
        if (sl != st->slice) {
            flush_slice(*sink, st);
            st->slice = sl;
        }
        st->count++;
    }
    // After the lane's last walk.
    __device__ __forceinline__ void drain() {
        if (sink->walks_per_slice > 0) flush_slice(*sink, slice_tally());
    }
    __device__ __forceinline__ void alphas(int, double& a_ret, double& a_out) const {
        a_ret = wc->a_ret;
        a_out = wc->a_out;
    }
    // Not warp-collective; every lane calls it.
    template <class C>
    __device__ __forceinline__ bool refill(const GraphDev& g, Lane& L, bool have, C& cnt) {
        while (!have && next < wc->num_walks) {
            const long long row = next;
            next += stride;
            have = begin_walk(g, *wc, -1, row, L);
            if (!have) finish(L, cnt, 0);
        }
        return have;
    }
};

// 16-byte loads through L2 only: queue entries and request descriptors of a
// served queue are rewritten by the host while the kernel runs, so no copy of
// them may come from an SM's L1.
__device__ __forceinline__ WalkConst load_walkconst(const WalkConst* p) {
    WalkConst w;
    const int4* src = reinterpret_cast<const int4*>(p);
    int4* dst = reinterpret_cast<int4*>(&w);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(WalkConst) / 16); ++i) dst[i] = __ldcg(src + i);
    return w;
}

// Iterations a warp with live walks lets pass before polling an empty served
// queue again (about 10-20 us: far below the latency a request sees anyway).
constexpr int kIdlePollSkip = 8;

// Batched and served: a warp takes queue entries (one request's walk range) and
// deals their walks to its lanes as lanes free up.  Served queues are ticket
// queues (see take_chunk), so the queue can keep growing while the kernel runs
// and no warp ever retries a contended compare-and-swap.
struct QueueFeed {
    const WalkConst* reqs;       // request table (device)
    const Chunk* chunks;         // queue entries (device ring of `ring` entries)
    unsigned long long* ctl;     // ctl[0] = next ticket (head), ctl[1] = entries published
                                 // (tail), ctl[2] = the host's heartbeat (served)
    unsigned long long ring;     // ring capacity (entries)
    long long idle_spins;        // served: polls of an empty queue before giving up; 0 batched
    int* exit_flag;              // served: set when the kernel should stop
    unsigned long long* done;    // served: per request, finished walks and transitions taken
                                 // (done[2 r], done[2 r + 1]); batched: nullptr
    unsigned* done_flags;        // served: per-request host-mapped completion flags
    int* status;                 // the graph's device status word
    // warp-uniform state
    long long cur_lo;
    int cur_left;
    int cur_req;
    int idle_polls;              // served: iterations to skip before polling an empty queue
                                 // again; < 0 once the queue is drained for good

    // Per-request constants differ between lanes: held in the lane.
    __device__ __forceinline__ unsigned long long seed(const Lane&) const { return wrec()->seed; }
    __device__ __forceinline__ uint4 trial(const Lane& L, unsigned k) const {
        return trial_block(wrec()->seed, L.w, L.s, k);
    }
    __device__ __forceinline__ int len(const Lane&) const { return wrec()->len; }
    __device__ __forceinline__ unsigned tm1_ret(const Lane&) const { return wrec()->tm1_ret; }
    __device__ __forceinline__ unsigned tm1_in(const Lane&) const { return wrec()->tm1_in; }
    __device__ __forceinline__ unsigned tm1_out(const Lane&) const { return wrec()->tm1_out; }
    __device__ __forceinline__ int* row(const Lane&) const { return wrec()->row; }
    __device__ __forceinline__ int suss_k(const Lane&) const { return 0; }   // exact walks

    __device__ __forceinline__ void drain() {}
    // steps: transitions the finished walk took.
    template <class C>
    __device__ __forceinline__ void finish(const Lane& L, C& cnt, int steps) {
        cnt.add(C_WALKS);
        if (done == nullptr) return;                 // batched: nothing to publish
        const int req = L.req;
        if (steps > 0) atomicAdd(done + 2 * req + 1, (unsigned long long)steps);
        // Each walk's count is a release: its rows are visible before it counts.
        // The walk that completes the request adds an acquire fence, so it has
        // seen every other walk's rows before it raises the host-visible flag.
        const long long nw = __ldcg(&reqs[req].num_walks);
        cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> c(done[2 * req]);
        const unsigned long long prev = c.fetch_add(1ull, cuda::memory_order_release);
        if (prev + 1 == (unsigned long long)nw) {
            cuda::atomic_thread_fence(cuda::memory_order_acquire, cuda::thread_scope_device);
            __threadfence_system();
            *(volatile unsigned*)(done_flags + req) = 1u;
        }
    }
    __device__ __forceinline__ void alphas(int req, double& a_ret, double& a_out) const {
        a_ret = __ldcg(&reqs[req].a_ret);
        a_out = __ldcg(&reqs[req].a_out);
    }

    // Take one queue entry for the warp (lane 0 decides, then broadcast).
    // Returns 1 with an entry; 0 when a served queue has nothing for this warp
    // right now (only when `wait` is false); -1 when the queue is drained
    // (batched), the server is shutting down, or a waiting warp's bounded wait
    // ran out.  Only a warp that holds no walk at all waits: a warp with walks
    // in flight looks once and carries on, so an empty queue never stalls live
    // walks.
    //
    // Served queues are ticket queues.  A warp draws a ticket h with one atomic
    // increment of the head and owns entry h once the published tail passes h.
    // The head runs ahead of the tail by at most one ticket per warp (a warp
    // keeps its ticket, in shared memory, until the ticket is served); the
    // server resets the head to the tail before each launch, when every
    // published entry has been taken.  A warp with live walks draws a ticket
    // only when the queue looks non-empty, so new work goes to waiting warps
    // first.  The waiting warp's wait is bounded: about idle_spins microseconds
    // of sleep without a new host heartbeat (ctl[2]), after which it raises
    // status bit 2 and leaves.
    __device__ __forceinline__ int take_chunk(int lane, bool wait) {
        long long lo = 0;
        int cnt = 0, rq = -1;
        int ok = -1;
        if (lane == 0) {
            unsigned long long h = 0;
            bool got = false;
            if (idle_spins <= 0) {
                // Batched: the tail is fixed for the launch (the head is reset
                // before each launch).
                h = atomicAdd(ctl, 1ull);
                got = h < ctl[1];
            } else {
                unsigned long long* const slot = warp_ticket();
                unsigned long long tk = *slot;
                long long slept = 0;
                unsigned long long beat = 0;
                unsigned nap = 1024u;                        // ns
                while (true) {
                    if (wait && *(volatile int*)exit_flag) break;     // shutdown
                    if (tk == kNoTicket) {
                        unsigned long long h0, t0;               // head and tail in one load
                        asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];"
                                     : "=l"(h0), "=l"(t0) : "l"(ctl));
                        if (!wait && h0 >= t0) {                 // nothing for a busy warp
                            ok = 0;
                            break;
                        }
                        tk = atomicAdd(ctl, 1ull);
                    }
                    if (tk < *(volatile unsigned long long*)(ctl + 1)) {
                        h = tk;
                        tk = kNoTicket;
                        got = true;
                        break;
                    }
                    if (!wait) {                                 // keep the ticket
                        ok = 0;
                        break;
                    }
                    // Back off (1 us doubling to 32 us), so thousands of waiting
                    // warps do not hammer the queue words while others work.
                    const unsigned long long b = *(volatile unsigned long long*)(ctl + 2);
                    if (b != beat) {
                        beat = b;
                        slept = 0;
                    }
                    slept += nap >> 10;
                    if (slept > idle_spins) {
                        atomicOr(status, 2);
                        break;
                    }
                    __nanosleep(nap);
                    nap = nap < 32768u ? 2u * nap : nap;
                }
                *slot = tk;
            }
            if (got) {
                __threadfence();     // the entry is read after the tail that covers it
                const int4 c = __ldcg(reinterpret_cast<const int4*>(chunks + (h % ring)));
                lo = (long long)(((unsigned long long)(unsigned)c.y << 32) | (unsigned)c.x);
                cnt = c.z;
                rq = c.w;
                ok = 1;
            }
        }
        ok = __shfl_sync(FULL, ok, 0);
        if (ok <= 0) return ok;
        cur_lo = __shfl_sync(FULL, lo, 0);
        cur_left = __shfl_sync(FULL, cnt, 0);
        cur_req = __shfl_sync(FULL, rq, 0);
        return 1;
    }

    // Warp-collective: every lane of the warp calls it.
    template <class C>
    __device__ __forceinline__ bool refill(const GraphDev& g, Lane& L, bool have, C& cnt) {
        const int lane = threadIdx.x & 31;
        while (true) {
            const unsigned need = __ballot_sync(FULL, !have);
            if (need == 0 || idle_polls < 0) break;
            if (cur_left == 0) {
                // A warp with live walks that found the served queue empty polls
                // again only after kIdlePollSkip iterations: each poll is a
                // dependent L2 round trip that would otherwise slow every
                // iteration of the warp while the queue stays empty.
                if (idle_polls > 0 && need != FULL) {
                    --idle_polls;
                    break;
                }
                const int got = take_chunk(lane, need == FULL);
                if (got == 0) {               // nothing queued yet: live walks go on
                    idle_polls = kIdlePollSkip;
                    break;
                }
                if (got < 0) {
                    idle_polls = -1;
                    break;
                }
                idle_polls = 0;
            }
            const int rank = __popc(need & ((1u << lane) - 1u));
            const int n_need = __popc(need);
            const int give = n_need < cur_left ? n_need : cur_left;
            if (!have && rank < give) {
                const WalkConst wc = load_walkconst(reqs + cur_req);
                have = begin_walk(g, wc, cur_req, cur_lo + rank, L);
                if (have) set_wrec(wc, cur_lo + rank);
                else finish(L, cnt, 0);
            }
            cur_lo += give;
            cur_left -= give;
        }
        return have;
    }
};

// ---------------------------------------------------------------------------
// The engine
// ---------------------------------------------------------------------------
// A proposal's entry and decision.
struct Prop {
    int x, deg;
    long long off;
    bool acc_a, acc_b;    // accept if x in N(t) / if not (equal when the class is known)
};

// HUB: the instantiation that carries the optional search schedules for long
// lists (sector pivots, warp-cooperative narrowing); without it they are
// compiled out and those tuning knobs have no effect.
template <bool WEIGHTED, bool HAS_P, bool HAS_Q, bool COUNT, class Feed, bool HUB = false>
struct Engine {
    const GraphDev& g;
    Feed& feed;
    unsigned trial_cap;
    int shorter_min;             // undirected: search the shorter of N(t), N(x) when
                                 // deg_t exceeds this
    bool interp;                 // place probes by interpolation between the value bounds
    int warp_min;                // new searches over lists longer than this are first narrowed
                                 // by the whole warp (INT_MAX: never)
    bool edge_hash;              // membership tests read the edge hash first (when the graph has one)
    int pivot_min;               // lists of at least this many entries are searched over their
                                 // sector pivots first (INT_MAX: never)
    Counts<COUNT>& cnt;
    int4& ld;                    // the gather in flight: a proposal entry or a probe
    int4& ld2;                   // sector, first and second 16 bytes

    // Emit x and move to it.  rt, wr: position of v in N(x) and the weight there;
    // jv, wj: position of x in N(v) and the weight there.  Returns true while the
    // walk continues.
    __device__ __forceinline__ bool advance(Lane& L, int x, long long off, int deg, float wmax,
                                            int rt, float wr, int jv, float wj) {
        const int len = feed.len(L);
        int* const row = feed.row(L);
        put(L, row, L.s, x, len);
        cnt.add(C_STEPS);
        TRec* tr = trec();
        tr->off_t = L.off_v;
        tr->deg_t = L.deg_v;
        tr->wmax_t = L.wmax_v;
        tr->jv = jv;
        tr->wj = wj;
        L.t = L.v;
        L.v = x;
        L.off_v = off;
        L.deg_v = deg;
        L.wmax_v = wmax;
        L.rt = rt;
        L.wr = wr;
        L.s++;
        L.k = 0;
        if (L.s >= len) {
            feed.finish(L, cnt, L.s - 1);
            return false;
        }
        if (deg == 0) {
            fill_dead(L, row, L.s, len);
            feed.finish(L, cnt, L.s - 1);
            return false;
        }
        return true;
    }

    // Move along the proposal whose entry is (a, b), at position idx of N(v).
    // Unweighted: the filter of N(v) becomes that of N(t), and the entry's
    // filter (of N(x)) that of N(v).
    __device__ __forceinline__ bool advance_entry(Lane& L, int4 a, int4 b, int idx) {
        if (!WEIGHTED) shift_filters((unsigned)b.x, (unsigned)b.y, (unsigned)b.w);
        else if (g.pair_filters) frec()->fv[0] = (unsigned)b.w;
        const long long off = (long long)(((unsigned long long)(unsigned)a.w << 32) | (unsigned)a.z);
        // the weight of (x -> v): the last word, or w_vx itself where that word
        // holds the pair filter (undirected graphs: equal weights)
        const int wxv = (WEIGHTED && g.pair_filters) ? b.x : b.w;
        return advance(L, a.x, off, a.y, __int_as_float(b.y), b.z, __int_as_float(wxv), idx,
                       __int_as_float(b.x));
    }

    __device__ __forceinline__ void shift_filters(unsigned f0, unsigned f1, unsigned f2) {
        FRec* fr = frec();
        const unsigned v0 = fr->fv[0], v1 = fr->fv[1], v2 = fr->fv[2];
        fr->ft[0] = v0;
        fr->ft[1] = v1;
        fr->ft[2] = v2;
        fr->fv[0] = f0;
        fr->fv[1] = f1;
        fr->fv[2] = f2;
    }

    // Unweighted: do the filters prove that x is not in N(t)?
    // Row filters: the filter of N(t) tests x; on undirected graphs x in N(t)
    // <=> t in N(x), so the filter of N(x), which arrived in x's entry (ld2),
    // tests t as well.
    // Pair filters (undirected): t is a neighbour of v, so x in N(t) <=> x in
    // N(t) n N(v), whose filter came with the entry the walk arrived by (fv),
    // <=> t in N(v) n N(x), whose filter is in x's entry.
    __device__ __forceinline__ bool filters_exclude(const Lane& L, int x) {
        const FRec* fr = frec();
        if (WEIGHTED) {            // 32-bit pair filters
            if (!((fr->fv[0] >> filter_bit32(x)) & 1u)) return true;
            return !(((unsigned)ld2.w >> filter_bit32(L.t)) & 1u);
        }
        const unsigned* f = g.pair_filters ? fr->fv : fr->ft;
        if (!filter_has(f[0], f[1], f[2], filter_bit(x))) return true;
        return g.undirected &&
               !filter_has((unsigned)ld2.x, (unsigned)ld2.y, (unsigned)ld2.w, filter_bit(L.t));
    }

    // Steps drawn by the exact fallback while the trial cap is spent.  Returns have.
    __device__ __forceinline__ bool fallback_steps(Lane& L) {
        while (L.k >= trial_cap) {
            cnt.add(C_FALLBACKS);
            double a_ret, a_out;
            feed.alphas(L.req, a_ret, a_out);
            const int j = exact_fallback<WEIGHTED>(g, L, feed.seed(L), a_ret, a_out, trial_cap,
                                                   feed.suss_k(L));
            int4 a, b;
            ld_sector(g.fat + 2 * (L.off_v + j), a, b);
            if (!advance_entry(L, a, b, j)) return false;
        }
        return true;
    }

    // Decide a proposal from its entry and acceptance uniform.
    __device__ __forceinline__ Prop eval(const Lane& L, unsigned r2) {
        Prop p;
        p.x = ld.x;
        p.deg = ld.y;
        p.off = (long long)(((unsigned long long)(unsigned)ld.w << 32) | (unsigned)ld.z);
        const float w = WEIGHTED ? __int_as_float(ld2.x) : 1.0f;
        // thresholds of the two possible classes: (in, out), or one class twice
        const bool first = L.t < 0;
        const bool ret = (HAS_P || HAS_Q) && !first && p.x == L.t;
        unsigned ta, tb;
        if (first) {
            ta = tb = 0xffffffffu;
        } else if (ret) {
            ta = tb = feed.tm1_ret(L);
        } else {
            ta = feed.tm1_in(L);
            tb = HAS_Q ? feed.tm1_out(L) : ta;
        }
        if (WEIGHTED) {
            weighted_accept2(r2, L.wmax_v, ta, tb, w, p.acc_a, p.acc_b);
        } else {
            p.acc_a = r2 <= ta;
            p.acc_b = r2 <= tb;
        }
        return p;
    }

    // Start the membership search that decides proposal p: is x in N(t)?
    // x in N(t) <=> t in N(x) for symmetric graphs: search the shorter row.
    __device__ __forceinline__ void begin_search(Lane& L, const Prop& p) {
        cnt.add(C_SEARCHES);
        int4* pe = parked_entry();
        pe[0] = ld;
        pe[1] = ld2;
        L.x = p.x;
        L.flags = (L.flags & ~(F_ACC_IN | F_ACC_OUT | F_KEY_T | F_BISECT | F_PIV | F_WARPQ |
                               F_HASH)) |
                  (p.acc_a ? F_ACC_IN : 0u) | (p.acc_b ? F_ACC_OUT : 0u);
        if (g.eh != nullptr && edge_hash) {
            // the pair (t, x), smaller id first on undirected graphs: its bucket
            // (as a slot index) and its tag
            unsigned long long a = (unsigned)L.t, b = (unsigned)p.x;
            if (g.undirected && b < a) {
                const unsigned long long c = a;
                a = b;
                b = c;
            }
            const int K = 2 * g.eh_k;
            const unsigned long long h = edge_hash_mix((a << g.eh_k) | b, K);
            L.sb = (long long)(h >> (K - g.eh_b)) * 8;
            L.vlo = (int)(h & ((1ull << (K - g.eh_b)) - 1ull)) + 1;
            L.sn = 8;
            L.flags |= F_HASH;
            return;
        }
        begin_list_search(L, p.off, p.deg);
    }

    // The sorted-list search of the membership test: x in N(t), or (undirected
    // graphs) t in N(x) when that row is the shorter (off_x, deg_x: x's row).
    __device__ __forceinline__ void begin_list_search(Lane& L, long long off_x, int deg_x) {
        const TRec* tr = trec();
        const int deg_t = tr->deg_t;
        const bool use_x = g.undirected && deg_t > shorter_min && deg_x < deg_t;
        L.sb = use_x ? off_x : tr->off_t;
        L.sn = use_x ? deg_x : deg_t;
        L.flags = (L.flags & ~(F_KEY_T | F_BISECT | F_PIV | F_WARPQ | F_HASH)) |
                  (use_x ? F_KEY_T : 0u);
        L.vlo = -1;                      // node ids lie in [0, n)
        L.vhi = (int)g.n;
        // A long list is first searched over its sector pivots: piv[j] for the
        // aligned sectors j0 < j <= j1 that start inside the list.  They bracket
        // the one sector that can hold the key, which is then read.
        if (HUB && g.piv != nullptr && L.sn >= pivot_min) {
            const long long j0 = L.sb >> 3, j1 = (L.sb + L.sn - 1) >> 3;
            if (j1 > j0) {
                L.flags |= F_PIV;
                L.sb = j0 + 1;
                L.sn = (int)(j1 - j0);
            }
        }
    }

    // Bounds of the list under search (the row of x, parked, or of t).
    __device__ __forceinline__ void list_bounds(const Lane& L, long long& b, int& n) const {
        if (L.flags & F_KEY_T) {
            const int4 a = parked_entry()[0];
            b = (long long)(((unsigned long long)(unsigned)a.w << 32) | (unsigned)a.z);
            n = a.y;
        } else {
            const TRec* tr = trec();
            b = tr->off_t;
            n = tr->deg_t;
        }
    }

    // The next probe of L's search: the aligned 32-byte sector of the list (or
    // of its pivots) around the position interpolated between the value bounds
    // (ids in a row are near-uniform after relabelling), or the midpoint.
    __device__ __forceinline__ const int4* probe_addr(Lane& L) {
        L.phase = PH_SEARCH;
        cnt.add(C_PROBES);
        if (L.flags & F_HASH) {
            L.sd = 0;
            cnt.add(C_HASH_PROBES);
            return reinterpret_cast<const int4*>(g.eh + L.sb);
        }
        int pos = L.sn >> 1;
        if (interp && !(L.flags & F_BISECT)) {
            const int kk = (L.flags & F_KEY_T) ? L.t : L.x;
            const float f = __fdividef((float)(kk - L.vlo), (float)(L.vhi - L.vlo));
            pos = min(max((int)(f * (float)L.sn), 0), max(L.sn - 1, 0));
        }
        const long long bi = (L.sb + pos) & ~7LL;
        const bool piv = HUB && (L.flags & F_PIV) != 0;
        L.sd = (int)(bi - L.sb);
        if (piv) cnt.add(C_PIVOT_PROBES);
        return reinterpret_cast<const int4*>((piv ? g.piv : g.dsts) + bi);
    }

    // Warp-cooperative narrowing (warp-collective; every lane calls it).  Each
    // lane whose new search waits (F_WARPQ) is served in turn: the 32 lanes read
    // the list at 32 evenly spaced positions and a ballot of (value <= key)
    // leaves 1/33 of the range, until at most kWarpLeft entries remain or the
    // key is met; then the lane issues its own first probe on what is left.
    static constexpr int kWarpLeft = 256;
    __device__ __forceinline__ void warp_search(Lane& L, bool have) {
        unsigned q = __ballot_sync(FULL, have && (L.flags & F_WARPQ));
        const int lane = threadIdx.x & 31;
        while (q) {
            const int src = __ffs(q) - 1;
            q &= q - 1;
            long long sb = __shfl_sync(FULL, L.sb, src);
            int sn = __shfl_sync(FULL, L.sn, src);
            const int key = __shfl_sync(FULL, (L.flags & F_KEY_T) ? L.t : L.x, src);
            int vlo = __shfl_sync(FULL, L.vlo, src), vhi = __shfl_sync(FULL, L.vhi, src);
            unsigned reads = 0;
            while (sn > kWarpLeft) {
                const int pos = (int)(((long long)(lane + 1) * sn) / 33);
                const int v = __ldg(g.dsts + sb + pos);
                reads += 32;
                const unsigned eq = __ballot_sync(FULL, v == key);
                if (eq) {                            // met: leave just that entry
                    sb += __shfl_sync(FULL, pos, __ffs(eq) - 1);
                    sn = 1;
                    vlo = key - 1;
                    vhi = key + 1;
                    break;
                }
                const int c = __popc(__ballot_sync(FULL, v < key));   // lanes below the key
                const int plo = __shfl_sync(FULL, pos, c == 0 ? 0 : c - 1);
                const int vl = __shfl_sync(FULL, v, c == 0 ? 0 : c - 1);
                const int phi = __shfl_sync(FULL, pos, c == 32 ? 31 : c);
                const int vh = __shfl_sync(FULL, v, c == 32 ? 31 : c);
                const int lo = c == 0 ? 0 : plo + 1;
                const int hi = c == 32 ? sn : phi;
                if (c > 0) vlo = vl;
                if (c < 32) vhi = vh;
                sb += lo;
                sn = hi - lo;
            }
            if (lane == src) {
                L.sb = sb;
                L.sn = sn;
                L.vlo = vlo;
                L.vhi = vhi;
                L.flags &= ~F_WARPQ;
                cnt.add_n(C_PROBES, reads);
                ld_sector(probe_addr(L), ld, ld2);
            }
        }
    }

    // One iteration for a lane that holds a walk.  Returns have.
    //
    // The proposal decision and the probe update are evaluated with selects;
    // then a lane that is not probing draws proposals until one needs its entry
    // read, deciding returns and certain rejections on the way.  The next gather
    // is one 32-byte sector: the next proposal's entry or the next probe sector.
    __device__ __forceinline__ bool step(Lane& L) {
        const int phase = L.phase;
        const bool srch = HAS_Q && phase == PH_SEARCH;
        // ---- outcome ----
        bool take = false;           // the walk moves to A (or to the searched proposal)
        bool probe = false;
        bool fresh = false;          // a search began in this iteration
        if (phase == PH_CAND) {
            const Prop A = eval(L, L.r2);
            if (A.acc_a == A.acc_b || !HAS_Q) {
                if (A.acc_a) take = true;
                else L.k++;
            } else if ((!WEIGHTED || g.pair_filters) && filters_exclude(L, A.x)) {
                cnt.add(C_FILTERED);            // x is not in N(t): the out class decides
                if (A.acc_b) take = true;
                else L.k++;
            } else {
                begin_search(L, A);
                fresh = true;
                probe = true;
            }
        } else if (srch) {
            if (L.flags & F_HASH) {
                // the pair's bucket: its tag decides; an overflowed bucket
                // without it sends the test to the sorted rows
                const unsigned tag = (unsigned)L.vlo;
                const bool hit = (unsigned)ld.x == tag || (unsigned)ld.y == tag ||
                                 (unsigned)ld.z == tag || (unsigned)ld.w == tag ||
                                 (unsigned)ld2.x == tag || (unsigned)ld2.y == tag ||
                                 (unsigned)ld2.z == tag || (unsigned)ld2.w == tag;
                if (hit || (unsigned)ld2.w != kHashOverflow) {
                    if ((L.flags & (hit ? F_ACC_IN : F_ACC_OUT)) != 0) take = true;
                    else L.k++;
                } else {
                    const int4 a = parked_entry()[0];
                    begin_list_search(L, (long long)(((unsigned long long)(unsigned)a.w << 32) |
                                                     (unsigned)a.z), a.y);
                    probe = true;
                }
            } else {
                // ---- probe view of the arrived sector of a sorted list ----
                const int key = (L.flags & F_KEY_T) ? L.t : L.x;
                int lo = 0, hi = L.sn;
                int vlo = L.vlo, vhi = L.vhi;
                bool found = false;
                {
                    const int vals[8] = {ld.x, ld.y, ld.z, ld.w, ld2.x, ld2.y, ld2.z, ld2.w};
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int dj = L.sd + j;
                        const bool in = (unsigned)dj < (unsigned)L.sn;
                        found |= in && vals[j] == key;
                        if (in && vals[j] < key && dj + 1 > lo) {
                            lo = dj + 1;
                            vlo = vals[j];
                        }
                        if (in && vals[j] > key && dj < hi) {
                            hi = dj;
                            vhi = vals[j];
                        }
                    }
                }
                const bool s_done = found || hi <= lo;
                if (HUB && s_done && !found && (L.flags & F_PIV)) {
                    // The pivots place the key in one sector of the list: pivots
                    // before position lo (of the narrowed range) are below it.
                    const long long sector = L.sb - 1 + lo;
                    long long rb;
                    int rn;
                    list_bounds(L, rb, rn);
                    const long long a = rb > 8 * sector ? rb : 8 * sector;
                    const long long b = (rb + rn) < (8 * sector + 8) ? (rb + rn) : (8 * sector + 8);
                    L.flags &= ~(F_PIV | F_BISECT);
                    L.sb = a;
                    L.sn = (int)(b - a);
                    L.vlo = vlo;
                    L.vhi = vhi;
                    probe = true;
                } else if (s_done) {
                    if ((L.flags & (found ? F_ACC_IN : F_ACC_OUT)) != 0) take = true;
                    else L.k++;
                } else {
                    // an interpolated probe that did not halve the range is followed
                    // by a bisecting one, so a search takes O(log deg) probes at worst
                    const bool slow = 2 * (hi - lo) > L.sn;
                    L.flags = ((L.flags & F_BISECT) || !slow) ? (L.flags & ~F_BISECT)
                                                              : (L.flags | F_BISECT);
                    L.sb += lo;
                    L.sn = hi - lo;
                    L.vlo = vlo;
                    L.vhi = vhi;
                    probe = true;
                }
            }
        }
        take = take || phase == PH_RET;
        if (take) {
            // one advance per iteration: along the arrived entry, the parked one
            // (after a search), or back to t (an accepted return)
            int4 a = ld, b = ld2;
            int jv = L.pidx;
            if (phase == PH_SEARCH) {
                const int4* pe = parked_entry();
                a = pe[0];
                b = pe[1];
            } else if (phase == PH_RET) {
                const TRec tr = *trec();
                a = make_int4(L.t, tr.deg_t, (int)(unsigned)tr.off_t,
                              (int)(unsigned)((unsigned long long)tr.off_t >> 32));
                if (WEIGHTED) {
                    // the last word: t's weight towards v, or with pair filters
                    // the filter of N(v) n N(t), the one the walk arrived by
                    const int last = g.pair_filters ? (int)frec()->fv[0] : __float_as_int(tr.wj);
                    b = make_int4(__float_as_int(L.wr), __float_as_int(tr.wmax_t), tr.jv, last);
                } else {
                    // back to t: the filter of the entry (v -> t) is the row
                    // filter of N(t), held as the previous node's, or the pair
                    // filter of N(v) n N(t), the one the walk arrived by
                    const FRec* fr = frec();
                    const unsigned* f = g.pair_filters ? fr->fv : fr->ft;
                    b = make_int4((int)f[0], (int)f[1], tr.jv, (int)f[2]);
                }
                jv = L.rt;
            }
            if (!advance_entry(L, a, b, jv)) return false;
        }
        const int4* addr = nullptr;
        if (probe) {
            if (HUB && fresh && L.sn > warp_min && !(L.flags & (F_PIV | F_HASH))) {
                L.flags |= F_WARPQ;          // warp_search issues this lane's first probe
                L.phase = PH_SEARCH;
            } else {
                addr = probe_addr(L);
            }
        } else {
            // Draw proposals until one needs its entry read, at most
            // kDrawsPerIter of them.  Past the first step the lane knows where t
            // sits in N(v): that proposal is the return, decided with the weight
            // of the entry it arrived by.  Any other proposal is rejected without
            // a read when r2 fails the larger of the in and out thresholds
            // (w <= wmax_v).
            const unsigned tin = feed.tm1_in(L);
            const unsigned tout = HAS_Q ? feed.tm1_out(L) : tin;
            const unsigned tmax = tin > tout ? tin : tout;
            L.phase = PH_DRAW;
#pragma unroll 1
            for (int d = 0; d < kDrawsPerIter; ++d) {
                if (L.k >= trial_cap) {
                    if (!fallback_steps(L)) return false;
                }
                const uint4 r = feed.trial(L, L.k);
                const int sk = feed.suss_k(L);
                const int idx = (sk > 0 && L.deg_v > sk)
                                    ? suss_pos(feed.seed(L), L.w, L.s, scale_index(r.x, r.y, sk),
                                               L.deg_v, sk)
                                    : scale_index(r.x, r.y, L.deg_v);
                cnt.add(C_TRIALS);
                if (L.t >= 0) {
                    if (idx == L.rt) {
                        if (accept_test<WEIGHTED>(r.z, L.wmax_v, feed.tm1_ret(L), L.wr)) {
                            L.phase = PH_RET;       // taken at the next iteration
                            break;
                        }
                        L.k++;
                        continue;
                    }
                    if (r.z > tmax) {
                        L.k++;
                        continue;
                    }
                }
                L.r2 = r.z;
                L.pidx = idx;
                L.phase = PH_CAND;
                addr = g.fat + 2 * (L.off_v + idx);
                cnt.add(C_GATHERS);
                break;
            }
        }
        // every gather is one aligned 32-byte sector, read by one 256-bit load
        if (addr) ld_sector(addr, ld, ld2);
        return true;
    }
};

// Search and fallback policy of a launch (grape_tuning_t's fields).
struct Policy {
    unsigned trial_cap;
    int shorter_min;
    int interp_search;
    int pivot_min;
    int warp_search_min;
    int edge_hash;
};

template <bool WEIGHTED, bool HAS_P, bool HAS_Q, bool COUNT, bool HUB = false, class Feed>
__device__ __forceinline__ void walk_loop(const GraphDev& g, Feed& feed, const Policy& pol) {
    Lane L;
    L.t = -1;
    L.req = -1;
    L.phase = PH_START;
    L.flags = 0;
    L.x = 0;
    L.sb = 0;
    L.sn = 0;
    L.sd = 0;
    L.vlo = -1;
    L.vhi = 0;
    L.r2 = 0;
    Counts<COUNT> cnt;
    cnt.clear();
    int4 ld = make_int4(0, 0, 0, 0);
    int4 ld2 = make_int4(0, 0, 0, 0);
    Engine<WEIGHTED, HAS_P, HAS_Q, COUNT, Feed, HUB> eng{g, feed, pol.trial_cap, pol.shorter_min,
                                                    pol.interp_search != 0, pol.warp_search_min,
                                                    pol.edge_hash != 0, pol.pivot_min, cnt, ld,
                                                    ld2};
    bool have = false;
    while (true) {
        have = feed.refill(g, L, have, cnt);
        if (!__any_sync(FULL, have)) break;
        if (have) have = eng.step(L);
        if (HUB && pol.warp_search_min != 0x7fffffff) eng.warp_search(L, have);
    }
    feed.drain();
    flush_counts(g, cnt);
}

}  // namespace grape
