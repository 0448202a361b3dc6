// walk_device.cuh -- device side of the node2vec walk engine (sm_103a).
//
// One lane owns one walk at a time.  All three launch shapes share the engine
// `walk_loop`: per call (grid-stride over walk ids), batched (a queue of
// (request, walk range) entries), and served (the same queue, fed while the
// kernel runs).  Each loop iteration makes ONE rejection trial for every lane
// that holds a walk, so lanes whose trial counts differ do not serialise the
// warp on nested loops.  A lane that finishes a walk takes the next one.
//
// Per trial (GRAPE, Methods, eq. alphaRW with the beta/gamma split of eqs. alpha, beta):
//   Philox4x32-10(key = seed, ctr = (w, s, k)) -> r0..r3
//   e = off_v + mulhi64(r1:r0, deg_v); x = dsts[e] (+ w_vx)
//   class: x == t -> return (1/p); x in N(t) -> in (1); else out (1/q)
//   accept iff r2 < T_class  (weighted: r2 * wmax_v < T_class * w_vx in fp64)
// The membership search runs only when the in and out thresholds give different
// answers for this r2.  The decision is the same function of (r2, class) as
// always, so the bytes written do not change.
#pragma once
#include <cstdint>
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

struct GraphDev {
    const int4* rec;            // [n] NodeRec viewed as int4
    const int* dsts;            // [m] sorted rows
    const int2* pairs;          // [m] (dst, weight bits) for weighted graphs, else nullptr
    long long n;
    int* status;                // device status word (1 = bad start id)
    unsigned long long* counters;  // [6] or nullptr
    int undirected;
};

// Per-request constants.  Thresholds are stored as T - 1 (T in [1, 2^32]):
// r2 < T  <=>  r2 <= T - 1.
struct WalkConst {
    const int* starts;          // nullptr: start i is node i
    int* out;                   // rows [num_walks][walk_len]
    long long num_starts;
    long long num_walks;        // rows of this launch
    long long walk_base;        // walk id of row 0 (a shard of a larger job), else 0
    unsigned long long seed;
    unsigned tm1_ret, tm1_in, tm1_out;
    int walk_len;
    double a_ret, a_out;        // 1/p and 1/q for the exact fallback
    int out_vec;                // 1 when out is 16-byte aligned
    int pad;
    unsigned long long* done;   // served requests: finished-walk counter, else nullptr
    unsigned* done_flag;        // served requests: host-mapped completion flag, else nullptr
};

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
        const unsigned hi0 = __umulhi(0xD2511F53u, c.x);
        const unsigned lo0 = 0xD2511F53u * c.x;
        const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z);
        const unsigned lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 trial_block(unsigned long long seed, long long w, int s,
                                             unsigned k) {
    const unsigned long long uw = (unsigned long long)w;
    return philox4x32_10(make_uint4((unsigned)uw, (unsigned)(uw >> 32), (unsigned)s, k),
                         make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
}

// ---------------------------------------------------------------------------
// Membership: is key in the sorted list a[0, n)?
// ---------------------------------------------------------------------------

// Lane-local branchless binary search: ceil(log2 n) + 1 dependent loads.
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

// Warp-cooperative 33-ary search for one query (all 32 lanes call it with the
// same a, n, key): each round every lane loads one pivot, a ballot locates the
// segment, and the range shrinks 33x; the last <= 32 entries are read as one
// coalesced segment.  ~log33(n) + 1 round trips instead of log2(n) + 1.
__device__ __forceinline__ bool warp_search(const int* __restrict__ a, long long n, int key,
                                            int lane) {
    long long lo = 0;
    while (n > 32) {
        const long long pj = lo + ((long long)(lane + 1) * n) / 33;
        const int val = __ldg(a + pj);
        const unsigned m = __ballot_sync(FULL, val <= key);
        const int c = __popc(m);
        const long long nlo = (c == 0) ? lo : lo + ((long long)c * n) / 33;
        const long long nhi = (c == 32) ? lo + n : lo + ((long long)(c + 1) * n) / 33;
        lo = nlo;
        n = nhi - nlo;
    }
    const bool hit = (lane < n) && (__ldg(a + lo + lane) == key);
    return __any_sync(FULL, hit);
}

// ---------------------------------------------------------------------------
// Lane state
// ---------------------------------------------------------------------------
struct Lane {
    long long w;          // walk id within its request
    long long e0;         // element index of the row start in `out`
    long long off_v, off_t;
    int* out;
    unsigned long long seed;
    unsigned tm1_ret, tm1_in, tm1_out;
    unsigned k;           // trial index within the step
    int s;                // index of the entry being produced (1 .. len-1)
    int len;
    int v, t;             // current and previous node (t < 0 on the first step)
    int deg_v, deg_t;
    float wmax_v;
    int req;              // request index (batched / served), -1 for per-call
    int out_vec;
    int b0, b1, b2, b3;   // last four entries written (16-byte store buffer)
};

struct LaneCounts {
    unsigned steps, trials, searches, warp_searches, fallbacks, walks;
};

// Row writer: entries that fill an aligned 16-byte group lying inside the row
// leave as one streaming 16-byte store when the group's last entry arrives;
// the (at most 3 + 3) entries at the ragged row ends are stored singly.
__device__ __forceinline__ void put(Lane& L, int s, int val) {
    L.b0 = L.b1; L.b1 = L.b2; L.b2 = L.b3; L.b3 = val;
    const long long e = L.e0 + s;
    const long long gs = e & ~3LL;
    const bool full = L.out_vec && (gs >= L.e0) && (gs + 3 < L.e0 + L.len);
    if (!full) {
        __stcs(L.out + e, val);
    } else if ((e & 3) == 3) {
        __stcs(reinterpret_cast<int4*>(L.out + gs), make_int4(L.b0, L.b1, L.b2, L.b3));
    }
}

__device__ __forceinline__ void fill_dead(Lane& L, int from) {
    for (int j = from; j < L.len; ++j) put(L, j, -1);
}

__device__ __forceinline__ NodeRec load_rec(const GraphDev& g, int x) {
    const int4 r = __ldg(g.rec + x);
    NodeRec n;
    n.off = (long long)(((unsigned long long)(unsigned)r.y << 32) | (unsigned)r.x);
    n.deg = r.z;
    n.wmax = __int_as_float(r.w);
    return n;
}

// fl(r2 * wmax) < fl(T * w) with both products rounded once (no FMA).
__device__ __forceinline__ bool weighted_accept(unsigned r2, float wmax, unsigned tm1, float w) {
    const double lhs = __dmul_rn((double)r2, (double)wmax);
    const double rhs = __dmul_rn((double)tm1 + 1.0, (double)w);
    return lhs < rhs;
}

template <bool WEIGHTED>
__device__ __forceinline__ bool accept_test(unsigned r2, float wmax, unsigned tm1, float w) {
    if (WEIGHTED) return weighted_accept(r2, wmax, tm1, w);
    return r2 <= tm1;
}

// Exact fallback after trial_cap rejections: inverse transform over the
// cumulative sum of pi in row order (GRAPE, "Efficient sampling for Node2Vec
// RWs"), in fp64 with every product and sum rounded separately.
template <bool WEIGHTED>
__device__ int exact_fallback(const GraphDev& g, const Lane& L, double a_ret, double a_out,
                              unsigned trial_cap) {
    const uint4 r = trial_block(L.seed, L.w, L.s, trial_cap);
    const bool first = (L.t < 0);
    double total = 0.0;
    for (int j = 0; j < L.deg_v; ++j) {
        const long long e = L.off_v + j;
        const int x = __ldg(g.dsts + e);
        double a = 1.0;
        if (!first) {
            if (x == L.t) a = a_ret;
            else if (!lane_search(g.dsts + L.off_t, L.deg_t, x)) a = a_out;
        }
        const double w = WEIGHTED ? (double)__int_as_float(__ldg(&g.pairs[e].y)) : 1.0;
        total = __dadd_rn(total, __dmul_rn(a, w));
    }
    const unsigned long long r64 = (unsigned long long)r.x | ((unsigned long long)r.y << 32);
    const double u = __dmul_rn(__dmul_rn((double)(r64 >> 11), 0x1p-53), total);
    double run = 0.0;
    for (int j = 0; j < L.deg_v; ++j) {
        const long long e = L.off_v + j;
        const int x = __ldg(g.dsts + e);
        double a = 1.0;
        if (!first) {
            if (x == L.t) a = a_ret;
            else if (!lane_search(g.dsts + L.off_t, L.deg_t, x)) a = a_out;
        }
        const double w = WEIGHTED ? (double)__int_as_float(__ldg(&g.pairs[e].y)) : 1.0;
        run = __dadd_rn(run, __dmul_rn(a, w));
        if (run > u) return x;
    }
    return __ldg(g.dsts + L.off_v + L.deg_v - 1);
}

// A finished walk: served requests count it and, on the last walk of the
// request, publish completion to the host.
__device__ __forceinline__ void finish_walk(const WalkConst& wc, LaneCounts& cnt) {
    cnt.walks++;
    if (wc.done != nullptr) {
        __threadfence();   // this walk's rows are visible before it is counted
        const unsigned long long prev = atomicAdd(wc.done, 1ull);
        if (prev + 1 == (unsigned long long)wc.num_walks) {
            __threadfence_system();
            *(volatile unsigned*)wc.done_flag = 1u;
        }
    }
}

// Start the walk of row `row` (walk id walk_base + row) of request wc on this lane.  Returns true when the walk needs
// transitions; false when it is already complete (length 1, dead start, or a
// start id out of range, whose row is all -1 and which sets the status word).
__device__ __forceinline__ bool begin_walk(const GraphDev& g, const WalkConst& wc, int req,
                                           long long row, Lane& L, LaneCounts& cnt) {
    const long long w = wc.walk_base + row;
    L.w = w;
    L.req = req;
    L.out = wc.out;
    L.len = wc.walk_len;
    L.e0 = row * (long long)wc.walk_len;
    L.seed = wc.seed;
    L.tm1_ret = wc.tm1_ret;
    L.tm1_in = wc.tm1_in;
    L.tm1_out = wc.tm1_out;
    L.out_vec = wc.out_vec;
    const long long i = w % wc.num_starts;
    const long long v0 = wc.starts ? (long long)__ldg(wc.starts + i) : i;
    if (v0 < 0 || v0 >= g.n) {
        atomicOr(g.status, 1);
        fill_dead(L, 0);
        finish_walk(wc, cnt);
        return false;
    }
    put(L, 0, (int)v0);
    const NodeRec r = load_rec(g, (int)v0);
    L.v = (int)v0;
    L.t = -1;
    L.off_v = r.off;
    L.deg_v = r.deg;
    L.wmax_v = r.wmax;
    L.s = 1;
    L.k = 0;
    if (L.len <= 1) {
        finish_walk(wc, cnt);
        return false;
    }
    if (r.deg == 0) {
        fill_dead(L, 1);
        finish_walk(wc, cnt);
        return false;
    }
    return true;
}

// Move to x.  Returns true while the walk continues.
__device__ __forceinline__ bool advance(const WalkConst& wc, Lane& L, int x, const NodeRec& rx,
                                        LaneCounts& cnt) {
    put(L, L.s, x);
    cnt.steps++;
    L.t = L.v;
    L.off_t = L.off_v;
    L.deg_t = L.deg_v;
    L.v = x;
    L.off_v = rx.off;
    L.deg_v = rx.deg;
    L.wmax_v = rx.wmax;
    L.s++;
    L.k = 0;
    if (L.s >= L.len) {
        finish_walk(wc, cnt);
        return false;
    }
    if (rx.deg == 0) {
        fill_dead(L, L.s);
        finish_walk(wc, cnt);
        return false;
    }
    return true;
}

__device__ __forceinline__ void flush_counts(const GraphDev& g, LaneCounts& c) {
    if (g.counters == nullptr) return;
    unsigned long long v[6] = {c.steps, c.trials, c.searches, c.warp_searches, c.fallbacks,
                               c.walks};
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        unsigned long long x = v[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd(g.counters + i, x);
    }
}

// ---------------------------------------------------------------------------
// Walk sources
// ---------------------------------------------------------------------------

// Per call: lane j of the grid takes walks j, j + stride, j + 2 * stride, ...
struct GridFeed {
    const WalkConst* wc;     // kernel-parameter copy
    long long next;
    long long stride;
    __device__ __forceinline__ const WalkConst& req(int) const { return *wc; }
    // Not warp-collective; every lane calls it.
    __device__ __forceinline__ bool refill(const GraphDev& g, Lane& L, bool have,
                                           LaneCounts& cnt) {
        while (!have && next < wc->num_walks) {
            const long long w = next;
            next += stride;
            have = begin_walk(g, *wc, -1, w, L, cnt);
        }
        return have;
    }
};

// Batched and served: a warp takes queue entries (one request's walk range) and
// deals their walks to its lanes as lanes free up.  The queue head is advanced
// with a bounded compare-and-swap loop that never passes the published tail,
// so a served queue can keep growing while the kernel runs.
struct QueueFeed {
    const WalkConst* reqs;       // request table (device)
    const Chunk* chunks;         // queue entries (device ring of `ring` entries)
    unsigned long long* head;    // next entry to take
    const volatile unsigned long long* tail;  // entries published so far
    unsigned long long ring;     // ring capacity (entries)
    long long idle_spins;        // served: polls of an empty queue before giving up
    int* exit_flag;              // served: set when the kernel should stop
    // warp-uniform state
    long long cur_lo;
    int cur_left;
    int cur_req;
    bool drained;

    __device__ __forceinline__ const WalkConst& req(int r) const { return reqs[r]; }

    // Take one queue entry for the warp (lane 0 decides, then broadcast).
    // Returns false when the queue is drained (batched) or idle too long (served).
    __device__ __forceinline__ bool take_chunk(int lane) {
        long long lo = 0;
        int cnt = 0, rq = -1;
        int ok = 0;
        if (lane == 0) {
            long long spins = 0;
            while (true) {
                if (exit_flag && *(volatile int*)exit_flag) break;   // served: shutdown
                const unsigned long long t = *tail;
                unsigned long long h;
                bool got = false;
                if (idle_spins <= 0) {
                    // Batched: the tail is fixed for the launch, so a plain
                    // increment suffices (the head is reset before each launch).
                    h = atomicAdd(head, 1ull);
                    got = h < t;
                } else {
                    // Served: never move the head past the published tail.  Every
                    // failed CAS means another warp took an entry, so the retries
                    // are bounded by the entries available.
                    h = *(volatile unsigned long long*)head;
                    while (h < t) {
                        const unsigned long long prev = atomicCAS(head, h, h + 1);
                        if (prev == h) { got = true; break; }
                        h = prev;
                    }
                }
                if (got) {
                    const Chunk c = chunks[h % ring];
                    lo = c.walk_lo;
                    cnt = c.count;
                    rq = c.req;
                    ok = 1;
                    break;
                }
                if (idle_spins <= 0) break;                  // batched: queue drained
                if (++spins > idle_spins) break;             // served: bounded idle wait
                __nanosleep(1000);
            }
        }
        ok = __shfl_sync(FULL, ok, 0);
        if (!ok) return false;
        cur_lo = __shfl_sync(FULL, lo, 0);
        cur_left = __shfl_sync(FULL, cnt, 0);
        cur_req = __shfl_sync(FULL, rq, 0);
        return true;
    }

    // Warp-collective: every lane of the warp calls it.
    __device__ __forceinline__ bool refill(const GraphDev& g, Lane& L, bool have,
                                           LaneCounts& cnt) {
        const int lane = threadIdx.x & 31;
        while (true) {
            const unsigned need = __ballot_sync(FULL, !have);
            if (need == 0 || drained) break;
            if (cur_left == 0) {
                if (!take_chunk(lane)) {
                    drained = true;
                    break;
                }
            }
            const int rank = __popc(need & ((1u << lane) - 1u));
            const int n_need = __popc(need);
            const int give = n_need < cur_left ? n_need : cur_left;
            if (!have && rank < give) {
                const WalkConst& wc = reqs[cur_req];
                have = begin_walk(g, wc, cur_req, cur_lo + rank, L, cnt);
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
template <bool WEIGHTED, bool HAS_P, bool HAS_Q, class Feed>
__device__ __forceinline__ void walk_loop(const GraphDev& g, Feed& feed, unsigned trial_cap,
                                          int warp_min, int shorter_list) {
    const int lane = threadIdx.x & 31;
    Lane L;
    L.t = -1;
    L.req = -1;
    LaneCounts cnt = {0, 0, 0, 0, 0, 0};
    bool have = false;

    while (true) {
        have = feed.refill(g, L, have, cnt);
        if (!__any_sync(FULL, have)) break;

        const WalkConst& wc = feed.req(L.req < 0 ? 0 : L.req);
        bool fallback = have && (L.k >= trial_cap);
        bool trial = have && !fallback;
        bool need = false, accept = false, acc_in = false, acc_out = false;
        int x = 0;
        float wx = 1.0f;
        NodeRec rx;
        rx.off = 0; rx.deg = 0; rx.wmax = 0.0f;
        bool have_rx = false;
        long long s_off = 0;
        int s_len = 0, s_key = 0;

        if (trial) {
            cnt.trials++;
            const uint4 r = trial_block(L.seed, L.w, L.s, L.k);
            const unsigned long long r64 = (unsigned long long)r.x | ((unsigned long long)r.y << 32);
            const long long e = L.off_v + (long long)__umul64hi(r64, (unsigned long long)L.deg_v);
            if (WEIGHTED) {
                const int2 pr = __ldg(g.pairs + e);
                x = pr.x;
                wx = __int_as_float(pr.y);
            } else {
                x = __ldg(g.dsts + e);
            }
            const unsigned r2 = r.z;
            if (L.t < 0) {
                accept = WEIGHTED ? weighted_accept(r2, L.wmax_v, 0xffffffffu, wx) : true;
            } else if ((HAS_P || HAS_Q) && x == L.t) {
                accept = accept_test<WEIGHTED>(r2, L.wmax_v, L.tm1_ret, wx);
            } else if (!HAS_Q) {
                accept = accept_test<WEIGHTED>(r2, L.wmax_v, L.tm1_in, wx);
            } else {
                acc_in = accept_test<WEIGHTED>(r2, L.wmax_v, L.tm1_in, wx);
                acc_out = accept_test<WEIGHTED>(r2, L.wmax_v, L.tm1_out, wx);
                if (acc_in == acc_out) accept = acc_in;
                else need = true;
            }
            if (accept || need) {
                rx = load_rec(g, x);
                have_rx = true;
            }
            if (need) {
                cnt.searches++;
                s_off = L.off_t;
                s_len = L.deg_t;
                s_key = x;
                if (shorter_list && g.undirected && rx.deg < L.deg_t) {
                    s_off = rx.off;
                    s_len = rx.deg;
                    s_key = L.t;
                }
            }
        }

        if (HAS_Q) {
            // Membership phase: short lists by the lane, long ones by the warp.
            bool found = false;
            if (need && s_len < warp_min) found = lane_search(g.dsts + s_off, s_len, s_key);
            unsigned wm = __ballot_sync(FULL, need && s_len >= warp_min);
            while (wm) {
                const int leader = __ffs(wm) - 1;
                wm &= wm - 1;
                const long long b = __shfl_sync(FULL, s_off, leader);
                const int n = __shfl_sync(FULL, s_len, leader);
                const int key = __shfl_sync(FULL, s_key, leader);
                const bool f = warp_search(g.dsts + b, n, key, lane);
                if (lane == leader) {
                    found = f;
                    cnt.warp_searches++;
                }
            }
            if (need) accept = found ? acc_in : acc_out;
        }

        if (trial) {
            if (accept) {
                have = advance(wc, L, x, rx, cnt);
            } else if (++L.k >= trial_cap) {
                fallback = true;
            }
        }
        if (fallback) {
            cnt.fallbacks++;
            const int xf = exact_fallback<WEIGHTED>(g, L, wc.a_ret, wc.a_out, trial_cap);
            const NodeRec rf = load_rec(g, xf);
            have = advance(wc, L, xf, rf, cnt);
        }
        (void)have_rx;
    }
    flush_counts(g, cnt);
}

}  // namespace grape
