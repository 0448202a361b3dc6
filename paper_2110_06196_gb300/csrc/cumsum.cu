// cumsum.cu -- node2vec walks drawn by the paper's own on-the-fly sampler
// (GRAPE, Methods, "Efficient sampling for Node2Vec RWs").  At every step from
// v (previous node t):
//   1. the un-normalised transition probability pi_vx = alpha(t, x) * w_vx of
//      each neighbour x, alpha from the return and in-out biases (eqs. alpha,
//      beta; 1 on the first step);
//   2. their cumulative sum in row order;
//   3. a uniform value u = ((r1:r0) >> 11) * 2^-53 * total, from the Philox
//      block of trial index 0 of the step;
//   4. the first neighbour whose cumulative sum exceeds u.
// Products and sums are fp64, each rounded once, in row order: the arithmetic
// of the rejection path's exact fallback, so these rows are grape_walks' rows
// with trial_cap = 0.  The step costs O(deg(v)) reads and searches whatever the
// acceptance rate, which is what makes it the alternative to rejection for
// (p, q, weight) settings that reject most proposals.
//
// One warp owns one walk.  The lanes read 32 consecutive entries of N(v) at a
// time (coalesced) and each tests its own x in N(t) by binary search, so
// the in-out bias, which the paper names as the bottleneck, runs 32 wide; the
// second pass takes the products of the first 256 entries from shared memory
// and the membership of the first 1024 from per-lane bit masks.  Step 4
// compares 32 cumulative sums at once (the warp's form of the paper's linear
// scan).  The cumulative sums must round as the sequential sum does: when every
// product of the row is a multiple of 2^lo and the row's total stays below
// 2^(lo + 53), no partial sum rounds, every order of additions gives the same
// values, and the warp adds with a shuffle scan; otherwise the warp adds in row
// order, one product after another.
#include <algorithm>
#include <climits>

#include "internal.h"

using namespace grape;

namespace {

constexpr int kCsThreads = 256;
constexpr int kCsWarps = kCsThreads / 32;
constexpr int kCsCache = 256;   // products a warp keeps from the first pass for the second
constexpr int kCsMaskRows = 1024;   // entries whose membership bits a lane keeps (32 chunks)

// p > 0 finite: p = m 2^b with m a 53-bit integer; lo = exponent of p's lowest
// set bit, hi = floor(log2 p).
__device__ __forceinline__ void product_bits(double p, int& lo, int& hi) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(p);
    const int E = (int)((bits >> 52) & 0x7ff);
    unsigned long long m = bits & ((1ull << 52) - 1);
    if (E) m |= 1ull << 52;
    const int b = (E ? E : 1) - 1075;
    lo = b + __ffsll((long long)m) - 1;
    hi = b + 63 - __clzll((long long)m);
}

// Is key in the sorted list a[0, n)?  Binary search: the 32 lanes of a warp
// search the same N(t) for 32 increasing keys, so their first probes share
// sectors, which stay cached while hub rows are searched again and again (an
// interpolation search, which spreads the lanes' probes at once, measured 3.3x
// slower here).
__device__ __forceinline__ bool in_sorted(const int* __restrict__ a, long long n, int key) {
    long long lo = 0, hi = n;
    while (lo < hi) {
        const long long mid = lo + ((hi - lo) >> 1);
        if (__ldg(a + mid) < key) lo = mid + 1;
        else hi = mid;
    }
    return lo < n && __ldg(a + lo) == key;
}

// alpha(t, x) of entry j of row v: a_ret, 1 or a_out (1 on the first step).
__device__ __forceinline__ double alpha_of(const GraphDev& g, int x, int t, long long off_t,
                                           long long deg_t, double a_ret, double a_out) {
    if (t < 0) return 1.0;
    if (x == t) return a_ret;
    return in_sorted(g.dsts + off_t, deg_t, x) ? 1.0 : a_out;
}

template <bool WEIGHTED>
__device__ __forceinline__ double weight_of(const GraphDev& g, long long e) {
    return WEIGHTED ? (double)__int_as_float(__ldg(&g.fat[2 * e + 1].x)) : 1.0;
}

// pi of entry j of row v: alpha(t, x) * w, rounded once.
template <bool WEIGHTED>
__device__ __forceinline__ double product(const GraphDev& g, long long off_v, long long j, int t,
                                          long long off_t, long long deg_t, double a_ret,
                                          double a_out) {
    const long long e = off_v + j;
    const int x = __ldg(g.dsts + e);
    return __dmul_rn(alpha_of(g, x, t, off_t, deg_t, a_ret, a_out), weight_of<WEIGHTED>(g, e));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

template <bool WEIGHTED>
__global__ void __launch_bounds__(kCsThreads)
cumsum_walk_kernel(GraphDev g, WalkConst wc) {
    __shared__ double cache[kCsWarps][kCsCache];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    double* const pc = cache[wid];
    const long long warps = (long long)gridDim.x * kCsWarps;
    for (long long row = (long long)blockIdx.x * kCsWarps + wid; row < wc.num_walks;
         row += warps) {
        const long long w = wc.walk_base + row;
        int* const rowp = wc.out + row * (long long)wc.walk_len;
        const int len = wc.walk_len;
        const long long i = w % wc.num_starts;
        const long long v0 = wc.starts ? (long long)__ldg(wc.starts + i) : i;
        if (v0 < 0 || v0 >= g.n) {
            if (lane == 0) atomicOr(g.status, 1);
            for (int s = lane; s < len; s += 32) rowp[s] = -1;
            continue;
        }
        if (lane == 0) rowp[0] = (int)v0;
        int v = (int)v0, t = -1;
        NodeRec rv = load_rec(g, v);
        long long off_t = 0, deg_t = 0;
        int s = 1;
        for (; s < len && rv.deg > 0; ++s) {
            const long long d = rv.deg;
            // 1-2: the products, the grid they sit on, and the lanes' partial sums
            int lo_min = INT_MAX, hi_max = INT_MIN;
            double part = 0.0;
            unsigned inmask = 0;       // bit c / 32: this lane's entry of chunk c is in N(t)
            // the product of entry j (j = c + lane) again: from the cache, from
            // the membership bits, or computed afresh
            auto again = [&](long long j) -> double {
                if (j < kCsCache) return pc[j];
                if (j >= kCsMaskRows)
                    return product<WEIGHTED>(g, rv.off, j, t, off_t, deg_t, wc.a_ret, wc.a_out);
                const long long e = rv.off + j;
                const int x = __ldg(g.dsts + e);
                const double a = t < 0 ? 1.0
                                       : (x == t ? wc.a_ret
                                                 : (((inmask >> (j >> 5)) & 1u) ? 1.0 : wc.a_out));
                return __dmul_rn(a, weight_of<WEIGHTED>(g, e));
            };
            for (long long c = 0; c < d; c += 32) {
                const long long j = c + lane;
                if (j < d) {
                    const long long e = rv.off + j;
                    const int x = __ldg(g.dsts + e);
                    double a = 1.0;
                    if (t >= 0) {
                        if (x == t) {
                            a = wc.a_ret;
                        } else {
                            const bool in = in_sorted(g.dsts + off_t, deg_t, x);
                            if (in && j < kCsMaskRows) inmask |= 1u << (j >> 5);
                            a = in ? 1.0 : wc.a_out;
                        }
                    }
                    const double p = __dmul_rn(a, weight_of<WEIGHTED>(g, e));
                    int lo, hi;
                    product_bits(p, lo, hi);
                    lo_min = min(lo_min, lo);
                    hi_max = max(hi_max, hi);
                    if (j < kCsCache) pc[j] = p;
                    part = __dadd_rn(part, p);
                }
            }
            lo_min = __reduce_min_sync(FULL, lo_min);
            hi_max = __reduce_max_sync(FULL, hi_max);
            const int clog = d <= 1 ? 0 : 64 - __clzll((long long)(d - 1));   // ceil(log2 d)
            // total < d 2^(hi_max + 1) <= 2^(hi_max + 1 + clog)
            const bool exact = hi_max + 1 + clog <= lo_min + 53;
            double total;
            if (exact) {
                total = warp_sum(part);
            } else {
                total = 0.0;
                for (long long c = 0; c < d; c += 32) {
                    const long long j = c + lane;
                    const double p = j < d ? again(j) : 0.0;
                    const int n = (int)min(32LL, d - c);
                    for (int k = 0; k < n; ++k) total = __dadd_rn(total, __shfl_sync(FULL, p, k));
                }
            }
            // 3: the uniform value below the total
            const uint4 r = trial_block(wc.seed, w, s, 0u);
            const unsigned long long r64 = (unsigned long long)r.x | ((unsigned long long)r.y << 32);
            const double u = __dmul_rn(__dmul_rn((double)(r64 >> 11), 0x1p-53), total);
            // 4: the first entry whose cumulative sum exceeds u
            long long pick = d - 1;
            double carry = 0.0;
            for (long long c = 0; c < d; c += 32) {
                const long long j = c + lane;
                const double p = j < d ? again(j) : 0.0;
                double S;
                if (exact) {
                    S = p;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const double y = __shfl_up_sync(FULL, S, o);
                        if (lane >= o) S = __dadd_rn(S, y);
                    }
                    S = __dadd_rn(S, carry);
                    carry = __shfl_sync(FULL, S, 31);
                } else {
                    double run = carry;
                    S = 0.0;
                    const int n = (int)min(32LL, d - c);
                    for (int k = 0; k < n; ++k) {
                        run = __dadd_rn(run, __shfl_sync(FULL, p, k));
                        if (lane == k) S = run;
                    }
                    carry = run;
                }
                const unsigned hit = __ballot_sync(FULL, j < d && S > u);
                if (hit) {
                    pick = c + __ffs(hit) - 1;
                    break;
                }
            }
            const int x = __ldg(g.dsts + rv.off + pick);
            if (lane == 0) rowp[s] = x;
            off_t = rv.off;
            deg_t = rv.deg;
            t = v;
            v = x;
            rv = load_rec(g, v);
            __syncwarp();           // the next step's first pass rewrites the cache
        }
        for (int s2 = s + lane; s2 < len; s2 += 32) rowp[s2] = -1;
    }
}

template <bool W>
cudaError_t launch_cumsum(const grape_graph* g, const WalkConst& wc, cudaStream_t stream) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cumsum_walk_kernel<W>,
                                                                  kCsThreads, 0);
    if (e != cudaSuccess) return e;
    per_sm = std::max(per_sm, 1);
    const long long need = (wc.num_walks + kCsWarps - 1) / kCsWarps;
    const int blocks = (int)std::max(1LL, std::min(need, (long long)g->num_sms * per_sm));
    cumsum_walk_kernel<W><<<blocks, kCsThreads, 0, stream>>>(g->dev(), wc);
    return cudaGetLastError();
}

}  // namespace

extern "C" grape_status_t grape_walks_cumsum(const grape_graph_t* g, const int32_t* starts,
                                             int64_t num_starts, int32_t walk_len,
                                             int32_t walks_per_node, double p, double q,
                                             uint64_t seed, int32_t* out,
                                             grape_stream_t stream_) {
    WalkConst wc;
    grape_status_t st = make_walk_const(g, starts, num_starts, walk_len, walks_per_node, p, q,
                                        seed, out, &wc);
    if (st != GRAPE_OK) return st;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    const cudaError_t e = g->weighted ? launch_cumsum<true>(g, wc, stream)
                                      : launch_cumsum<false>(g, wc, stream);
    return cuda_status(e);
}
