// graph.cu -- graph residency and preparation: CSR checks, node records, status
// word, tuning and counters.
//
// The graph is stored as GRAPE stores it (Methods, "Graph data structures":
// CSR with each adjacency list sorted), re-laid out for the walk kernels:
//   rec[v]   16-byte record {row offset (int64), degree (int32), max row weight (fp32)}
//            so that one aligned 16-byte load gives everything a step needs about v;
//   dsts[e]  int32 sorted rows, read by the membership searches (padded by 8);
//   fat      one 32-byte proposal entry per CSR entry e (row v, target x):
//            {x, deg_x, off_x lo, off_x hi} {w_vx, wmax_x, rev, w_xv}, rev being
//            the position of v in N(x) (-1 when absent) and w_xv its weight;
//            unweighted graphs hold a 96-bit filter of N(x) in place of the
//            three weights.  A proposal reads its target,
//            the target's row, the weight and the target's row maximum from one
//            sector, so an accepted step needs no further gather (edge-inlined
//            records); rev tells the walk where its previous node sits in the
//            next row, so proposals of the return class need no gather at all.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "internal.h"

using grape::NodeRec;

namespace {

enum : int {
    BAD_OFFSETS = 1,
    BAD_IDS = 2,
    BAD_ORDER = 4,
    BAD_WEIGHTS = 8,
    BAD_SYMMETRY = 16,
};

__global__ void check_offsets_kernel(const int64_t* __restrict__ offsets, long long n,
                                     long long m, int* bad) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v <= n;
         v += (long long)gridDim.x * blockDim.x) {
        const long long a = offsets[v];
        bool ok = (a >= 0 && a <= m);
        if (v == 0) ok = ok && (a == 0);
        if (v == n) ok = ok && (a == m);
        if (v < n) {
            const long long b = offsets[v + 1];
            ok = ok && (b >= a) && (b <= m);
        }
        if (!ok) atomicOr(bad, BAD_OFFSETS);
    }
}

// One warp per row: ids in range (always, so no later kernel can read out of
// bounds), strict order and weights (when validating), the node record and
// the weighted pair array.
__global__ void build_rows_kernel(const int64_t* __restrict__ offsets,
                                  const int32_t* __restrict__ dsts,
                                  const float* __restrict__ weights, long long n, int validate,
                                  int4* __restrict__ rec, int* bad, int* max_deg) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x / 32);
    for (long long v = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32; v < n;
         v += warps) {
        const long long a = offsets[v], b = offsets[v + 1];
        float wmax = 0.0f;
        int flags = 0;
        for (long long e = a + lane; e < b; e += 32) {
            const int x = dsts[e];
            if (x < 0 || x >= n) flags |= BAD_IDS;
            if (validate && e > a && dsts[e - 1] >= x) flags |= BAD_ORDER;
            if (weights) {
                const float w = weights[e];
                if (validate && !(isfinite(w) && w > 0.0f)) flags |= BAD_WEIGHTS;
                wmax = fmaxf(wmax, w);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            wmax = fmaxf(wmax, __shfl_xor_sync(grape::FULL, wmax, o));
            flags |= __shfl_xor_sync(grape::FULL, flags, o);
        }
        if (lane == 0) {
            const unsigned long long off = (unsigned long long)a;
            const int deg = (int)(b - a);
            rec[v] = make_int4((int)(unsigned)off, (int)(unsigned)(off >> 32), deg,
                               __float_as_int(wmax));
            if (flags) atomicOr(bad, flags);
            atomicMax(max_deg, deg);
        }
    }
}

// Unweighted graphs: the 96-bit neighbour filter of every row (one warp per
// row), filt[v] = {bits 0-31, 32-63, 64-95, 0}.
__global__ void build_filters_kernel(const int32_t* __restrict__ dsts, const int4* __restrict__ rec,
                                     long long n, int4* __restrict__ filt) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x / 32);
    for (long long v = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32; v < n;
         v += warps) {
        const int4 rv = rec[v];
        const long long a = (long long)(((unsigned long long)(unsigned)rv.y << 32) | (unsigned)rv.x);
        unsigned f[3] = {0u, 0u, 0u};
        for (long long e = a + lane; e < a + rv.z; e += 32) {
            const int b = grape::filter_bit(dsts[e]);
            f[b >> 5] |= 1u << (b & 31);
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) f[j] = __reduce_or_sync(grape::FULL, f[j]);
        if (lane == 0) filt[v] = make_int4((int)f[0], (int)f[1], (int)f[2], 0);
    }
}

// Proposal entries: fat[2e] = {x, deg_x, off_x lo, off_x hi}, and
// fat[2e + 1] = {w_vx bits, wmax_x bits, rev, w_xv bits} (weighted) or
// {filter of N(x) words 0, 1, rev, word 2} (unweighted, filt given).  One warp
// per row v, so the row's own bounds are known; ids were checked by
// build_rows_kernel.  rev = position of v in N(x) (binary search), or -1, and
// then w_xv = 0.
__global__ void build_fat_kernel(const int32_t* __restrict__ dsts, const float* __restrict__ weights,
                                 const int4* __restrict__ rec, const int4* __restrict__ filt,
                                 long long n, int4* __restrict__ fat) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x / 32);
    for (long long v = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32; v < n;
         v += warps) {
        const int4 rv = rec[v];
        const long long a = (long long)(((unsigned long long)(unsigned)rv.y << 32) | (unsigned)rv.x);
        const long long b = a + rv.z;
        for (long long e = a + lane; e < b; e += 32) {
            const int x = dsts[e];
            const int4 r = rec[x];
            const long long xa = (long long)(((unsigned long long)(unsigned)r.y << 32) | (unsigned)r.x);
            long long lo = xa, hi = xa + r.z;
            while (lo < hi) {
                const long long mid = lo + (hi - lo) / 2;
                if (dsts[mid] < v) lo = mid + 1; else hi = mid;
            }
            const bool back = lo < xa + r.z && dsts[lo] == v;
            const int rev = back ? (int)(lo - xa) : -1;
            fat[2 * e] = make_int4(x, r.z, r.x, r.y);
            if (weights) {
                const int w = __float_as_int(weights[e]);
                const int wrev = back ? __float_as_int(weights[lo]) : 0;
                fat[2 * e + 1] = make_int4(w, r.w, rev, wrev);
            } else {
                const int4 f = filt[x];
                fat[2 * e + 1] = make_int4(f.x, f.y, rev, f.z);
            }
        }
    }
}

// Undirected graphs: every entry v -> x has a reverse entry x -> v with the same weight.
__global__ void check_symmetry_kernel(const int4* __restrict__ rec, const int32_t* __restrict__ dsts,
                                      const int4* __restrict__ fat, int weighted, long long n,
                                      int* bad) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x / 32);
    for (long long v = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32; v < n;
         v += warps) {
        const int4 rv = rec[v];
        const long long a = (long long)(((unsigned long long)(unsigned)rv.y << 32) | (unsigned)rv.x);
        const long long b = a + rv.z;
        int flags = 0;
        for (long long e = a + lane; e < b; e += 32) {
            const int x = dsts[e];
            const int4 rx = rec[x];
            const long long xa = (long long)(((unsigned long long)(unsigned)rx.y << 32) | (unsigned)rx.x);
            // lower bound of v in row x
            long long lo = xa, hi = xa + rx.z;
            while (lo < hi) {
                const long long mid = lo + (hi - lo) / 2;
                if (dsts[mid] < v) lo = mid + 1; else hi = mid;
            }
            if (lo >= xa + rx.z || dsts[lo] != v) {
                flags |= BAD_SYMMETRY;
            } else if (weighted && fat[2 * lo + 1].x != fat[2 * e + 1].x) {
                flags |= BAD_SYMMETRY;
            }
        }
        flags = __reduce_or_sync(grape::FULL, flags);
        if (lane == 0 && flags) atomicOr(bad, flags);
    }
}

// piv[j] = dsts[8 j] for every aligned 32-byte sector j of the rows; the 8
// entries of padding after the last hold INT_MAX.
__global__ void build_pivots_kernel(const int32_t* __restrict__ dsts, long long sectors,
                                    int32_t* __restrict__ piv) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < sectors + 8;
         j += (long long)gridDim.x * blockDim.x)
        piv[j] = j < sectors ? dsts[8 * j] : 0x7fffffff;
}

// Edge hash: one warp per row inserts the row's pairs (undirected graphs: the
// pairs with v <= x, each pair once).  A slot is claimed by counting the
// bucket's pairs; the ninth and later pairs of a bucket are not stored.
__global__ void build_edge_hash_kernel(const int4* __restrict__ rec,
                                       const int32_t* __restrict__ dsts, long long n, int k, int b,
                                       int undirected, unsigned* __restrict__ table,
                                       unsigned* __restrict__ count) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x / 32);
    const int K = 2 * k;
    const unsigned long long rmask = (K - b >= 64) ? ~0ull : ((1ull << (K - b)) - 1ull);
    for (long long v = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32; v < n; v += warps) {
        const int4 r = rec[v];
        const long long a = (long long)(((unsigned long long)(unsigned)r.y << 32) | (unsigned)r.x);
        for (long long e = a + lane; e < a + r.z; e += 32) {
            const long long x = dsts[e];
            if (undirected && x < v) continue;
            const unsigned long long key = ((unsigned long long)v << k) | (unsigned long long)x;
            const unsigned long long h = grape::edge_hash_mix(key, K);
            const unsigned long long bucket = h >> (K - b);
            const unsigned slot = atomicAdd(count + bucket, 1u);
            if (slot < 8) table[8 * bucket + slot] = (unsigned)(h & rmask) + 1u;
        }
    }
}

// Is the pair (a, b) in the edge hash?  1 yes, 0 no, -1 its bucket overflowed
// without holding it (unknown).
__device__ __forceinline__ int hash_has_pair(const unsigned* __restrict__ table, int k, int b,
                                             int undirected, long long a_, long long b_) {
    unsigned long long a = (unsigned long long)a_, c = (unsigned long long)b_;
    if (undirected && c < a) {
        const unsigned long long d = a;
        a = c;
        c = d;
    }
    const int K = 2 * k;
    const unsigned long long h = grape::edge_hash_mix((a << k) | c, K);
    const unsigned tag = (unsigned)(h & ((1ull << (K - b)) - 1ull)) + 1u;
    const uint4* bk = reinterpret_cast<const uint4*>(table + (h >> (K - b)) * 8);
    const uint4 s0 = __ldg(bk), s1 = __ldg(bk + 1);
    if (s0.x == tag || s0.y == tag || s0.z == tag || s0.w == tag || s1.x == tag || s1.y == tag ||
        s1.z == tag || s1.w == tag)
        return 1;
    return s1.w == grape::kHashOverflow ? -1 : 0;
}

// Undirected graphs: the neighbour filter of entry (v -> x) becomes that of
// C(v, x) = N(v) n N(x), the common neighbours of the edge's nodes (96 bits in
// an unweighted entry; 32 bits in the last word of a weighted one, in place of
// the reverse weight, which equals w_vx on an undirected graph).
// For a walk at v that came from t (a neighbour of v), x in N(t) holds exactly
// when x is in C(t, v) and when t is in C(v, x); these sets are much smaller
// than the rows, so their filters prove far more non-memberships.
//
// Work is cut into chunks of kPairChunk consecutive entries of the whole entry
// array, one warp per chunk (grid stride), so the rows of hubs spread over many
// warps.  The warp finds the row of the chunk's first entry by a 32-ary search
// of the row offsets, loads 32 targets and their records at a time, and takes
// the entries with x > v in turn: the lanes test the entries of the shorter row
// against the other node in the edge hash (an overflowed bucket counts as a
// member), OR their bits, and lane 0 writes the filter into (v -> x) and,
// through rev, into (x -> v).  Pairs whose shorter row exceeds `cap` entries
// get an all-ones filter; unweighted self-loops keep the row filter
// (C(v, v) = N(v)), weighted ones get all ones.
constexpr int kPairChunk = 512;

__device__ __forceinline__ long long rec_off(int4 r) {
    return (long long)(((unsigned long long)(unsigned)r.y << 32) | (unsigned)r.x);
}

// Warp-collective: the last row v with off_v <= e (the row holding entry e,
// for 0 <= e < m: that row is not empty), by a 32-ary search over the offsets.
__device__ long long row_of_entry(const int4* __restrict__ rec, long long n, long long e) {
    const int lane = threadIdx.x & 31;
    long long lo = 0, hi = n;                  // off_lo <= e; the row lies in [lo, hi)
    while (hi - lo > 32) {
        const long long step = (hi - lo + 31) / 32;
        const long long q = lo + lane * step;
        const bool ok = q < hi && rec_off(rec[q]) <= e;
        const int j = 31 - __clz((int)__ballot_sync(grape::FULL, ok));   // lane 0: q = lo
        const long long top = lo + (long long)(j + 1) * step;
        lo += (long long)j * step;
        if (top < hi) hi = top;
    }
    const long long q = lo + lane;
    const bool ok = q < hi && rec_off(rec[q]) <= e;
    return lo + (31 - __clz((int)__ballot_sync(grape::FULL, ok)));
}

__global__ void build_pair_filters_kernel(const int4* __restrict__ rec,
                                          const int32_t* __restrict__ dsts,
                                          const unsigned* __restrict__ table, int k, int b,
                                          long long n, long long m, int cap, int weighted,
                                          int4* __restrict__ fat) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x / 32);
    const long long chunks = (m + kPairChunk - 1) / kPairChunk;
    for (long long c = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32; c < chunks;
         c += warps) {
        const long long e0 = c * kPairChunk;
        const long long e1 = e0 + kPairChunk < m ? e0 + kPairChunk : m;
        long long v = row_of_entry(rec, n, e0);
        int4 rv = rec[v];
        long long off_v = rec_off(rv);
        long long end_v = off_v + rv.z;
        for (long long base = e0; base < e1; base += 32) {
            // 32 targets and their records at once
            const long long el = base + lane;
            int xl = -1;
            int4 rxl = make_int4(0, 0, 0, 0);
            if (el < e1) {
                xl = dsts[el];
                if ((unsigned long long)(long long)xl < (unsigned long long)n) rxl = rec[xl];
                else xl = -1;                 // out of range (unvalidated graph): no filter
            }
            const int cnt = (int)(e1 - base < 32 ? e1 - base : 32);
            for (int j = 0; j < cnt; ++j) {
                const long long e = base + j;
                while (e >= end_v && v + 1 < n) {     // the next non-empty row
                    ++v;
                    rv = rec[v];
                    off_v = rec_off(rv);
                    end_v = off_v + rv.z;
                }
                if (e < off_v || e >= end_v) continue;    // inconsistent offsets: no filter
                const int x = __shfl_sync(grape::FULL, xl, j);
                if (x == v && weighted && lane == 0) fat[2 * e + 1].w = -1;   // no filter: all ones
                if (x < 0 || x <= v) continue;
                int4 rx;
                rx.x = __shfl_sync(grape::FULL, rxl.x, j);
                rx.y = __shfl_sync(grape::FULL, rxl.y, j);
                rx.z = __shfl_sync(grape::FULL, rxl.z, j);
                const long long off_x = rec_off(rx);
                const bool v_short = rv.z <= rx.z;
                const long long so = v_short ? off_v : off_x;
                const int sn = v_short ? rv.z : rx.z;
                const long long other = v_short ? x : v;
                unsigned f[3] = {~0u, ~0u, ~0u};
                if (sn <= cap) {
                    f[0] = f[1] = f[2] = 0u;
                    // four entries per lane per round, so their row and hash
                    // reads are in flight together
                    for (int i0 = lane; i0 < sn; i0 += 128) {
                        int y[4];
                        bool in[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            in[u] = i0 + 32 * u < sn;
                            y[u] = in[u] ? dsts[so + i0 + 32 * u] : 0;
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            if (in[u] && hash_has_pair(table, k, b, 1, other, y[u]) != 0) {
                                const int bit = weighted ? grape::filter_bit32(y[u])
                                                         : grape::filter_bit(y[u]);
                                f[bit >> 5] |= 1u << (bit & 31);
                            }
                        }
                    }
                    f[0] = __reduce_or_sync(grape::FULL, f[0]);
                    f[1] = __reduce_or_sync(grape::FULL, f[1]);
                    f[2] = __reduce_or_sync(grape::FULL, f[2]);
                }
                if (lane == 0) {
                    // unweighted: the three filter words; weighted: the last word
                    // (the reverse weight, equal to w_vx on an undirected graph)
                    int4 w = fat[2 * e + 1];
                    const int rev = w.z;                       // v sits at rev in N(x)
                    if (weighted) {
                        w.w = (int)f[0];
                    } else {
                        w.x = (int)f[0];
                        w.y = (int)f[1];
                        w.w = (int)f[2];
                    }
                    fat[2 * e + 1] = w;
                    // (x -> v); an unvalidated graph declared undirected may lack it
                    if (rev >= 0 && rev < rx.z) {
                        const long long er = off_x + rev;
                        int4 wr = fat[2 * er + 1];
                        if (weighted) {
                            wr.w = (int)f[0];
                        } else {
                            wr.x = (int)f[0];
                            wr.y = (int)f[1];
                            wr.w = (int)f[2];
                        }
                        fat[2 * er + 1] = wr;
                    }
                }
            }
        }
    }
}

__global__ void mark_edge_hash_overflow_kernel(unsigned* __restrict__ table,
                                               const unsigned* __restrict__ count,
                                               long long buckets) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < buckets;
         i += (long long)gridDim.x * blockDim.x)
        if (count[i] > 8) table[8 * i + 7] = grape::kHashOverflow;
}

// Pairs whose shorter row is longer than this keep an all-ones pair filter:
// the work of building a filter is one edge-hash read per entry of the shorter
// row, and a filter of more than about 1,000 common neighbours is saturated.
constexpr int kPairFilterCap = 1024;

void free_graph(grape_graph* g) {
    if (!g) return;
    cudaFree(g->rec);
    cudaFree(g->dsts);
    cudaFree(g->piv);
    cudaFree(g->eh);
    cudaFree(g->fat);
    cudaFree(g->status);
    cudaFree(g->counters);
    delete g;
}

int grid_for(int num_sms, long long items, int per_block) {
    long long b = (items + per_block - 1) / per_block;
    long long cap = (long long)num_sms * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

extern "C" {

const char* grape_status_string(grape_status_t s) {
    switch (s) {
        case GRAPE_OK: return "ok";
        case GRAPE_ERR_INVALID_ARG: return "invalid argument";
        case GRAPE_ERR_INVALID_GRAPH: return "invalid graph";
        case GRAPE_ERR_NOMEM: return "out of memory";
        case GRAPE_ERR_CUDA: return "CUDA runtime error";
        case GRAPE_ERR_TIMEOUT: return "timed out";
        case GRAPE_ERR_BUSY: return "busy";
        case GRAPE_ERR_CANCELLED: return "cancelled";
        case GRAPE_ERR_DEVICE: return "device reported an error (start id out of range)";
        case GRAPE_ERR_NOT_FOUND: return "unknown ticket";
    }
    return "unknown status";
}

grape_status_t grape_graph_create(const int64_t* offsets, const int32_t* dsts,
                                  const float* weights, int64_t num_nodes,
                                  int64_t num_entries, uint32_t flags,
                                  grape_stream_t stream_, grape_graph_t** out) {
    if (!out) return GRAPE_ERR_INVALID_ARG;
    *out = nullptr;
    if (!offsets || num_nodes < 1 || num_nodes > 0x7fffffffLL || num_entries < 0 ||
        num_entries > (1LL << 62) || (num_entries > 0 && !dsts) ||
        (flags & ~(GRAPE_UNDIRECTED | GRAPE_VALIDATE)))
        return GRAPE_ERR_INVALID_ARG;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);

    grape_graph* g = new (std::nothrow) grape_graph();
    if (!g) return GRAPE_ERR_NOMEM;
    g->n = num_nodes;
    g->m = num_entries;
    g->weighted = (weights != nullptr);
    g->undirected = (flags & GRAPE_UNDIRECTED) != 0;
    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&g->max_window, cudaDevAttrMaxAccessPolicyWindowSize, g->device);
    // dsts is padded by four entries so that a search probe, which reads the
    // aligned 16-byte block around a list position, never leaves the allocation.
    const size_t m_alloc = (size_t)num_entries + 8;
    // proposal entries, padded to a whole sector: a proposal reads the aligned
    // 32-byte sector that holds its entry
    const size_t fat_words = (num_entries > 0 ? (size_t)num_entries : 1) * 2;
    if (e == cudaSuccess) e = cudaMalloc(&g->rec, sizeof(int4) * (size_t)num_nodes);
    if (e == cudaSuccess) e = cudaMalloc(&g->dsts, sizeof(int32_t) * m_alloc);
    if (e == cudaSuccess) e = cudaMalloc(&g->fat, sizeof(int4) * fat_words);
    const long long sectors = (num_entries + 7) / 8;
    if (e == cudaSuccess) e = cudaMalloc(&g->piv, sizeof(int32_t) * (size_t)(sectors + 8));
    if (e == cudaSuccess) e = cudaMalloc(&g->status, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&g->counters, sizeof(unsigned long long) * grape::C_COUNT);
    if (e != cudaSuccess) {
        free_graph(g);
        return grape::cuda_status(e);
    }
    g->device_bytes = (int64_t)(sizeof(int4) * num_nodes + sizeof(int32_t) * m_alloc +
                                sizeof(int4) * fat_words + sizeof(int32_t) * (sectors + 8));
    int* scratch = g->status;   // [0] status word, [1] bad flags, [2] max degree
    int host[4] = {0, 0, 0, 0};
    e = cudaMemsetAsync(g->status, 0, sizeof(int) * 4, stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(g->counters, 0, sizeof(unsigned long long) * grape::C_COUNT, stream);

    // 1. Offsets first: nothing reads a row before its bounds are known good.
    if (e == cudaSuccess) {
        check_offsets_kernel<<<grid_for(g->num_sms, num_nodes + 1, 256), 256, 0, stream>>>(
            offsets, num_nodes, num_entries, scratch + 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, scratch, sizeof(int) * 4, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess || host[1] != 0) {
        free_graph(g);
        return e != cudaSuccess ? grape::cuda_status(e) : GRAPE_ERR_INVALID_GRAPH;
    }
    // 2. Rows: copy, ids, order, weights, records.
    if (num_entries > 0)
        e = cudaMemcpyAsync(g->dsts, dsts, sizeof(int32_t) * (size_t)num_entries,
                            cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(g->dsts + num_entries, 0, sizeof(int32_t) * 8, stream);   // padding
    if (e == cudaSuccess) {
        build_pivots_kernel<<<grid_for(g->num_sms, sectors + 8, 256), 256, 0, stream>>>(
            g->dsts, sectors, g->piv);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        build_rows_kernel<<<grid_for(g->num_sms, num_nodes * 32, 256), 256, 0, stream>>>(
            offsets, dsts, weights, num_nodes, (flags & GRAPE_VALIDATE) ? 1 : 0, g->rec,
            scratch + 1, scratch + 2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, scratch, sizeof(int) * 4, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess || host[1] != 0) {
        free_graph(g);
        return e != cudaSuccess ? grape::cuda_status(e) : GRAPE_ERR_INVALID_GRAPH;
    }
    // 3. Proposal entries (ids are known in range now); unweighted graphs first
    //    build the neighbour filters, in scratch freed once the entries hold them.
    if (num_entries > 0) {
        int4* filt = nullptr;
        if (!weights) {
            e = cudaMallocAsync(&filt, sizeof(int4) * (size_t)num_nodes, stream);
            if (e == cudaSuccess) {
                build_filters_kernel<<<grid_for(g->num_sms, num_nodes * 32, 256), 256, 0, stream>>>(
                    g->dsts, g->rec, num_nodes, filt);
                e = cudaGetLastError();
            }
        }
        if (e == cudaSuccess) {
            build_fat_kernel<<<grid_for(g->num_sms, num_nodes * 32, 256), 256, 0, stream>>>(
                g->dsts, weights, g->rec, filt, num_nodes, g->fat);
            e = cudaGetLastError();
        }
        if (filt) {
            const cudaError_t ef = cudaFreeAsync(filt, stream);
            if (e == cudaSuccess) e = ef;
        }
        if (e != cudaSuccess) {
            free_graph(g);
            return grape::cuda_status(e);
        }
    }
    // 4. Edge hash (membership by one 32-byte read).  Sized for about 3.5
    //    pairs per 8-slot bucket; the remainder must fit 31 bits.  Left out when
    //    it would be larger than the sorted rows twice over.
    if (num_entries > 0 && e == cudaSuccess) {
        int k = 1;
        while (k < 31 && (1LL << k) < num_nodes) ++k;
        const int K = 2 * k;
        const double pairs = g->undirected ? 0.5 * (double)num_entries : (double)num_entries;
        int b = 0;
        while (b < K && (double)(1ULL << b) * 3.5 < pairs) ++b;
        if (K - b > 31) b = K - 31;
        const long long buckets = 1LL << b;
        const size_t bytes = sizeof(unsigned) * 8 * (size_t)buckets;
        if (bytes <= std::max<size_t>(2 * sizeof(int32_t) * m_alloc, (size_t)64 << 20)) {
            unsigned* count = nullptr;
            e = cudaMalloc(&g->eh, bytes);
            if (e == cudaSuccess) e = cudaMemsetAsync(g->eh, 0, bytes, stream);
            if (e == cudaSuccess) e = cudaMallocAsync(&count, sizeof(unsigned) * (size_t)buckets, stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(unsigned) * (size_t)buckets, stream);
            if (e == cudaSuccess) {
                build_edge_hash_kernel<<<grid_for(g->num_sms, num_nodes * 32, 256), 256, 0, stream>>>(
                    g->rec, g->dsts, num_nodes, k, b, g->undirected ? 1 : 0, g->eh, count);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) {
                mark_edge_hash_overflow_kernel<<<grid_for(g->num_sms, buckets, 256), 256, 0, stream>>>(
                    g->eh, count, buckets);
                e = cudaGetLastError();
            }
            if (count) {
                const cudaError_t ef = cudaFreeAsync(count, stream);
                if (e == cudaSuccess) e = ef;
            }
            if (e == cudaSuccess) {
                g->eh_k = k;
                g->eh_b = b;
                g->eh_bytes = (int64_t)bytes;
                g->device_bytes += (int64_t)bytes;
            }
            // undirected graphs: filters of common neighbours
            if (e == cudaSuccess && g->undirected) {
                const long long chunks = (num_entries + kPairChunk - 1) / kPairChunk;
                build_pair_filters_kernel<<<grid_for(g->num_sms, chunks * 32, 256), 256, 0,
                                            stream>>>(g->rec, g->dsts, g->eh, k, b, num_nodes,
                                                      num_entries, kPairFilterCap,
                                                      weights ? 1 : 0, g->fat);
                e = cudaGetLastError();
                if (e == cudaSuccess) g->pair_filters = true;
            }
        }
        if (e != cudaSuccess) {
            free_graph(g);
            return grape::cuda_status(e);
        }
    }
    // 5. Symmetry.
    if ((flags & GRAPE_VALIDATE) && g->undirected) {
        check_symmetry_kernel<<<grid_for(g->num_sms, num_nodes * 32, 256), 256, 0, stream>>>(
            g->rec, g->dsts, g->fat, g->weighted ? 1 : 0, num_nodes, scratch + 1);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(host, scratch, sizeof(int) * 4, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess || host[1] != 0) {
            free_graph(g);
            return e != cudaSuccess ? grape::cuda_status(e) : GRAPE_ERR_INVALID_GRAPH;
        }
    }
    g->max_degree = host[2];
    e = cudaMemsetAsync(g->status, 0, sizeof(int) * 4, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        free_graph(g);
        return grape::cuda_status(e);
    }

    g->tuning.trial_cap = 4096;
    g->tuning.shorter_min = 8;
    g->tuning.block_threads = 256;
    g->tuning.blocks_per_sm = 0;
    g->tuning.chunk_walks = 64;
    g->tuning.interp_search = 1;
    g->tuning.l2_fetch_bytes = 0;
    g->tuning.pivot_min = 0x7fffffff;
    g->tuning.warp_search_min = 0x7fffffff;
    g->tuning.l2_persist_mb = 0;
    g->tuning.edge_hash = 1;
    *out = g;
    return GRAPE_OK;
}

void grape_graph_destroy(grape_graph_t* g) {
    if (!g) return;
    cudaDeviceSynchronize();
    free_graph(g);
}

grape_status_t grape_graph_info(const grape_graph_t* g, grape_graph_info_t* info) {
    if (!g || !info) return GRAPE_ERR_INVALID_ARG;
    std::memset(info, 0, sizeof(*info));
    info->num_nodes = g->n;
    info->num_entries = g->m;
    info->max_degree = g->max_degree;
    info->weighted = g->weighted ? 1 : 0;
    info->undirected = g->undirected ? 1 : 0;
    info->device_bytes = g->device_bytes;
    info->edge_hash_bytes = g->eh_bytes;
    return GRAPE_OK;
}

grape_status_t grape_graph_get_tuning(const grape_graph_t* g, grape_tuning_t* t) {
    if (!g || !t) return GRAPE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(const_cast<grape_graph*>(g)->mu);
    *t = g->tuning;
    return GRAPE_OK;
}

grape_status_t grape_graph_set_tuning(grape_graph_t* g, const grape_tuning_t* t) {
    if (!g || !t) return GRAPE_ERR_INVALID_ARG;
    if (t->trial_cap < 0 || t->trial_cap > 0x7fffffffLL || t->shorter_min < 0 ||
        t->block_threads < 32 || t->block_threads > 256 || (t->block_threads % 32) ||
        t->blocks_per_sm < 0 || t->chunk_walks < 1 || (t->interp_search != 0 && t->interp_search != 1) ||
        (t->l2_fetch_bytes != 0 && t->l2_fetch_bytes != 32 && t->l2_fetch_bytes != 64 &&
         t->l2_fetch_bytes != 128) ||
        t->pivot_min < 1 || t->warp_search_min < 0 || t->l2_persist_mb < 0 ||
        (t->edge_hash != 0 && t->edge_hash != 1))
        return GRAPE_ERR_INVALID_ARG;
    if (t->l2_persist_mb > 0) {
        // A per-context limit (released with the context): the L2 set-aside
        // for persisting accesses, capped at what the device allows.
        int dev = 0, cap = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&cap, cudaDevAttrMaxPersistingL2CacheSize, dev) != cudaSuccess)
            return GRAPE_ERR_CUDA;
        const size_t want = std::min((size_t)t->l2_persist_mb << 20, (size_t)cap);
        if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) != cudaSuccess)
            return GRAPE_ERR_CUDA;
    }
    if (t->l2_fetch_bytes != 0) {
        // A per-context limit (released with the context): how far the L2
        // widens a miss when it fetches from DRAM.
        if (cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)t->l2_fetch_bytes) !=
            cudaSuccess)
            return GRAPE_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g->mu);
    g->tuning = *t;
    return GRAPE_OK;
}

grape_status_t grape_stream_status(const grape_graph_t* g, grape_stream_t stream_) {
    if (!g) return GRAPE_ERR_INVALID_ARG;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    int word = 0;
    GRAPE_CUDA_TRY(cudaStreamSynchronize(stream));
    GRAPE_CUDA_TRY(cudaMemcpyAsync(&word, g->status, sizeof(int), cudaMemcpyDeviceToHost, stream));
    GRAPE_CUDA_TRY(cudaMemsetAsync(g->status, 0, sizeof(int), stream));
    GRAPE_CUDA_TRY(cudaStreamSynchronize(stream));
    return word ? GRAPE_ERR_DEVICE : GRAPE_OK;
}

grape_status_t grape_counters_enable(grape_graph_t* g, int32_t enable) {
    if (!g) return GRAPE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g->mu);
    g->counting = enable != 0;
    return GRAPE_OK;
}

grape_status_t grape_counters_read(grape_graph_t* g, grape_walk_counters_t* out) {
    if (!g || !out) return GRAPE_ERR_INVALID_ARG;
    unsigned long long c[grape::C_COUNT];
    GRAPE_CUDA_TRY(cudaDeviceSynchronize());
    GRAPE_CUDA_TRY(cudaMemcpy(c, g->counters, sizeof(c), cudaMemcpyDeviceToHost));
    GRAPE_CUDA_TRY(cudaMemset(g->counters, 0, sizeof(c)));
    GRAPE_CUDA_TRY(cudaDeviceSynchronize());
    out->steps = (int64_t)c[grape::C_STEPS];
    out->trials = (int64_t)c[grape::C_TRIALS];
    out->gathers = (int64_t)c[grape::C_GATHERS];
    out->searches = (int64_t)c[grape::C_SEARCHES];
    out->probes = (int64_t)c[grape::C_PROBES];
    out->fallbacks = (int64_t)c[grape::C_FALLBACKS];
    out->walks = (int64_t)c[grape::C_WALKS];
    out->filtered = (int64_t)c[grape::C_FILTERED];
    out->pivot_probes = (int64_t)c[grape::C_PIVOT_PROBES];
    out->hash_probes = (int64_t)c[grape::C_HASH_PROBES];
    return GRAPE_OK;
}

}  // extern "C"
