// walks.cu -- per-call walks, batched walks (persistent queue kernel replayed
// from a CUDA graph), the batched-path autotuner, and diagnostics.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "internal.h"

using namespace grape;

namespace {

constexpr int kMaxThreads = 256;
// Resident blocks per SM the register allocation is held to: more warps keep
// more independent gathers in flight, which is what this latency-bound loop
// needs (4 x 256 threads -> at most 64 registers per thread).
constexpr int kMinBlocksWalk = 4;
constexpr int kMinBlocksQueue = 4;

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

// Per-call walk kernel: the eight specialisations of GRAPE ("Implementation of
// second-order RWs": p == 1, q == 1, weighted or not) as template arguments.
// COUNT: the instantiation that also keeps the work counters.
// SUSS: the approximated walks (GRAPE, Methods, "Approximated RWs"), only with
// the general p, q specialisation.
template <bool W, bool P, bool Q, bool COUNT, bool SUSS = false>
__global__ void __launch_bounds__(kMaxThreads, kMinBlocksWalk)
walk_kernel(GraphDev g, WalkConst wc, RoundKeys rk, unsigned trial_cap, int shorter_min,
            int interp_search) {
    GridFeed<SUSS> f;
    f.wc = &wc;
    f.rk = &rk;
    f.next = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    f.stride = (long long)gridDim.x * blockDim.x;
    walk_loop<W, P, Q, COUNT>(g, f, trial_cap, shorter_min, interp_search);
}

// Batched / served kernel: persistent grid draining a queue of walk ranges.
template <bool W, bool COUNT>
__global__ void __launch_bounds__(kMaxThreads, kMinBlocksQueue)
queue_kernel(GraphDev g, const WalkConst* reqs, const Chunk* chunks, unsigned long long* ctl,
             unsigned long long ring, long long idle_spins, int* exit_flag,
             unsigned long long* done, unsigned* done_flags, unsigned trial_cap, int shorter_min,
             int interp_search) {
    QueueFeed f;
    f.reqs = reqs;
    f.chunks = chunks;
    f.ctl = ctl;
    f.ring = ring;
    f.idle_spins = idle_spins;
    f.exit_flag = exit_flag;
    f.done = done;
    f.done_flags = done_flags;
    f.status = g.status;
    f.cur_lo = 0;
    f.cur_left = 0;
    f.cur_req = 0;
    f.idle_polls = 0;
    if ((threadIdx.x & 31) == 0) *warp_ticket() = kNoTicket;
    __syncwarp();
    walk_loop<W, true, true, COUNT>(g, f, trial_cap, shorter_min, interp_search);
}

__global__ void philox_kernel(const uint32_t* __restrict__ ck, long long n, uint32_t* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const uint32_t* p = ck + 6 * i;
        const uint4 r = philox4x32_10(make_uint4(p[0], p[1], p[2], p[3]), make_uint2(p[4], p[5]));
        out[4 * i + 0] = r.x;
        out[4 * i + 1] = r.y;
        out[4 * i + 2] = r.z;
        out[4 * i + 3] = r.w;
    }
}

// Random-sector gather probe: 8 independent sector reads in flight per thread.
// mode selects the load's cache path: 0 ld.global.nc (read-only path through
// L1), 1 ld.global.cg (L2 only), 2 ld.global.cs (streaming).
template <int MODE>
__global__ void __launch_bounds__(256)
sector_probe_kernel(const int4* __restrict__ buf, unsigned long long nsec, long long reads_per_thread,
                    unsigned long long seed, uint32_t* sink) {
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    unsigned acc = 0;
    for (long long j = 0; j < reads_per_thread; j += 8) {
        unsigned long long idx[8];
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
            const uint4 r = trial_block(seed, tid, (int)(j >> 3), (unsigned)u);
            const unsigned long long a = (unsigned long long)r.x | ((unsigned long long)r.y << 32);
            const unsigned long long b = (unsigned long long)r.z | ((unsigned long long)r.w << 32);
            idx[u] = __umul64hi(a, nsec);
            idx[u + 1] = __umul64hi(b, nsec);
        }
        int4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int4* p = buf + 2 * idx[u];
            v[u] = MODE == 0 ? __ldg(p) : (MODE == 1 ? __ldcg(p) : __ldcs(p));
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) acc ^= (unsigned)(v[u].x ^ v[u].w);
    }
    if (acc == 0x9e3779b9u) atomicXor(sink, acc);   // practically never; keeps the loads live
}

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------
// Dynamic shared memory of the walk kernels: one 32-byte output staging slot per thread.
inline size_t stage_bytes(int threads) { return (size_t)threads * kLaneSharedBytes; }

template <class K>
int occupancy_blocks(K kernel, int threads) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, stage_bytes(threads)) !=
            cudaSuccess ||
        nb < 1)
        nb = 1;
    return nb;
}

template <bool W, bool P, bool Q, bool C, bool S = false>
cudaError_t launch_walk_c(const grape_graph* g, const grape_tuning_t& t, const WalkConst& wc,
                          cudaStream_t stream) {
    const int threads = std::min(t.block_threads, kMaxThreads);
    int per_sm = t.blocks_per_sm;
    if (per_sm <= 0) per_sm = occupancy_blocks(walk_kernel<W, P, Q, C, S>, threads);
    long long blocks = (wc.num_walks + threads - 1) / threads;
    const long long cap = (long long)g->num_sms * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    walk_kernel<W, P, Q, C, S><<<(unsigned)blocks, threads, stage_bytes(threads), stream>>>(
        g->dev(), wc, round_keys(wc.seed), (unsigned)t.trial_cap, t.shorter_min,
        t.interp_search);
    return cudaGetLastError();
}

template <bool W, bool P, bool Q>
cudaError_t launch_walk(const grape_graph* g, const grape_tuning_t& t, const WalkConst& wc,
                        cudaStream_t stream) {
    return g->counting ? launch_walk_c<W, P, Q, true>(g, t, wc, stream)
                       : launch_walk_c<W, P, Q, false>(g, t, wc, stream);
}

cudaError_t dispatch_walk(const grape_graph* g, const grape_tuning_t& t, const WalkConst& wc,
                          bool has_p, bool has_q, cudaStream_t s) {
    if (wc.suss_k > 0) {
        if (g->weighted)
            return g->counting ? launch_walk_c<true, true, true, true, true>(g, t, wc, s)
                               : launch_walk_c<true, true, true, false, true>(g, t, wc, s);
        return g->counting ? launch_walk_c<false, true, true, true, true>(g, t, wc, s)
                           : launch_walk_c<false, true, true, false, true>(g, t, wc, s);
    }
    if (g->weighted) {
        if (has_p) return has_q ? launch_walk<true, true, true>(g, t, wc, s)
                                : launch_walk<true, true, false>(g, t, wc, s);
        return has_q ? launch_walk<true, false, true>(g, t, wc, s)
                     : launch_walk<true, false, false>(g, t, wc, s);
    }
    if (has_p) return has_q ? launch_walk<false, true, true>(g, t, wc, s)
                            : launch_walk<false, true, false>(g, t, wc, s);
    return has_q ? launch_walk<false, false, true>(g, t, wc, s)
                 : launch_walk<false, false, false>(g, t, wc, s);
}

bool valid_pq(double x) { return std::isfinite(x) && x > 0.0; }

// grape_walks_host: at most this many slices, of at least this many bytes.
constexpr size_t kHostSlices = 16;
constexpr size_t kHostSliceBytes = 64u << 20;

// One non-blocking stream per device for grape_walks_host's copies out.
cudaError_t host_copy_stream(cudaStream_t* out) {
    static std::mutex mu;
    static cudaStream_t streams[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!streams[dev]) {
        e = cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
    }
    *out = streams[dev];
    return cudaSuccess;
}

grape_tuning_t tuning_of(const grape_graph* g) {
    std::lock_guard<std::mutex> lk(const_cast<grape_graph*>(g)->mu);
    return g->tuning;
}

}  // namespace

namespace grape {

grape_status_t make_walk_const(const grape_graph* g, const int32_t* starts, int64_t num_starts,
                               int32_t walk_len, int32_t walks_per_node, double p, double q,
                               uint64_t seed, int32_t* out, WalkConst* wc) {
    if (!g) return GRAPE_ERR_INVALID_ARG;
    return make_walk_const_n(g->n, starts, num_starts, walk_len, walks_per_node, p, q, seed, out,
                             wc);
}

grape_status_t make_walk_const_n(int64_t num_nodes, const int32_t* starts, int64_t num_starts,
                                 int32_t walk_len, int32_t walks_per_node, double p, double q,
                                 uint64_t seed, int32_t* out, WalkConst* wc) {
    if (!out || !wc || num_starts < 1 || walk_len < 1 || walks_per_node < 1 ||
        !valid_pq(p) || !valid_pq(q))
        return GRAPE_ERR_INVALID_ARG;
    if (!starts && num_starts > num_nodes) return GRAPE_ERR_INVALID_ARG;
    if (num_starts > (INT64_MAX / walks_per_node) / walk_len) return GRAPE_ERR_INVALID_ARG;
    std::memset(wc, 0, sizeof(*wc));
    wc->starts = starts;
    wc->out = out;
    wc->num_starts = num_starts;
    wc->num_walks = num_starts * walks_per_node;
    wc->walk_base = 0;
    wc->seed = seed;
    wc->walk_len = walk_len;
    // Class thresholds: T_c = floor(alpha_c / amax * 2^32), alpha = (1/p, 1, 1/q).
    const double alpha[3] = {1.0 / p, 1.0, 1.0 / q};
    double amax = alpha[0];
    if (alpha[1] > amax) amax = alpha[1];
    if (alpha[2] > amax) amax = alpha[2];
    unsigned tm1[3];
    for (int c = 0; c < 3; ++c) {
        const double ratio = alpha[c] / amax;
        const unsigned long long T = (unsigned long long)std::floor(ratio * 4294967296.0);
        if (T < 1) return GRAPE_ERR_INVALID_ARG;   // p/q ratio beyond 2^32: unsupported
        tm1[c] = (unsigned)(T - 1);
    }
    wc->tm1_ret = tm1[0];
    wc->tm1_in = tm1[1];
    wc->tm1_out = tm1[2];
    wc->a_ret = alpha[0];
    wc->a_out = alpha[2];
    wc->out_vec = ((reinterpret_cast<uintptr_t>(out) & 31u) == 0) ? 1 : 0;
    return GRAPE_OK;
}

grape_status_t restrict_walks(WalkConst* wc, int64_t walk_begin, int64_t walk_count) {
    if (walk_begin < 0 || walk_count < 0 || walk_begin > wc->num_walks ||
        walk_count > wc->num_walks - walk_begin)
        return GRAPE_ERR_INVALID_ARG;
    wc->walk_base = walk_begin;
    wc->num_walks = walk_count;
    return GRAPE_OK;
}

LaunchShape queue_launch_shape(const grape_graph* g, const grape_tuning_t& t, int weighted) {
    LaunchShape s;
    s.threads = std::min(t.block_threads, kMaxThreads);
    int per_sm = t.blocks_per_sm;
    if (per_sm <= 0)
        per_sm = weighted ? occupancy_blocks(queue_kernel<true, false>, s.threads)
                          : occupancy_blocks(queue_kernel<false, false>, s.threads);
    s.blocks = g->num_sms * per_sm;
    return s;
}

cudaError_t launch_queue_kernel(const grape_graph* g, const grape_tuning_t& t,
                                const WalkConst* reqs, const Chunk* chunks,
                                unsigned long long* ctl, unsigned long long ring,
                                long long idle_spins, int* exit_flag, unsigned long long* done,
                                unsigned* done_flags, int blocks, cudaStream_t stream) {
    const LaunchShape s = queue_launch_shape(g, t, g->weighted);
    const int nb = blocks > 0 ? blocks : s.blocks;
    const size_t sh = stage_bytes(s.threads);
    const unsigned cap = (unsigned)t.trial_cap;
#define GRAPE_QUEUE_LAUNCH(W, C)                                                                 \
    queue_kernel<W, C><<<nb, s.threads, sh, stream>>>(g->dev(), reqs, chunks, ctl, ring,     \
                                                      idle_spins, exit_flag, done, done_flags, \
                                                      cap, t.shorter_min, t.interp_search)
    if (g->weighted) {
        if (g->counting) GRAPE_QUEUE_LAUNCH(true, true);
        else GRAPE_QUEUE_LAUNCH(true, false);
    } else {
        if (g->counting) GRAPE_QUEUE_LAUNCH(false, true);
        else GRAPE_QUEUE_LAUNCH(false, false);
    }
#undef GRAPE_QUEUE_LAUNCH
    return cudaGetLastError();
}

}  // namespace grape

// ---------------------------------------------------------------------------
// Batch plans
// ---------------------------------------------------------------------------
struct grape_batch_plan {
    const grape_graph* g = nullptr;
    WalkConst* d_reqs = nullptr;
    Chunk* d_chunks = nullptr;
    unsigned long long* d_ctl = nullptr;   // [0] head, [1] tail
    long long num_chunks = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static void free_plan(grape_batch_plan* p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    cudaFree(p->d_reqs);
    cudaFree(p->d_chunks);
    cudaFree(p->d_ctl);
    delete p;
}

static grape_status_t build_plan(const grape_graph* g, const grape_walk_request_t* reqs, int32_t n,
                                 const grape_tuning_t& t, grape_batch_plan** out) {
    *out = nullptr;
    if (!g || !reqs || n < 1) return GRAPE_ERR_INVALID_ARG;
    std::vector<WalkConst> wcs((size_t)n);
    for (int i = 0; i < n; ++i) {
        const grape_walk_request_t& r = reqs[i];
        grape_status_t st = make_walk_const(g, r.starts, r.num_starts, r.walk_len,
                                            r.walks_per_node, r.p, r.q, r.seed, r.out, &wcs[i]);
        if (st != GRAPE_OK) return st;
    }
    // Queue entries, longest walks first, so the slowest work starts early and
    // the short tail fills in behind it.
    std::vector<int> order((size_t)n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return wcs[a].walk_len > wcs[b].walk_len; });
    std::vector<Chunk> chunks;
    const long long cw = t.chunk_walks;
    for (int i : order) {
        for (long long lo = 0; lo < wcs[i].num_walks; lo += cw) {
            Chunk c;
            c.walk_lo = lo;
            c.count = (int)std::min(cw, wcs[i].num_walks - lo);
            c.req = i;
            chunks.push_back(c);
        }
    }
    grape_batch_plan* p = new (std::nothrow) grape_batch_plan();
    if (!p) return GRAPE_ERR_NOMEM;
    p->g = g;
    p->num_chunks = (long long)chunks.size();
    cudaError_t e = cudaMalloc(&p->d_reqs, sizeof(WalkConst) * wcs.size());
    if (e == cudaSuccess) e = cudaMalloc(&p->d_chunks, sizeof(Chunk) * chunks.size());
    if (e == cudaSuccess) e = cudaMalloc(&p->d_ctl, sizeof(unsigned long long) * 2);
    if (e == cudaSuccess)
        e = cudaMemcpy(p->d_reqs, wcs.data(), sizeof(WalkConst) * wcs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p->d_chunks, chunks.data(), sizeof(Chunk) * chunks.size(),
                       cudaMemcpyHostToDevice);
    unsigned long long ctl[2] = {0ull, (unsigned long long)chunks.size()};
    if (e == cudaSuccess) e = cudaMemcpy(p->d_ctl, ctl, sizeof(ctl), cudaMemcpyHostToDevice);
    // Capture: reset the queue head, then the persistent kernel.
    cudaStream_t cap = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e1 = cudaMemsetAsync(p->d_ctl, 0, sizeof(unsigned long long), cap);
        cudaError_t e2 = e1 == cudaSuccess
                             ? launch_queue_kernel(g, t, p->d_reqs, p->d_chunks, p->d_ctl,
                                                   (unsigned long long)chunks.size(), 0, nullptr,
                                                   nullptr, nullptr, 0, cap)
                             : e1;
        cudaError_t e3 = cudaStreamEndCapture(cap, &p->graph);
        e = e2 != cudaSuccess ? e2 : e3;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (cap) cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        free_plan(p);
        return grape::cuda_status(e);
    }
    *out = p;
    return GRAPE_OK;
}

extern "C" {

grape_status_t grape_walks(const grape_graph_t* g, const int32_t* starts, int64_t num_starts,
                           int32_t walk_len, int32_t walks_per_node, double p, double q,
                           uint64_t seed, int32_t* out, grape_stream_t stream) {
    WalkConst wc;
    grape_status_t st = make_walk_const(g, starts, num_starts, walk_len, walks_per_node, p, q,
                                        seed, out, &wc);
    if (st != GRAPE_OK) return st;
    const grape_tuning_t t = tuning_of(g);
    return grape::cuda_status(dispatch_walk(g, t, wc, p != 1.0, q != 1.0,
                                            reinterpret_cast<cudaStream_t>(stream)));
}

grape_status_t grape_walks_approx(const grape_graph_t* g, const int32_t* starts,
                                  int64_t num_starts, int32_t walk_len, int32_t walks_per_node,
                                  double p, double q, uint64_t seed, int32_t suss_k, int32_t* out,
                                  grape_stream_t stream) {
    if (suss_k < 0) return GRAPE_ERR_INVALID_ARG;
    WalkConst wc;
    grape_status_t st = make_walk_const(g, starts, num_starts, walk_len, walks_per_node, p, q,
                                        seed, out, &wc);
    if (st != GRAPE_OK) return st;
    wc.suss_k = suss_k;
    const grape_tuning_t t = tuning_of(g);
    return grape::cuda_status(dispatch_walk(g, t, wc, p != 1.0, q != 1.0,
                                            reinterpret_cast<cudaStream_t>(stream)));
}

grape_status_t grape_walks_range(const grape_graph_t* g, const int32_t* starts,
                                 int64_t num_starts, int32_t walk_len, int32_t walks_per_node,
                                 double p, double q, uint64_t seed, int64_t walk_begin,
                                 int64_t walk_count, int32_t* out, grape_stream_t stream) {
    WalkConst wc;
    grape_status_t st = make_walk_const(g, starts, num_starts, walk_len, walks_per_node, p, q,
                                        seed, out, &wc);
    if (st != GRAPE_OK) return st;
    st = restrict_walks(&wc, walk_begin, walk_count);
    if (st != GRAPE_OK) return st;
    if (walk_count == 0) return GRAPE_OK;
    const grape_tuning_t t = tuning_of(g);
    return grape::cuda_status(dispatch_walk(g, t, wc, p != 1.0, q != 1.0,
                                            reinterpret_cast<cudaStream_t>(stream)));
}

grape_status_t grape_walks_host(const grape_graph_t* g, const int32_t* starts, int64_t num_starts,
                                int32_t walk_len, int32_t walks_per_node, double p, double q,
                                uint64_t seed, int32_t* out, grape_stream_t stream_) {
    if (!g || !out) return GRAPE_ERR_INVALID_ARG;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    WalkConst probe;
    grape_status_t st = make_walk_const(g, starts, num_starts, walk_len, walks_per_node, p, q,
                                        seed, out, &probe);
    if (st != GRAPE_OK) return st;
    cudaStream_t copy = nullptr;
    if (host_copy_stream(&copy) != cudaSuccess) return GRAPE_ERR_CUDA;
    int32_t* d_starts = nullptr;
    int32_t* d_out = nullptr;
    const int64_t nw = probe.num_walks;
    const size_t row_bytes = sizeof(int32_t) * (size_t)walk_len;
    const size_t out_bytes = row_bytes * (size_t)nw;
    // Scratch comes from the device's stream-ordered pool, which keeps freed
    // blocks for reuse, so repeated calls do not pay for fresh allocations.
    static std::once_flag pool_once;
    std::call_once(pool_once, [] {
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    });
    // The rows leave in slices of walk ids: slice i is copied to the host on a
    // copy stream while the later slices are still being walked, so only the
    // last slice's copy is exposed.  A slice holds at least kHostSliceBytes of
    // rows and at least 16 walks per resident lane (each launch ends in a tail
    // of lanes finishing unevenly).  Slice bounds are multiples of 8 rows,
    // which keeps every slice's device rows 32-byte aligned.
    const int64_t lanes = (int64_t)g->num_sms * kMinBlocksWalk * kMaxThreads;
    const int64_t want = std::max<int64_t>(
        1, std::min<int64_t>({(int64_t)kHostSlices, (int64_t)(out_bytes / kHostSliceBytes),
                              nw / (16 * lanes)}));
    const int64_t per = ((nw + want - 1) / want + 7) / 8 * 8;
    const int nslices = (int)((nw + per - 1) / per);
    std::vector<cudaEvent_t> walked((size_t)nslices, nullptr);
    cudaEvent_t copied = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&copied, cudaEventDisableTiming);
    for (int i = 0; i < nslices && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&walked[(size_t)i], cudaEventDisableTiming);
    if (e == cudaSuccess && starts)
        e = cudaMallocAsync(&d_starts, sizeof(int32_t) * (size_t)num_starts, stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_out, out_bytes, stream);
    if (e == cudaSuccess && starts)
        e = cudaMemcpyAsync(d_starts, starts, sizeof(int32_t) * (size_t)num_starts,
                            cudaMemcpyHostToDevice, stream);
    int launched = 0;
    for (int i = 0; i < nslices && e == cudaSuccess && st == GRAPE_OK; ++i) {
        const int64_t b = (int64_t)i * per;
        const int64_t c = std::min<int64_t>(per, nw - b);
        st = grape_walks_range(g, d_starts, num_starts, walk_len, walks_per_node, p, q, seed, b, c,
                               d_out + (size_t)b * (size_t)walk_len, stream_);
        if (st == GRAPE_OK) e = cudaEventRecord(walked[(size_t)i], stream);
        if (st == GRAPE_OK && e == cudaSuccess) ++launched;
    }
    // Copies after all launches, so that a pageable destination (whose copies
    // block the host) still overlaps the walks of later slices.
    for (int i = 0; i < launched && e == cudaSuccess; ++i) {
        const int64_t b = (int64_t)i * per;
        const int64_t c = std::min<int64_t>(per, nw - b);
        e = cudaStreamWaitEvent(copy, walked[(size_t)i], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out + (size_t)b * (size_t)walk_len,
                                d_out + (size_t)b * (size_t)walk_len, row_bytes * (size_t)c,
                                cudaMemcpyDeviceToHost, copy);
    }
    // the scratch is freed on `stream` after the copies that read it
    cudaError_t e2 = cudaEventRecord(copied, copy);
    if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(stream, copied, 0);
    if (e2 != cudaSuccess) cudaStreamSynchronize(copy);
    if (d_starts) cudaFreeAsync(d_starts, stream);
    if (d_out) cudaFreeAsync(d_out, stream);
    const cudaError_t e3 = cudaStreamSynchronize(stream);
    for (cudaEvent_t ev : walked)
        if (ev) cudaEventDestroy(ev);
    if (copied) cudaEventDestroy(copied);
    if (st != GRAPE_OK) return st;
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = e3;
    return grape::cuda_status(e);
}

grape_status_t grape_batch_plan_create(const grape_graph_t* g, const grape_walk_request_t* reqs,
                                       int32_t n, grape_stream_t, grape_batch_plan_t** out) {
    if (!out) return GRAPE_ERR_INVALID_ARG;
    *out = nullptr;
    if (!g || !reqs || n < 1) return GRAPE_ERR_INVALID_ARG;
    return build_plan(g, reqs, n, tuning_of(g), out);
}

grape_status_t grape_batch_plan_launch(grape_batch_plan_t* p, grape_stream_t stream) {
    if (!p || !p->exec) return GRAPE_ERR_INVALID_ARG;
    return grape::cuda_status(cudaGraphLaunch(p->exec, reinterpret_cast<cudaStream_t>(stream)));
}

void grape_batch_plan_destroy(grape_batch_plan_t* p) {
    if (!p) return;
    cudaDeviceSynchronize();
    free_plan(p);
}

grape_status_t grape_walks_batched(const grape_graph_t* g, const grape_walk_request_t* reqs,
                                   int32_t n, grape_stream_t stream) {
    if (!g || !reqs || n < 1) return GRAPE_ERR_INVALID_ARG;
    grape_batch_plan* p = nullptr;
    grape_status_t st = build_plan(g, reqs, n, tuning_of(g), &p);
    if (st != GRAPE_OK) return st;
    st = grape_batch_plan_launch(p, stream);
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    free_plan(p);
    if (st != GRAPE_OK) return st;
    return grape::cuda_status(e);
}

grape_status_t grape_autotune_batched(grape_graph_t* g, const grape_walk_request_t* reqs,
                                      int32_t n, grape_stream_t stream_, grape_tuning_t* best) {
    if (!g || !reqs || n < 1) return GRAPE_ERR_INVALID_ARG;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    const grape_tuning_t base = tuning_of(g);
    const int chunk_grid[] = {16, 32, 64, 128, 256};
    const int shorter_grid[] = {8, 0x7fffffff};
    const int interp_grid[] = {0, 1};
    cudaEvent_t e0, e1;
    GRAPE_CUDA_TRY(cudaEventCreate(&e0));
    GRAPE_CUDA_TRY(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    grape_tuning_t best_t = base;
    grape_status_t result = GRAPE_OK;
    for (int cw : chunk_grid) {
        for (int sm : shorter_grid) for (int pw : interp_grid) {
            grape_tuning_t t = base;
            t.chunk_walks = cw;
            t.shorter_min = sm;
            t.interp_search = pw;
            grape_batch_plan* p = nullptr;
            grape_status_t st = build_plan(g, reqs, n, t, &p);
            if (st != GRAPE_OK) { result = st; break; }
            cudaError_t e = cudaGraphLaunch(p->exec, stream);           // warm-up
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventRecord(e0, stream);
            if (e == cudaSuccess) e = cudaGraphLaunch(p->exec, stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            free_plan(p);
            if (e != cudaSuccess) { result = grape::cuda_status(e); break; }
            if (ms < best_ms) {
                best_ms = ms;
                best_t = t;
            }
        }
        if (result != GRAPE_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result != GRAPE_OK) return result;
    {
        std::lock_guard<std::mutex> lk(g->mu);
        g->tuning.chunk_walks = best_t.chunk_walks;
        g->tuning.shorter_min = best_t.shorter_min;
        g->tuning.interp_search = best_t.interp_search;
    }
    if (best) *best = best_t;
    return GRAPE_OK;
}

grape_status_t grape_philox4x32_10(const uint32_t* ctr_key, int64_t n, uint32_t* out,
                                   grape_stream_t stream) {
    if (n < 0 || (n > 0 && (!ctr_key || !out))) return GRAPE_ERR_INVALID_ARG;
    if (n == 0) return GRAPE_OK;
    const long long blocks = std::min<long long>((n + 255) / 256, 65535);
    philox_kernel<<<(unsigned)blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(ctr_key, n, out);
    return grape::cuda_status(cudaGetLastError());
}

grape_status_t grape_sector_probe(const void* buf, int64_t buf_bytes, int64_t n_reads,
                                  uint64_t seed, int32_t mode, uint32_t* sink,
                                  grape_stream_t stream) {
    if (!buf || !sink || buf_bytes < 32 || n_reads < 1 || mode < 0 || mode > 2 ||
        (reinterpret_cast<uintptr_t>(buf) & 31u))
        return GRAPE_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    GRAPE_CUDA_TRY(cudaGetDevice(&dev));
    GRAPE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256;
    const long long blocks = (long long)sms * 8;
    const long long total_threads = blocks * threads;
    long long per_thread = (n_reads + total_threads - 1) / total_threads;
    per_thread = ((per_thread + 7) / 8) * 8;
    const unsigned long long nsec = (unsigned long long)(buf_bytes / 32);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int4* b4 = reinterpret_cast<const int4*>(buf);
    if (mode == 0) sector_probe_kernel<0><<<(unsigned)blocks, threads, 0, st>>>(b4, nsec, per_thread, seed, sink);
    else if (mode == 1) sector_probe_kernel<1><<<(unsigned)blocks, threads, 0, st>>>(b4, nsec, per_thread, seed, sink);
    else sector_probe_kernel<2><<<(unsigned)blocks, threads, 0, st>>>(b4, nsec, per_thread, seed, sink);
    return grape::cuda_status(cudaGetLastError());
}

}  // extern "C"
