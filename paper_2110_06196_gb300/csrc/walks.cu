// walks.cu -- per-call walks, batched walks (persistent queue kernel replayed
// from a CUDA graph), the batched-path autotuner, and diagnostics.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "internal.h"

using namespace grape;

namespace {

constexpr int kMaxThreads = 256;
// Resident blocks per SM the register allocation is held to: more warps keep
// more independent gathers in flight, which is what this latency-bound loop
// needs (4 x 256 threads -> at most 64 registers per thread).
#ifndef GRAPE_MIN_BLOCKS_WALK
#define GRAPE_MIN_BLOCKS_WALK 4
#endif
constexpr int kMinBlocksWalk = GRAPE_MIN_BLOCKS_WALK;
constexpr int kMinBlocksQueue = 4;

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

// Per-call walk kernel: the eight specialisations of GRAPE ("Implementation of
// second-order RWs": p == 1, q == 1, weighted or not) as template arguments.
// COUNT: the instantiation that also keeps the work counters.
// MODE 1: the approximated walks (GRAPE, Methods, "Approximated RWs"); MODE 2:
// the exact walks with the optional long-list search schedules (sector pivots,
// warp-cooperative narrowing); both only with the general p, q specialisation.
constexpr int kExact = 0, kSuss = 1, kHub = 2;

template <bool W, bool P, bool Q, bool COUNT, int MODE = kExact>
__global__ void __launch_bounds__(kMaxThreads, kMinBlocksWalk)
walk_kernel(GraphDev g, WalkConst wc, RoundKeys rk, SliceSink sink, Policy pol) {
    GridFeed<MODE == kSuss> f;
    f.wc = &wc;
    f.rk = &rk;
    f.sink = &sink;
    if (sink.walks_per_slice > 0) {
        SliceTally* st = slice_tally();
        st->slice = -1;
        st->count = 0;
    }
    f.next = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    f.stride = (long long)gridDim.x * blockDim.x;
    walk_loop<W, P, Q, COUNT, MODE == kHub>(g, f, pol);
}

// Batched / served kernel: persistent grid draining a queue of walk ranges.
// HUB: with the optional long-list search schedules.
template <bool W, bool COUNT, bool HUB = false>
__global__ void __launch_bounds__(kMaxThreads, kMinBlocksQueue)
queue_kernel(GraphDev g, const WalkConst* reqs, const Chunk* chunks, unsigned long long* ctl,
             unsigned long long ring, long long idle_spins, int* exit_flag,
             unsigned long long* done, unsigned* done_flags, Policy pol) {
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
    walk_loop<W, true, true, COUNT, HUB>(g, f, pol);
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

// Random-sector gather probe: the ceiling of independent random 32-byte
// reads.  Each thread keeps LOADS reads in flight, each of WIDTH bytes (4, 16
// or 32: one 32-bit, 128-bit or 256-bit load) at the start of a random aligned
// 32-byte sector, then folds what arrived into a checksum.  MODE picks the
// cache path: 0 ld.global.nc (read-only, through L1), 1 ld.global.cg (L2
// only), 2 ld.global.cs (streaming).  Positions come from the SplitMix64 output
// function of a per-thread counter (cheap next to a Philox block, so the
// probe measures the memory system, not the generator).
__device__ __forceinline__ unsigned long long probe_mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// One sector read of WIDTH bytes into w[0 .. WIDTH/4).  Volatile, so the
// loads stay above the warp barrier that precedes the fold.
template <int WIDTH, int MODE>
__device__ __forceinline__ void probe_load(const char* p, unsigned* w) {
    if (WIDTH == 4) {
        if (MODE == 0) asm volatile("ld.global.nc.u32 %0, [%1];" : "=r"(w[0]) : "l"(p));
        else if (MODE == 1) asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(w[0]) : "l"(p));
        else asm volatile("ld.global.cs.u32 %0, [%1];" : "=r"(w[0]) : "l"(p));
    } else if (WIDTH == 16) {
        if (MODE == 0)
            asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
                : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]) : "l"(p));
        else if (MODE == 1)
            asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
                : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]) : "l"(p));
        else
            asm volatile("ld.global.cs.v4.u32 {%0, %1, %2, %3}, [%4];"
                : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]) : "l"(p));
    } else {
        if (MODE == 0)
            asm volatile("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]),
                  "=r"(w[6]), "=r"(w[7]) : "l"(p));
        else if (MODE == 1)
            asm volatile("ld.global.cg.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]),
                  "=r"(w[6]), "=r"(w[7]) : "l"(p));
        else
            asm volatile("ld.global.cs.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]),
                  "=r"(w[6]), "=r"(w[7]) : "l"(p));
    }
}

// WIDTH 64: both 32-byte sectors of a random aligned 64-byte block (two
// 256-bit loads), to see what the second sector of a DRAM burst costs.
template <int LOADS, int WIDTH, int MODE>
__global__ void __launch_bounds__(256)
sector_probe_kernel(const char* __restrict__ buf, unsigned long long nsec, long long rounds,
                    unsigned long long seed, uint32_t* sink) {
    constexpr int WORDS = WIDTH / 4;
    constexpr int STRIDE = WIDTH == 64 ? 64 : 32;
    const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    unsigned long long ctr = probe_mix(seed ^ (tid * 0x9E3779B97F4A7C15ull));
    const unsigned long long nblk = WIDTH == 64 ? nsec / 2 : nsec;
    unsigned acc = 0;
    for (long long j = 0; j < rounds; ++j) {
        unsigned v[LOADS * WORDS];
#pragma unroll
        for (int u = 0; u < LOADS; ++u) {
            ctr += 0x9E3779B97F4A7C15ull;
            const unsigned long long idx = __umul64hi(probe_mix(ctr), nblk);
            if (WIDTH == 64) {
                probe_load<32, MODE>(buf + STRIDE * idx, v + u * WORDS);
                probe_load<32, MODE>(buf + STRIDE * idx + 32, v + u * WORDS + 8);
            } else {
                probe_load<WIDTH, MODE>(buf + STRIDE * idx, v + u * WORDS);
            }
        }
        // The fold mixes in a value read after the last load is issued, so no
        // fold can start before every read of the round is in flight.
        unsigned k;
        asm volatile("mov.u32 %0, %%clock;" : "=r"(k));
#pragma unroll
        for (int u = 0; u < LOADS * WORDS; ++u) acc ^= v[u] + k;
    }
    if (acc == 0x9e3779b9u) atomicXor(sink, acc);   // practically never; keeps the loads live
}

// The probe's (loads, width) pairs: at most 128 registers of loads in flight.
template <int LOADS, int WIDTH>
cudaError_t launch_probe_lw(int mode, const char* buf, unsigned long long nsec, long long n_reads,
                            unsigned long long seed, uint32_t* sink, int num_sms, int blocks_per_sm,
                            int* resident, long long* reads_done, cudaStream_t st) {
    auto k = mode == 0 ? sector_probe_kernel<LOADS, WIDTH, 0>
                       : (mode == 1 ? sector_probe_kernel<LOADS, WIDTH, 1>
                                    : sector_probe_kernel<LOADS, WIDTH, 2>);
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, 256, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    const int per_sm = blocks_per_sm > 0 ? std::min(blocks_per_sm, occ) : occ;
    const long long threads = (long long)num_sms * per_sm * 256;
    const long long rounds = std::max<long long>(1, (n_reads + threads * LOADS - 1) / (threads * LOADS));
    k<<<(unsigned)(num_sms * per_sm), 256, 0, st>>>(buf, nsec, rounds, seed, sink);
    if (resident) *resident = per_sm;
    if (reads_done) *reads_done = rounds * threads * LOADS * (WIDTH == 64 ? 2 : 1);
    return cudaGetLastError();
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

template <bool W, bool P, bool Q, bool C, int S = kExact>
cudaError_t launch_walk_c(const grape_graph* g, const grape_tuning_t& t, const WalkConst& wc,
                          const SliceSink& sink, cudaStream_t stream) {
    const int threads = std::min(t.block_threads, kMaxThreads);
    int per_sm = t.blocks_per_sm;
    if (per_sm <= 0) per_sm = occupancy_blocks(walk_kernel<W, P, Q, C, S>, threads);
    long long blocks = (wc.num_walks + threads - 1) / threads;
    const long long cap = (long long)g->num_sms * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = stage_bytes(threads);
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = (unsigned)walk_launch_attrs(g, t, attr);
    return cudaLaunchKernelEx(&cfg, walk_kernel<W, P, Q, C, S>, g->dev(), wc, round_keys(wc.seed),
                              sink, policy_of(t));
}

template <bool W, bool P, bool Q>
cudaError_t launch_walk(const grape_graph* g, const grape_tuning_t& t, const WalkConst& wc,
                        const SliceSink& k, cudaStream_t stream) {
    return g->counting ? launch_walk_c<W, P, Q, true>(g, t, wc, k, stream)
                       : launch_walk_c<W, P, Q, false>(g, t, wc, k, stream);
}

constexpr SliceSink kNoSlices = {nullptr, nullptr, 0, 0};

// Does the tuning turn on a long-list search schedule (the HUB kernels)?
bool hub_schedules(const grape_tuning_t& t) {
    return t.pivot_min != 0x7fffffff || t.warp_search_min != 0x7fffffff;
}

cudaError_t dispatch_walk(const grape_graph* g, const grape_tuning_t& t, const WalkConst& wc,
                          bool has_p, bool has_q, cudaStream_t s,
                          const SliceSink& k = kNoSlices) {
    if (wc.suss_k > 0) {
        if (g->weighted)
            return g->counting ? launch_walk_c<true, true, true, true, kSuss>(g, t, wc, k, s)
                               : launch_walk_c<true, true, true, false, kSuss>(g, t, wc, k, s);
        return g->counting ? launch_walk_c<false, true, true, true, kSuss>(g, t, wc, k, s)
                           : launch_walk_c<false, true, true, false, kSuss>(g, t, wc, k, s);
    }
    if (hub_schedules(t)) {
        if (g->weighted)
            return g->counting ? launch_walk_c<true, true, true, true, kHub>(g, t, wc, k, s)
                               : launch_walk_c<true, true, true, false, kHub>(g, t, wc, k, s);
        return g->counting ? launch_walk_c<false, true, true, true, kHub>(g, t, wc, k, s)
                           : launch_walk_c<false, true, true, false, kHub>(g, t, wc, k, s);
    }
    if (g->weighted) {
        if (has_p) return has_q ? launch_walk<true, true, true>(g, t, wc, k, s)
                                : launch_walk<true, true, false>(g, t, wc, k, s);
        return has_q ? launch_walk<true, false, true>(g, t, wc, k, s)
                     : launch_walk<true, false, false>(g, t, wc, k, s);
    }
    if (has_p) return has_q ? launch_walk<false, true, true>(g, t, wc, k, s)
                            : launch_walk<false, true, false>(g, t, wc, k, s);
    return has_q ? launch_walk<false, false, true>(g, t, wc, k, s)
                 : launch_walk<false, false, false>(g, t, wc, k, s);
}

bool valid_pq(double x) { return std::isfinite(x) && x > 0.0; }

// grape_walks_host: at most this many slices, of at least this many bytes.
constexpr int kHostSlices = 64;
constexpr size_t kHostSliceBytes = 64u << 20;

// Non-blocking streams per device for grape_walks_host's copies out; slices
// go round-robin over them.  While the walks run, the copies compete with the
// walk kernel's random reads for the memory system; on the R-MAT scale-24 job
// two streams measured 380-425 ms a call against 690-750 ms for one or four.
#ifndef GRAPE_COPY_STREAMS
#define GRAPE_COPY_STREAMS 2
#endif
constexpr int kCopyStreams = GRAPE_COPY_STREAMS;

cudaError_t host_copy_streams(cudaStream_t* out) {
    static std::mutex mu;
    static cudaStream_t streams[64][kCopyStreams] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    for (int i = 0; i < kCopyStreams; ++i) {
        if (!streams[dev][i]) {
            e = cudaStreamCreateWithFlags(&streams[dev][i], cudaStreamNonBlocking);
            if (e != cudaSuccess) return e;
        }
        out[i] = streams[dev][i];
    }
    return cudaSuccess;
}

// Slice-completion flags in mapped host memory (kHostSlices per array), kept
// per device and reused: a call takes an array and gives it back, so
// concurrent calls never share one and no call pays for a pinned allocation
// after the first.
struct SliceFlags {
    unsigned* host = nullptr;
    unsigned* dev = nullptr;
};

std::mutex g_flags_mu;
std::vector<SliceFlags> g_flags_free[64];

cudaError_t take_slice_flags(int dev, SliceFlags* out) {
    {
        std::lock_guard<std::mutex> lk(g_flags_mu);
        if (!g_flags_free[dev].empty()) {
            *out = g_flags_free[dev].back();
            g_flags_free[dev].pop_back();
            return cudaSuccess;
        }
    }
    SliceFlags f;
    cudaError_t e = cudaHostAlloc(&f.host, sizeof(unsigned) * kHostSlices, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&f.dev, f.host, 0);
    if (e != cudaSuccess) {
        if (f.host) cudaFreeHost(f.host);
        return e;
    }
    *out = f;
    return cudaSuccess;
}

void give_slice_flags(int dev, const SliceFlags& f) {
    std::lock_guard<std::mutex> lk(g_flags_mu);
    g_flags_free[dev].push_back(f);
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
    const Policy pol = policy_of(t);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)nb);
    cfg.blockDim = dim3((unsigned)s.threads);
    cfg.dynamicSmemBytes = sh;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = (unsigned)walk_launch_attrs(g, t, attr);
    const GraphDev gd = g->dev();
#define GRAPE_QUEUE_LAUNCH(W, C, H)                                                           \
    cudaLaunchKernelEx(&cfg, queue_kernel<W, C, H>, gd, reqs, chunks, ctl, ring, idle_spins,  \
                       exit_flag, done, done_flags, pol)
    if (hub_schedules(t)) {
        if (g->weighted)
            return g->counting ? GRAPE_QUEUE_LAUNCH(true, true, true)
                               : GRAPE_QUEUE_LAUNCH(true, false, true);
        return g->counting ? GRAPE_QUEUE_LAUNCH(false, true, true)
                           : GRAPE_QUEUE_LAUNCH(false, false, true);
    }
    if (g->weighted)
        return g->counting ? GRAPE_QUEUE_LAUNCH(true, true, false)
                           : GRAPE_QUEUE_LAUNCH(true, false, false);
    return g->counting ? GRAPE_QUEUE_LAUNCH(false, true, false)
                       : GRAPE_QUEUE_LAUNCH(false, false, false);
#undef GRAPE_QUEUE_LAUNCH
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
    WalkConst wc;
    grape_status_t st = make_walk_const(g, starts, num_starts, walk_len, walks_per_node, p, q,
                                        seed, out, &wc);
    if (st != GRAPE_OK) return st;
    int dev = 0;
    GRAPE_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return GRAPE_ERR_CUDA;
    cudaStream_t copy[kCopyStreams] = {};
    GRAPE_CUDA_TRY(host_copy_streams(copy));
    const int64_t nw = wc.num_walks;
    const size_t row_bytes = sizeof(int32_t) * (size_t)walk_len;
    const size_t out_bytes = row_bytes * (size_t)nw;
    // Scratch comes from the device's stream-ordered pool, which keeps freed
    // blocks for reuse, so repeated calls do not pay for fresh allocations.
    static std::once_flag pool_once;
    std::call_once(pool_once, [] {
        int d = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&d) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, d) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    });
    // One launch walks the whole job.  Its rows are cut into slices of walk
    // ids (at least kHostSliceBytes each, at most kHostSlices); the walk that
    // completes a slice raises that slice's flag in mapped host memory, and
    // this thread then copies the slice out on the copy stream while the
    // launch goes on.  Lanes take walk ids in grid-stride order, so slices
    // complete roughly in order and only the last slice's copy is exposed.
    const int64_t want = std::max<int64_t>(
        1, std::min<int64_t>((int64_t)kHostSlices, (int64_t)(out_bytes / kHostSliceBytes)));
    const int64_t per = ((nw + want - 1) / want + 7) / 8 * 8;
    const int nslices = (int)((nw + per - 1) / per);
    SliceFlags flags;
    GRAPE_CUDA_TRY(take_slice_flags(dev, &flags));
    for (int i = 0; i < nslices; ++i) flags.host[i] = 0u;
    int32_t* d_starts = nullptr;
    int32_t* d_out = nullptr;
    unsigned long long* d_done = nullptr;
    cudaEvent_t walked = nullptr, copied[kCopyStreams] = {};
    cudaError_t e = cudaEventCreateWithFlags(&walked, cudaEventDisableTiming);
    for (int i = 0; i < kCopyStreams && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&copied[i], cudaEventDisableTiming);
    if (e == cudaSuccess && starts)
        e = cudaMallocAsync(&d_starts, sizeof(int32_t) * (size_t)num_starts, stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_out, out_bytes, stream);
    if (e == cudaSuccess)
        e = cudaMallocAsync(&d_done, sizeof(unsigned long long) * (size_t)nslices, stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(d_done, 0, sizeof(unsigned long long) * (size_t)nslices, stream);
    if (e == cudaSuccess && starts)
        e = cudaMemcpyAsync(d_starts, starts, sizeof(int32_t) * (size_t)num_starts,
                            cudaMemcpyHostToDevice, stream);
    bool launched = false;
    if (e == cudaSuccess) {
        wc.starts = d_starts;
        wc.out = d_out;
        wc.out_vec = ((reinterpret_cast<uintptr_t>(d_out) & 31u) == 0) ? 1 : 0;
        const SliceSink sink = {d_done, flags.dev, per, nw};
        e = dispatch_walk(g, tuning_of(g), wc, p != 1.0, q != 1.0, stream, sink);
        if (e == cudaSuccess) e = cudaEventRecord(walked, stream);
        launched = e == cudaSuccess;
    }
    // Copy each slice out once its flag is up.  Should the launch end with a
    // flag still down, the remaining slices are copied after the launch.
    int next = 0;
    bool after_launch = false;
    while (launched && next < nslices && e == cudaSuccess) {
        const bool ready = after_launch || ((volatile unsigned*)flags.host)[next] != 0u;
        if (ready) {
            const int64_t b = (int64_t)next * per;
            const int64_t c = std::min<int64_t>(per, nw - b);
            e = cudaMemcpyAsync(out + (size_t)b * (size_t)walk_len,
                                d_out + (size_t)b * (size_t)walk_len, row_bytes * (size_t)c,
                                cudaMemcpyDeviceToHost, copy[next % kCopyStreams]);
            ++next;
            continue;
        }
        const cudaError_t qe = cudaEventQuery(walked);
        if (qe == cudaSuccess) {
            after_launch = true;
            for (int i = 0; i < kCopyStreams && e == cudaSuccess; ++i)
                e = cudaStreamWaitEvent(copy[i], walked, 0);
        } else if (qe != cudaErrorNotReady) {
            e = qe;
        } else {
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    }
    // the scratch is freed on `stream` after the copies that read it
    cudaError_t e2 = cudaSuccess;
    for (int i = 0; i < kCopyStreams; ++i) {
        cudaError_t ei = copied[i] ? cudaEventRecord(copied[i], copy[i]) : cudaErrorInvalidValue;
        if (ei == cudaSuccess) ei = cudaStreamWaitEvent(stream, copied[i], 0);
        if (ei != cudaSuccess) {
            cudaStreamSynchronize(copy[i]);
            e2 = ei;
        }
    }
    if (d_starts) cudaFreeAsync(d_starts, stream);
    if (d_out) cudaFreeAsync(d_out, stream);
    if (d_done) cudaFreeAsync(d_done, stream);
    const cudaError_t e3 = cudaStreamSynchronize(stream);
    if (walked) cudaEventDestroy(walked);
    for (int i = 0; i < kCopyStreams; ++i)
        if (copied[i]) cudaEventDestroy(copied[i]);
    // the flags array is free once the launch that writes it has finished
    if (e3 == cudaSuccess) give_slice_flags(dev, flags);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = e3;
    return grape::cuda_status(e);
}

grape_status_t grape_trim_scratch(int64_t keep_bytes) {
    if (keep_bytes < 0) return GRAPE_ERR_INVALID_ARG;
    int dev = 0;
    cudaMemPool_t pool;
    GRAPE_CUDA_TRY(cudaGetDevice(&dev));
    GRAPE_CUDA_TRY(cudaDeviceGetDefaultMemPool(&pool, dev));
    GRAPE_CUDA_TRY(cudaDeviceSynchronize());
    return grape::cuda_status(cudaMemPoolTrimTo(pool, (size_t)keep_bytes));
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
    cudaEvent_t e0, e1;
    GRAPE_CUDA_TRY(cudaEventCreate(&e0));
    GRAPE_CUDA_TRY(cudaEventCreate(&e1));
    // Time one tuning: build its plan, one warm-up replay, one timed replay.
    auto time_one = [&](const grape_tuning_t& t, float* ms) -> grape_status_t {
        grape_batch_plan* p = nullptr;
        grape_status_t st = build_plan(g, reqs, n, t, &p);
        if (st != GRAPE_OK) return st;
        cudaError_t e = cudaGraphLaunch(p->exec, stream);
        if (e == cudaSuccess) e = cudaEventRecord(e0, stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(p->exec, stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
        free_plan(p);
        return grape::cuda_status(e);
    };
    float best_ms = 1e30f;
    grape_tuning_t best_t = base;
    grape_status_t result = GRAPE_OK;
    // Stage 1: queue granularity and list policy.
    const int chunk_grid[] = {16, 32, 64, 128, 256};
    const int shorter_grid[] = {8, 0x7fffffff};
    const int interp_grid[] = {0, 1};
    for (int cw : chunk_grid) {
        for (int sm : shorter_grid) {
            for (int pw : interp_grid) {
                if (result != GRAPE_OK) break;
                grape_tuning_t t = base;
                t.chunk_walks = cw;
                t.shorter_min = sm;
                t.interp_search = pw;
                float ms = 0.f;
                result = time_one(t, &ms);
                if (result == GRAPE_OK && ms < best_ms) {
                    best_ms = ms;
                    best_t = t;
                }
            }
        }
    }
    // Stage 2, from the best of stage 1: the hub thresholds (sector pivots
    // from a list length on; warp-cooperative narrowing above one).
    const int pivot_grid[] = {0x7fffffff, 32, 128, 512, 2048};
    const int warp_grid[] = {0x7fffffff, 1024, 8192};
    const grape_tuning_t stage1 = best_t;
    for (int pv : pivot_grid) {
        for (int wm : warp_grid) {
            if (result != GRAPE_OK) break;
            if (pv == stage1.pivot_min && wm == stage1.warp_search_min) continue;
            grape_tuning_t t = stage1;
            t.pivot_min = pv;
            t.warp_search_min = wm;
            float ms = 0.f;
            result = time_one(t, &ms);
            if (result == GRAPE_OK && ms < best_ms) {
                best_ms = ms;
                best_t = t;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result != GRAPE_OK) return result;
    {
        std::lock_guard<std::mutex> lk(g->mu);
        g->tuning.chunk_walks = best_t.chunk_walks;
        g->tuning.shorter_min = best_t.shorter_min;
        g->tuning.interp_search = best_t.interp_search;
        g->tuning.pivot_min = best_t.pivot_min;
        g->tuning.warp_search_min = best_t.warp_search_min;
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
                                  uint64_t seed, int32_t mode, int32_t load_bytes,
                                  int32_t loads_in_flight, int32_t blocks_per_sm, uint32_t* sink,
                                  int32_t* resident_blocks_per_sm, int64_t* reads_done,
                                  grape_stream_t stream) {
    if (!buf || !sink || buf_bytes < 64 || n_reads < 1 || mode < 0 || mode > 2 ||
        blocks_per_sm < 0 || (reinterpret_cast<uintptr_t>(buf) & 31u))
        return GRAPE_ERR_INVALID_ARG;
    const bool ok_shape = (load_bytes == 4 && (loads_in_flight == 8 || loads_in_flight == 16 ||
                                               loads_in_flight == 32 || loads_in_flight == 64)) ||
                          (load_bytes == 16 && (loads_in_flight == 8 || loads_in_flight == 16 ||
                                                loads_in_flight == 32)) ||
                          (load_bytes == 32 && (loads_in_flight == 4 || loads_in_flight == 8 ||
                                                loads_in_flight == 16)) ||
                          (load_bytes == 64 && (loads_in_flight == 4 || loads_in_flight == 8));
    if (!ok_shape) return GRAPE_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    GRAPE_CUDA_TRY(cudaGetDevice(&dev));
    GRAPE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned long long nsec = (unsigned long long)(buf_bytes / 32);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const char* b = static_cast<const char*>(buf);
    int res = 0;
    long long done = 0;
    cudaError_t e = cudaSuccess;
#define GRAPE_PROBE(L, W)                                                                        \
    e = launch_probe_lw<L, W>(mode, b, nsec, n_reads, seed, sink, sms, blocks_per_sm, &res, &done, st)
    if (load_bytes == 4) {
        if (loads_in_flight == 8) GRAPE_PROBE(8, 4);
        else if (loads_in_flight == 16) GRAPE_PROBE(16, 4);
        else if (loads_in_flight == 32) GRAPE_PROBE(32, 4);
        else GRAPE_PROBE(64, 4);
    } else if (load_bytes == 16) {
        if (loads_in_flight == 8) GRAPE_PROBE(8, 16);
        else if (loads_in_flight == 16) GRAPE_PROBE(16, 16);
        else GRAPE_PROBE(32, 16);
    } else if (load_bytes == 32) {
        if (loads_in_flight == 4) GRAPE_PROBE(4, 32);
        else if (loads_in_flight == 8) GRAPE_PROBE(8, 32);
        else GRAPE_PROBE(16, 32);
    } else {
        if (loads_in_flight == 4) GRAPE_PROBE(4, 64);
        else GRAPE_PROBE(8, 64);
    }
#undef GRAPE_PROBE
    if (resident_blocks_per_sm) *resident_blocks_per_sm = res;
    if (reads_done) *reads_done = done;
    return grape::cuda_status(e);
}

}  // extern "C"
