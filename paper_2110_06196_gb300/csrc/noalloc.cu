// noalloc.cu -- batched walks that allocate nothing.
//
// grape_walks_batched builds its request table, queue entries and queue head
// in memory it allocates with cudaMalloc.  Some callers cannot allocate device
// memory at the moment they want walks: code running under a memory budget
// enforced by another allocator, code inside a region where allocation is
// forbidden, or callers on a device whose memory is already fully committed.
// For them, grape_walks_batched_static keeps the same state in one file-scope
// device array of fixed size instead.  It takes the queue entries implicitly
// from a prefix table (entry h belongs to the request whose prefix range holds
// h), so the array's size depends only on the number of requests.
//
// The array is a host-side stand-in in host code: the kernel gets the device
// address that cudaGetSymbolAddress returns, fetched once per device at set-up.
#include <cstring>
#include <mutex>

#include "internal.h"

using namespace grape;

namespace {

constexpr int kStaticMaxRequests = 4096;

struct StaticScratch {
    WalkConst reqs[kStaticMaxRequests];
    long long chunk_end[kStaticMaxRequests];   // inclusive prefix of per-request entry counts
    unsigned long long head;                   // next queue entry to take
};

constexpr size_t kStaticScratchBytes = (sizeof(StaticScratch) + 255) & ~size_t(255);

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_batch_scratch[kStaticScratchBytes];

// Per-device set-up, done by the first call on a device: the device address of
// g_batch_scratch and the walk kernel's resident blocks per SM.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
struct DeviceSetup {
    void* addr = nullptr;
    int per_sm[2][2] = {{0, 0}, {0, 0}};    // [weighted][counting]
};
DeviceSetup g_setup[kMaxDevices];

// Requests uploaded per table-fill launch.  The batch travels as a kernel
// parameter, which the launch copies, so nothing on the host has to outlive
// the call.
constexpr int kBatch = 32;
struct TableBatch {
    WalkConst reqs[kBatch];
    long long chunk_end[kBatch];
};

// Queue entries without a stored entry list: entry h is entry
// h - chunk_end[r - 1] of the request r whose prefix range holds h.
struct StaticQueueFeed {
    const StaticScratch* sc;
    unsigned long long* head;
    long long total_chunks;
    int num_reqs;
    int chunk_walks;
    long long cur_lo;
    int cur_left;
    int cur_req;
    bool drained;

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

    template <class C>
    __device__ __forceinline__ void finish(const Lane&, C& cnt, int) { cnt.add(C_WALKS); }
    __device__ __forceinline__ void drain() {}
    __device__ __forceinline__ void alphas(int req, double& a_ret, double& a_out) const {
        a_ret = sc->reqs[req].a_ret;
        a_out = sc->reqs[req].a_out;
    }

    __device__ __forceinline__ bool take_chunk(int lane) {
        long long lo = 0;
        int cnt = 0, rq = -1, ok = 0;
        if (lane == 0) {
            const unsigned long long h = atomicAdd(head, 1ull);
            if ((long long)h < total_chunks) {
                // request whose prefix range holds h: first r with chunk_end[r] > h
                int a = 0, b = num_reqs - 1;
                while (a < b) {
                    const int m = (a + b) >> 1;
                    if (sc->chunk_end[m] > (long long)h) b = m; else a = m + 1;
                }
                const long long first = a ? sc->chunk_end[a - 1] : 0;
                const long long nw = sc->reqs[a].num_walks;
                lo = ((long long)h - first) * chunk_walks;
                cnt = (int)((nw - lo) < chunk_walks ? (nw - lo) : chunk_walks);
                rq = a;
                ok = 1;
            }
        }
        ok = __shfl_sync(FULL, ok, 0);
        if (!ok) return false;
        cur_lo = __shfl_sync(FULL, lo, 0);
        cur_left = __shfl_sync(FULL, cnt, 0);
        cur_req = __shfl_sync(FULL, rq, 0);
        return true;
    }

    template <class C>
    __device__ __forceinline__ bool refill(const GraphDev& g, Lane& L, bool have, C& cnt) {
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
                have = begin_walk(g, sc->reqs[cur_req], cur_req, cur_lo + rank, L);
                if (have) set_wrec(sc->reqs[cur_req], cur_lo + rank);
                else finish(L, cnt, 0);
            }
            cur_lo += give;
            cur_left -= give;
        }
        return have;
    }
};

__global__ void table_fill_kernel(StaticScratch* sc, TableBatch b, int first, int count) {
    const int j = threadIdx.x;
    if (j < count) {
        sc->reqs[first + j] = b.reqs[j];
        sc->chunk_end[first + j] = b.chunk_end[j];
    }
}

template <bool W, bool COUNT>
__global__ void __launch_bounds__(256, 4)
static_queue_kernel(GraphDev g, const StaticScratch* sc, long long total_chunks, int num_reqs,
                    int chunk_walks, Policy pol) {
    StaticQueueFeed f;
    f.sc = sc;
    f.head = const_cast<unsigned long long*>(&sc->head);
    f.total_chunks = total_chunks;
    f.num_reqs = num_reqs;
    f.chunk_walks = chunk_walks;
    f.cur_lo = 0;
    f.cur_left = 0;
    f.cur_req = 0;
    f.drained = false;
    walk_loop<W, true, true, COUNT>(g, f, pol);
}

template <bool W, bool C>
cudaError_t occupancy(int threads, int* out) {
    int nb = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &nb, static_queue_kernel<W, C>, threads, (size_t)threads * kLaneSharedBytes);
    *out = nb < 1 ? 1 : nb;
    return e;
}

// The current device's set-up (done on first use, with that device current).
grape_status_t device_setup(int threads, StaticScratch** addr, const DeviceSetup** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GRAPE_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    DeviceSetup& d = g_setup[dev];
    if (!d.addr) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_batch_scratch);
        if (e != cudaSuccess || !p) return GRAPE_ERR_CUDA;
        if (e == cudaSuccess) e = occupancy<false, false>(threads, &d.per_sm[0][0]);
        if (e == cudaSuccess) e = occupancy<false, true>(threads, &d.per_sm[0][1]);
        if (e == cudaSuccess) e = occupancy<true, false>(threads, &d.per_sm[1][0]);
        if (e == cudaSuccess) e = occupancy<true, true>(threads, &d.per_sm[1][1]);
        if (e != cudaSuccess) return cuda_status(e);
        d.addr = p;
    }
    *addr = static_cast<StaticScratch*>(d.addr);
    *out = &d;
    return GRAPE_OK;
}

}  // namespace

extern "C" {

grape_status_t grape_walks_batched_static(const grape_graph_t* g,
                                          const grape_walk_request_t* reqs, int32_t n,
                                          grape_stream_t stream_) {
    if (!g || !reqs || n < 1) return GRAPE_ERR_INVALID_ARG;
    if (n > kStaticMaxRequests) return GRAPE_ERR_INVALID_ARG;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    grape_tuning_t t;
    grape_graph_get_tuning(g, &t);
    const int cw = t.chunk_walks;
    // Validate every request before touching the shared array.
    long long total = 0;
    for (int i = 0; i < n; ++i) {
        WalkConst wc;
        const grape_walk_request_t& r = reqs[i];
        const grape_status_t st = make_walk_const(g, r.starts, r.num_starts, r.walk_len,
                                                  r.walks_per_node, r.p, r.q, r.seed, r.out, &wc);
        if (st != GRAPE_OK) return st;
        total += (wc.num_walks + cw - 1) / cw;
    }
    // Blocks of the graph's tuned size (at most 256, the kernel's launch bounds).
    constexpr int kDefaultThreads = 256;
    const int threads = t.block_threads < kDefaultThreads ? t.block_threads : kDefaultThreads;
    StaticScratch* sc = nullptr;
    const DeviceSetup* dev = nullptr;
    grape_status_t st = device_setup(kDefaultThreads, &sc, &dev);
    if (st != GRAPE_OK) return st;
    long long run = 0;
    for (int i0 = 0; i0 < n; i0 += kBatch) {
        const int m = (n - i0) < kBatch ? (n - i0) : kBatch;
        TableBatch b;
        std::memset(&b, 0, sizeof(b));
        for (int j = 0; j < m; ++j) {
            const grape_walk_request_t& r = reqs[i0 + j];
            make_walk_const(g, r.starts, r.num_starts, r.walk_len, r.walks_per_node, r.p, r.q,
                            r.seed, r.out, &b.reqs[j]);
            run += (b.reqs[j].num_walks + cw - 1) / cw;
            b.chunk_end[j] = run;
        }
        table_fill_kernel<<<1, kBatch, 0, stream>>>(sc, b, i0, m);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_status(e);
    }
    // The queue head is the only state that must start at zero.
    cudaError_t e = cudaMemsetAsync(&sc->head, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return cuda_status(e);
    const int w = g->weighted ? 1 : 0, c = g->counting ? 1 : 0;
    int per_sm = t.blocks_per_sm;
    if (per_sm <= 0 && threads == kDefaultThreads) per_sm = dev->per_sm[w][c];
    if (per_sm <= 0) {
        e = w ? (c ? occupancy<true, true>(threads, &per_sm) : occupancy<true, false>(threads, &per_sm))
              : (c ? occupancy<false, true>(threads, &per_sm) : occupancy<false, false>(threads, &per_sm));
        if (e != cudaSuccess) return cuda_status(e);
    }
    const int blocks = g->num_sms * per_sm;
    const size_t sh = (size_t)threads * kLaneSharedBytes;
#define GRAPE_STATIC_LAUNCH(W, C)                                                              \
    static_queue_kernel<W, C><<<blocks, threads, sh, stream>>>(                                 \
        g->dev(), sc, total, n, cw, policy_of(t))
    if (g->weighted) {
        if (g->counting) GRAPE_STATIC_LAUNCH(true, true);
        else GRAPE_STATIC_LAUNCH(true, false);
    } else {
        if (g->counting) GRAPE_STATIC_LAUNCH(false, true);
        else GRAPE_STATIC_LAUNCH(false, false);
    }
#undef GRAPE_STATIC_LAUNCH
    return cuda_status(cudaGetLastError());
}

}  // extern "C"
