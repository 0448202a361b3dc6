// internal.h -- host-side definitions shared by the library's translation units.
#pragma once
#include <atomic>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/grape_walk.h"
#include "walk_device.cuh"

struct grape_graph {
    int64_t n = 0;
    int64_t m = 0;
    int32_t max_degree = 0;
    bool weighted = false;
    bool undirected = false;
    int device = 0;
    int num_sms = 0;
    int max_window = 0;           // cudaDevAttrMaxAccessPolicyWindowSize
    int4* rec = nullptr;          // NodeRec[n]
    int32_t* dsts = nullptr;      // [m + 8]
    int32_t* piv = nullptr;       // [ceil(m / 8) + 8] sector pivots: piv[j] = dsts[8 j]
    unsigned* eh = nullptr;       // edge hash [2^eh_b][8] (see walk_device.cuh), or nullptr
    int eh_k = 0, eh_b = 0;
    int64_t eh_bytes = 0;
    bool pair_filters = false;    // unweighted entries hold filters of N(v) n N(x), not of N(x)
    int4* fat = nullptr;          // [m] proposal entries (edge-inlined records)
    int* status = nullptr;        // device status word
    unsigned long long* counters = nullptr;  // [grape::C_COUNT]
    bool counting = false;
    int64_t device_bytes = 0;
    grape_tuning_t tuning{};
    std::mutex mu;                // guards tuning / counting updates

    grape::GraphDev dev() const {
        grape::GraphDev g;
        g.rec = rec;
        g.dsts = dsts;
        g.fat = fat;
        g.piv = piv;
        g.eh = eh;
        g.eh_k = eh_k;
        g.eh_b = eh_b;
        g.pair_filters = pair_filters ? 1 : 0;
        g.n = n;
        g.status = status;
        g.counters = counting ? counters : nullptr;
        g.undirected = undirected ? 1 : 0;
        return g;
    }
};

namespace grape {

// Fill the per-request constants from (p, q, seed, ...): the three class
// thresholds T = floor(alpha / max(1/p, 1, 1/q) * 2^32), stored as T - 1.
grape_status_t make_walk_const(const grape_graph* g, const int32_t* starts, int64_t num_starts,
                               int32_t walk_len, int32_t walks_per_node, double p, double q,
                               uint64_t seed, int32_t* out, WalkConst* wc);

// The same for a graph of num_nodes nodes held in another store.
grape_status_t make_walk_const_n(int64_t num_nodes, const int32_t* starts, int64_t num_starts,
                                 int32_t walk_len, int32_t walks_per_node, double p, double q,
                                 uint64_t seed, int32_t* out, WalkConst* wc);

// Restrict wc to the walk ids [walk_begin, walk_begin + walk_count).
grape_status_t restrict_walks(WalkConst* wc, int64_t walk_begin, int64_t walk_count);

// Launch configuration of the walk kernels for this graph's tuning.
struct LaunchShape {
    int threads;
    int blocks;
};

LaunchShape queue_launch_shape(const grape_graph* g, const grape_tuning_t& t, int weighted);

// Launch the queue (batched / served) kernel.
// ctl[0] is the queue head and ctl[1] the published tail; done (two counters per
// request: finished walks, transitions taken) and done_flags (host-mapped) are
// the per-request completion state of a served queue (nullptr for batched
// launches).
cudaError_t launch_queue_kernel(const grape_graph* g, const grape_tuning_t& t,
                                const WalkConst* reqs, const Chunk* chunks,
                                unsigned long long* ctl, unsigned long long ring,
                                long long idle_spins, int* exit_flag, unsigned long long* done,
                                unsigned* done_flags, int blocks, cudaStream_t stream);

inline Policy policy_of(const grape_tuning_t& t) {
    Policy p;
    p.trial_cap = (unsigned)t.trial_cap;
    p.shorter_min = t.shorter_min;
    p.interp_search = t.interp_search;
    p.pivot_min = t.pivot_min;
    p.warp_search_min = t.warp_search_min;
    p.edge_hash = t.edge_hash;
    return p;
}

// The launch attribute of a walk launch: with l2_persist_mb > 0, a persisting
// access-policy window over the graph's sector pivots (hit ratio: the share of
// the window the set-aside can hold).  Returns the number of attributes (0 or 1).
inline int walk_launch_attrs(const grape_graph* g, const grape_tuning_t& t,
                             cudaLaunchAttribute* attr) {
    if (t.l2_persist_mb <= 0 || !g->piv || g->max_window <= 0) return 0;
    const size_t bytes = sizeof(int32_t) * (size_t)((g->m + 7) / 8 + 8);
    const size_t win = bytes < (size_t)g->max_window ? bytes : (size_t)g->max_window;
    const double ratio = (double)((size_t)t.l2_persist_mb << 20) / (double)win;
    attr->id = cudaLaunchAttributeAccessPolicyWindow;
    attr->val.accessPolicyWindow.base_ptr = g->piv;
    attr->val.accessPolicyWindow.num_bytes = win;
    attr->val.accessPolicyWindow.hitRatio = (float)(ratio < 1.0 ? ratio : 1.0);
    attr->val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    attr->val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    return 1;
}

inline grape_status_t cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return GRAPE_OK;
    if (e == cudaErrorMemoryAllocation) return GRAPE_ERR_NOMEM;
    return GRAPE_ERR_CUDA;
}

}  // namespace grape

#define GRAPE_CUDA_TRY(expr)                                   \
    do {                                                       \
        cudaError_t _e = (expr);                               \
        if (_e != cudaSuccess) return grape::cuda_status(_e);  \
    } while (0)
