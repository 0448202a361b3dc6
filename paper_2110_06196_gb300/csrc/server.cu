// server.cu -- continuous-batching walk server.
//
// The graph stays resident.  Requests are admitted while output-arena bytes,
// request slots and queue entries allow (FIFO, no overtaking).  An admitted
// request is cut into queue entries of `chunk_walks` walks, and those are
// appended to a device ring that a resident queue kernel is draining.  The
// kernel's workers take entries with a compare-and-swap that never passes the
// published tail, so work that is admitted while the kernel runs joins it at
// once.  Each finished walk bumps its request's counter.  The last one raises a
// completion flag in mapped host memory.  The driver thread then copies the
// rows to the caller's host buffer on a separate copy stream while the kernel
// keeps working, and frees the arena bytes.
//
// Waits are bounded on both sides.  Warps without walks poll the tail; the
// driver raises an exit flag once nothing has been in flight for
// `idle_exit_us`, and relaunches the kernel when work is queued and no kernel
// is running.  Shutdown raises the same flag, which the kernel reads before
// taking each entry.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

using namespace grape;

namespace {

using Clock = std::chrono::steady_clock;

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch())
        .count();
}

// First-fit allocator over [0, cap) with coalescing; 256-byte granules.
class Arena {
  public:
    explicit Arena(int64_t cap) : cap_(cap) { free_[0] = cap; }
    static int64_t round(int64_t b) { return (b + 255) & ~int64_t(255); }
    bool alloc(int64_t bytes, int64_t* off) {
        bytes = round(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const int64_t rest = it->second - bytes;
                const int64_t start = it->first + bytes;
                free_.erase(it);
                if (rest > 0) free_[start] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(int64_t off, int64_t bytes) {
        bytes = round(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    int64_t used() const { return used_; }

  private:
    int64_t cap_;
    int64_t used_ = 0;
    std::map<int64_t, int64_t> free_;
};

enum class St { Pending, Admitted, Copying, Done, Cancelled, Failed };

struct Req {
    uint64_t ticket = 0;
    grape_walk_request_t r{};
    std::vector<int32_t> starts;   // host copy (empty when r.starts == NULL)
    int32_t* host_out = nullptr;
    int64_t num_walks = 0;
    int64_t out_bytes = 0;
    int64_t starts_bytes = 0;
    int64_t alloc_bytes = 0;
    int64_t arena_off = -1;
    int slot = -1;
    uint64_t first_chunk = 0;
    uint64_t num_chunks = 0;
    int chunk = 0;                  // walks per queue entry of this request
    St st = St::Pending;
    bool cancel = false;
    bool retired = false;
    bool inflight = false;          // counted in stats.inflight (admitted, not complete)
    grape_status_t result = GRAPE_OK;
    cudaEvent_t copied = nullptr;
    int64_t t_submit = 0, t_admit = 0, t_done = 0;
};

}  // namespace

// Queue entries staged in pinned host memory per copy (4 MiB).
constexpr int64_t kChunkStage = 1 << 18;
// Pinned staging of requests' start ids, in bytes.  An upload straight from
// pageable memory would be staged by the driver, synchronously, and while such
// uploads run the copy stream's transfers of finished rows slow to a few GB/s.
constexpr size_t kStartsStage = (size_t)32 << 20;

struct grape_server {
    const grape_graph* g = nullptr;
    grape_server_config_t cfg{};
    grape_tuning_t tuning{};
    int chunk_walks = 64;              // 0: chosen per request (chunk_for)
    int resident_warps = 1;            // warps of one resident-kernel launch

    // device state
    char* arena_base = nullptr;
    WalkConst* d_reqs = nullptr;
    unsigned long long* d_done = nullptr;   // per slot: finished walks, transitions taken
    unsigned long long* h_steps = nullptr;  // pinned: per slot, transitions of the finished request
    Chunk* d_chunks = nullptr;
    unsigned long long* d_ctl = nullptr;   // [0] head (next ticket), [1] tail, [2] heartbeat
    int* d_exit = nullptr;
    unsigned* h_flags = nullptr;           // mapped host memory
    unsigned* d_flags = nullptr;           // its device address
    WalkConst* h_wc = nullptr;             // pinned staging of request descriptors, per slot
    unsigned long long* h_tail = nullptr;  // pinned queue-tail values, per slot
    unsigned long long* h_misc = nullptr;  // pinned: [0] head at launch, [1] heartbeat,
                                           // [2] the exit word (driver thread), [3] shutdown
    uint64_t pub_tail = 0;                 // queue entries published to the device
    Chunk* h_chunks = nullptr;             // pinned staging of queue entries (driver thread)
    size_t h_chunks_cap = 0;               // min(max_chunks, kChunkStage)
    char* h_starts = nullptr;              // pinned staging of start ids (kStartsStage bytes)
    cudaStream_t compute = nullptr, copy = nullptr, ctl = nullptr;
    cudaEvent_t kernel_done = nullptr;
    bool kernel_launched = false;
    std::atomic<bool> no_heartbeat{false};   // injected host failure: the heartbeat stops
    bool exit_raised = false;          // d_exit is set for the running kernel
    int64_t idle_since = 0;            // when the server last became idle (ns)

    // host state
    std::unique_ptr<Arena> arena;
    std::mutex mu;
    std::condition_variable cv;       // signalled on every state change
    std::deque<std::shared_ptr<Req>> pending;
    std::unordered_map<uint64_t, std::shared_ptr<Req>> live;   // not yet retired
    std::vector<std::shared_ptr<Req>> by_slot;
    std::vector<int> free_slots;
    std::vector<int> active;          // slots in use, in no particular order
    std::vector<int> active_pos;      // slot -> index in active, or -1
    std::deque<uint64_t> finished;    // completed, not retired (for wait_any)
    uint64_t next_ticket = 1;
    uint64_t tail = 0;                // queue entries published
    bool stop = false;
    bool accepting = true;
    grape_server_stats_t stats{};
    std::thread driver;

    void run();
    bool admit_locked(const std::shared_ptr<Req>& q);
    grape_status_t publish(const std::vector<std::shared_ptr<Req>>& reqs);
    uint64_t oldest_live_chunk_locked() const;
    int chunk_for(int64_t num_walks) const;
    // q is taken by value: callers may pass an element of by_slot, which this resets.
    void finish_locked(std::shared_ptr<Req> q, St st, grape_status_t res);
    void release_slot_locked(Req& q);
};

uint64_t grape_server::oldest_live_chunk_locked() const {
    uint64_t oldest = tail;
    for (const int slot : active) {
        const auto& q = by_slot[(size_t)slot];
        if (q && q->first_chunk < oldest) oldest = q->first_chunk;
    }
    return oldest;
}

// Walks per queue entry for a request of num_walks walks: the configured size,
// or (configured 0) the graph's tuned size raised so that the request's
// entries give each resident lane up to 16 walks: a large request is then cut
// into about one entry per resident warp instead of thousands of small ones.
int grape_server::chunk_for(int64_t num_walks) const {
    if (chunk_walks > 0) return chunk_walks;
    const int64_t lanes = 32LL * resident_warps;
    int64_t per_lane = (num_walks + lanes - 1) / lanes;
    if (per_lane < 1) per_lane = 1;
    if (per_lane > 16) per_lane = 16;
    const int64_t c = 32 * per_lane;
    return (int)std::max<int64_t>(c, tuning.chunk_walks);
}

bool grape_server::admit_locked(const std::shared_ptr<Req>& q) {
    if (free_slots.empty()) return false;
    const int chunk = chunk_for(q->num_walks);
    const uint64_t nch = (uint64_t)((q->num_walks + chunk - 1) / chunk);
    const uint64_t used = tail - oldest_live_chunk_locked();
    if (used + nch > (uint64_t)cfg.max_chunks) return false;
    int64_t off = 0;
    if (!arena->alloc(q->alloc_bytes, &off)) return false;
    q->arena_off = off;
    q->slot = free_slots.back();
    free_slots.pop_back();
    q->first_chunk = tail;
    q->num_chunks = nch;
    q->chunk = chunk;
    tail += nch;
    by_slot[q->slot] = q;
    active_pos[(size_t)q->slot] = (int)active.size();
    active.push_back(q->slot);
    q->st = St::Admitted;
    q->t_admit = now_ns();
    q->inflight = true;
    stats.admitted++;
    stats.inflight++;
    stats.bytes_reserved = arena->used();
    return true;
}

grape_status_t grape_server::publish(const std::vector<std::shared_ptr<Req>>& reqs) {
    // Per request: its descriptor, starts and queue entries, then the tail
    // that covers them, all on one stream, so a worker that sees a tail also
    // sees what it covers, and the resident kernel starts on the first request
    // while later ones are still being copied.  Descriptors, start ids, entries
    // and tail values are staged in pinned memory allocated with the server (no
    // allocation here: freeing or allocating pinned memory may synchronise the
    // device, and the resident kernel may be waiting for exactly this work).
    // A full entry or start-id stage is waited for on the control stream before
    // reuse.
    if (reqs.empty()) return GRAPE_OK;
    const uint64_t ring = (uint64_t)cfg.max_chunks;
    uint64_t pos = reqs.front()->first_chunk;     // ring position of the first staged entry
    size_t nstaged = 0;       // entries in the stage
    size_t ncopied = 0;       // of which already enqueued for copy
    size_t starts_used = 0;   // bytes of the start-id stage in use
    cudaError_t e = cudaSuccess;
    auto copy_staged = [&]() -> cudaError_t {
        while (ncopied < nstaged) {
            const uint64_t slot = pos % ring;
            const size_t n = (size_t)std::min<uint64_t>(nstaged - ncopied, ring - slot);
            const cudaError_t ec = cudaMemcpyAsync(d_chunks + slot, h_chunks + ncopied,
                                                   sizeof(Chunk) * n, cudaMemcpyHostToDevice, ctl);
            if (ec != cudaSuccess) return ec;
            ncopied += n;
            pos += n;
        }
        return cudaSuccess;
    };
    for (const auto& q : reqs) {
        char* base = arena_base + q->arena_off;
        int32_t* d_starts = nullptr;
        if (!q->starts.empty()) {
            d_starts = reinterpret_cast<int32_t*>(base + Arena::round(q->out_bytes));
            const char* src = reinterpret_cast<const char*>(q->starts.data());
            const size_t total = (size_t)q->starts_bytes;
            for (size_t done = 0; done < total;) {
                if (starts_used == kStartsStage) {
                    // every earlier entry is already enqueued (each request's
                    // are, before the next request's starts)
                    e = cudaStreamSynchronize(ctl);
                    if (e != cudaSuccess) return cuda_status(e);
                    starts_used = 0;
                    nstaged = ncopied = 0;
                }
                const size_t n = std::min(total - done, kStartsStage - starts_used);
                std::memcpy(h_starts + starts_used, src + done, n);
                e = cudaMemcpyAsync(reinterpret_cast<char*>(d_starts) + done, h_starts + starts_used,
                                    n, cudaMemcpyHostToDevice, ctl);
                if (e != cudaSuccess) return cuda_status(e);
                starts_used += n;
                done += n;
            }
        }
        WalkConst* wc = h_wc + q->slot;
        grape_status_t st = make_walk_const(g, d_starts, q->r.num_starts, q->r.walk_len,
                                            q->r.walks_per_node, q->r.p, q->r.q, q->r.seed,
                                            reinterpret_cast<int32_t*>(base), wc);
        if (st != GRAPE_OK) return st;
        h_flags[q->slot] = 0u;
        e = cudaMemcpyAsync(d_reqs + q->slot, wc, sizeof(WalkConst), cudaMemcpyHostToDevice, ctl);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(d_done + 2 * q->slot, 0, 2 * sizeof(unsigned long long), ctl);
        if (e != cudaSuccess) return cuda_status(e);
        for (uint64_t c = 0; c < q->num_chunks; ++c) {
            if (nstaged == h_chunks_cap) {
                e = copy_staged();
                if (e == cudaSuccess) e = cudaStreamSynchronize(ctl);
                if (e != cudaSuccess) return cuda_status(e);
                nstaged = ncopied = 0;
                starts_used = 0;
            }
            Chunk& ch = h_chunks[nstaged++];
            ch.walk_lo = (long long)(c * (uint64_t)q->chunk);
            ch.count = (int)std::min<int64_t>(q->chunk, q->num_walks - ch.walk_lo);
            ch.req = q->slot;
        }
        e = copy_staged();
        if (e != cudaSuccess) return cuda_status(e);
        h_tail[q->slot] = q->first_chunk + q->num_chunks;
        e = cudaMemcpyAsync(d_ctl + 1, h_tail + q->slot, sizeof(unsigned long long),
                            cudaMemcpyHostToDevice, ctl);
        if (e != cudaSuccess) return cuda_status(e);
        pub_tail = h_tail[q->slot];
    }
    e = cudaStreamSynchronize(ctl);
    return cuda_status(e);
}

// Return q's slot to the free list and drop it from the active list.
void grape_server::release_slot_locked(Req& q) {
    if (q.slot < 0) return;
    const size_t slot = (size_t)q.slot;
    by_slot[slot].reset();
    free_slots.push_back(q.slot);
    const int i = active_pos[slot];
    if (i >= 0) {
        const int last = active.back();
        active[(size_t)i] = last;
        active_pos[(size_t)last] = i;
        active.pop_back();
        active_pos[slot] = -1;
    }
    q.slot = -1;
}

void grape_server::finish_locked(std::shared_ptr<Req> q, St st, grape_status_t res) {
    if (q->arena_off >= 0) {
        arena->release(q->arena_off, q->alloc_bytes);
        q->arena_off = -1;
    }
    release_slot_locked(*q);
    if (q->inflight) {
        q->inflight = false;
        stats.inflight--;
    }
    if (q->copied) {
        cudaEventDestroy(q->copied);
        q->copied = nullptr;
    }
    q->st = st;
    q->result = res;
    q->t_done = now_ns();
    if (st == St::Done) stats.completed++;
    if (st == St::Cancelled) stats.cancelled++;
    if (st == St::Failed) stats.rejected++;
    stats.bytes_reserved = arena->used();
    finished.push_back(q->ticket);
    cv.notify_all();
}

// The resident kernel's lifetime is decided here, for all of its warps at
// once.  Its warps never retire for lack of work on their own (a warp that did
// would leave the next request to the warps that happened to stay); after the
// server has had nothing in flight for idle_exit_us, the driver raises the
// exit flag and every warp leaves.  The kernel's own idle wait is only a
// safety bound (kernel_wait_ms of sleep without a host heartbeat, 2 s by
// default) for the case that the host stops: a warp whose wait runs out raises
// bit 2 of the graph's status word and leaves.  A kernel that ends without
// being asked to is counted in stats.kernel_timeouts; requests it left
// unfinished fail with GRAPE_ERR_TIMEOUT (an entry published as its last warp
// gave up may have no taker), and the next request relaunches it.
void grape_server::run() {
    const int64_t wait_ms = cfg.kernel_wait_ms > 0 ? cfg.kernel_wait_ms : 2000;
    const long long idle_spins = (long long)wait_ms * 1000;   // about a microsecond per unit
    // the heartbeat comes several times within one wait bound
    const int64_t beat_ns = std::min<int64_t>(100000000, wait_ms * 1000000 / 4);
    auto set_exit = [&](int v) {
        int* word = reinterpret_cast<int*>(h_misc + 2);   // pinned: the copy is a plain DMA
        *word = v;
        cudaError_t e = cudaMemcpyAsync(d_exit, word, sizeof(int), cudaMemcpyHostToDevice, ctl);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctl);
        return e;
    };
    // Launch the resident kernel unless one is running.
    // Entries are only ever published to a kernel that will take them: once
    // the exit flag is raised (with nothing in flight), the kernel is let go
    // before anything new is published.  The queue head is a ticket counter
    // that waiting warps may have run past the tail; when no kernel runs every
    // published entry has been taken, so the next kernel starts its tickets at
    // the published tail.
    auto ensure_kernel = [&]() {
        if (kernel_launched && cudaEventQuery(kernel_done) == cudaErrorNotReady) {
            if (!exit_raised) return;            // running, and staying
            cudaEventSynchronize(kernel_done);   // leaving: its warps are on their way out
        }
        cudaError_t e = exit_raised ? set_exit(0) : cudaSuccess;
        if (e == cudaSuccess) exit_raised = false;
        if (e == cudaSuccess) {
            h_misc[0] = pub_tail;
            e = cudaMemcpyAsync(d_ctl, h_misc, sizeof(unsigned long long), cudaMemcpyHostToDevice,
                                compute);
        }
        if (e == cudaSuccess)
            e = launch_queue_kernel(g, tuning, d_reqs, d_chunks, d_ctl,
                                    (unsigned long long)cfg.max_chunks, idle_spins, d_exit, d_done,
                                    d_flags, 0, compute);
        if (e == cudaSuccess) e = cudaEventRecord(kernel_done, compute);
        std::lock_guard<std::mutex> lk(mu);
        if (e == cudaSuccess) {
            kernel_launched = true;
            stats.kernel_launches++;
        } else {
            const std::vector<int> snapshot = active;   // finish_locked edits active
            for (const int slot : snapshot)
                if (by_slot[(size_t)slot])
                    finish_locked(by_slot[(size_t)slot], St::Failed, GRAPE_ERR_CUDA);
        }
    };
    int64_t last_beat = 0;
    while (true) {
        bool busy = false;
        std::vector<std::shared_ptr<Req>> admitted;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (stop) break;
            while (!pending.empty()) {
                auto q = pending.front();
                if (q->cancel) {
                    pending.pop_front();
                    finish_locked(q, St::Cancelled, GRAPE_ERR_CANCELLED);
                    continue;
                }
                if (!accepting) {
                    pending.pop_front();
                    finish_locked(q, St::Cancelled, GRAPE_ERR_CANCELLED);
                    continue;
                }
                if (admit_locked(q)) {
                    pending.pop_front();
                    admitted.push_back(q);
                    continue;
                }
                if (cfg.admit_timeout_ms > 0 &&
                    now_ns() - q->t_submit > (int64_t)cfg.admit_timeout_ms * 1000000) {
                    pending.pop_front();
                    finish_locked(q, St::Failed, GRAPE_ERR_BUSY);
                    continue;
                }
                break;
            }
        }
        if (!admitted.empty()) {
            busy = true;
            // a resident kernel first, so it starts on the first request while
            // later ones are still being published
            ensure_kernel();
            grape_status_t st = publish(admitted);
            if (st != GRAPE_OK) {
                std::lock_guard<std::mutex> lk(mu);
                for (auto& q : admitted) finish_locked(q, St::Failed, st);
            }
        }
        // Keep a resident kernel running while admitted work remains.
        bool inflight;
        {
            std::lock_guard<std::mutex> lk(mu);
            inflight = stats.inflight > 0;
        }
        const bool running = kernel_launched && cudaEventQuery(kernel_done) == cudaErrorNotReady;
        // Heartbeat for the kernel's waiting warps: their bounded wait only runs
        // out if the host stops beating.
        if (running && !no_heartbeat.load() && now_ns() - last_beat > beat_ns) {
            last_beat = now_ns();
            h_misc[1] += 1;
            cudaMemcpyAsync(d_ctl + 2, h_misc + 1, sizeof(unsigned long long),
                            cudaMemcpyHostToDevice, ctl);
        }
        if (!inflight) {
            if (idle_since == 0) idle_since = now_ns();
            if (running && !exit_raised &&
                now_ns() - idle_since > cfg.idle_exit_us * 1000) {
                if (set_exit(1) == cudaSuccess) exit_raised = true;
            }
        } else {
            idle_since = 0;
        }
        if (inflight && !running) ensure_kernel();
        // Completions: flag -> copy out -> done.
        {
            std::lock_guard<std::mutex> lk(mu);
            const std::vector<int> snapshot = active;   // finish_locked edits active
            for (const int slot : snapshot) {
                const std::shared_ptr<Req> q = by_slot[(size_t)slot];
                if (!q) continue;
                if (q->st == St::Admitted && ((volatile unsigned*)h_flags)[q->slot] != 0u) {
                    busy = true;
                    if (q->cancel) {
                        finish_locked(q, St::Cancelled, GRAPE_ERR_CANCELLED);
                        continue;
                    }
                    // the request's transition count, and its rows unless they
                    // stay in the arena until wait() hands them over
                    cudaError_t e = cudaEventCreateWithFlags(&q->copied, cudaEventDisableTiming);
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(h_steps + q->slot, d_done + 2 * q->slot + 1,
                                            sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                            copy);
                    if (e == cudaSuccess && q->host_out)
                        e = cudaMemcpyAsync(q->host_out, arena_base + q->arena_off,
                                            (size_t)q->out_bytes, cudaMemcpyDeviceToHost, copy);
                    if (e == cudaSuccess) e = cudaEventRecord(q->copied, copy);
                    if (e != cudaSuccess) {
                        finish_locked(q, St::Failed, cuda_status(e));
                        continue;
                    }
                    q->st = St::Copying;
                } else if (q->st == St::Copying) {
                    const cudaError_t e = cudaEventQuery(q->copied);
                    if (e == cudaSuccess) {
                        busy = true;
                        if (!q->cancel) stats.steps += (int64_t)h_steps[q->slot];
                        if (q->cancel) {
                            finish_locked(q, St::Cancelled, GRAPE_ERR_CANCELLED);
                        } else if (q->host_out) {
                            finish_locked(q, St::Done, GRAPE_OK);
                        } else {
                            // rows stay in the arena until wait() hands them over
                            cudaEventDestroy(q->copied);
                            q->copied = nullptr;
                            q->st = St::Done;
                            q->t_done = now_ns();
                            q->inflight = false;
                            stats.inflight--;
                            stats.completed++;
                            finished.push_back(q->ticket);
                            cv.notify_all();
                        }
                    } else if (e != cudaErrorNotReady) {
                        finish_locked(q, St::Failed, cuda_status(e));
                    }
                }
            }
        }
        // A kernel that ended without the exit flag: its waits ran out.  Its
        // completion flags are final now; what it left unfinished fails.
        if (kernel_launched && !exit_raised &&
            cudaEventQuery(kernel_done) != cudaErrorNotReady) {
            busy = true;
            std::lock_guard<std::mutex> lk(mu);
            kernel_launched = false;
            stats.kernel_timeouts++;
            const std::vector<int> snapshot = active;   // finish_locked edits active
            for (const int slot : snapshot) {
                const std::shared_ptr<Req> q = by_slot[(size_t)slot];
                if (q && q->st == St::Admitted && ((volatile unsigned*)h_flags)[q->slot] == 0u)
                    finish_locked(q, St::Failed, GRAPE_ERR_TIMEOUT);
            }
        }
        if (!busy) {
            std::unique_lock<std::mutex> lk(mu);
            if (stats.inflight > 0)
                cv.wait_for(lk, std::chrono::microseconds(20));
            else if (!stop)
                cv.wait_for(lk, std::chrono::milliseconds(2),
                            [&] { return stop || !pending.empty(); });
        }
    }
}

extern "C" {

grape_status_t grape_walk_server_create(const grape_graph_t* g, const grape_server_config_t* cfg,
                                        grape_server_t** out) {
    if (!out) return GRAPE_ERR_INVALID_ARG;
    *out = nullptr;
    if (!g || !cfg || cfg->output_cap_bytes < 4096 || cfg->max_inflight < 1 ||
        cfg->max_inflight > 65536 || cfg->chunk_walks < 0 || cfg->max_chunks < 1 ||
        cfg->idle_exit_us < 1 || cfg->admit_timeout_ms < 0 || cfg->kernel_wait_ms < 0)
        return GRAPE_ERR_INVALID_ARG;
    grape_server* s = new (std::nothrow) grape_server();
    if (!s) return GRAPE_ERR_NOMEM;
    s->g = g;
    s->cfg = *cfg;
    grape_graph_get_tuning(g, &s->tuning);
    s->chunk_walks = cfg->chunk_walks;
    {
        const LaunchShape ls = queue_launch_shape(g, s->tuning, g->weighted);
        s->resident_warps = std::max(1, ls.blocks * (ls.threads / 32));
    }
    s->arena.reset(new Arena(cfg->output_cap_bytes));
    const int slots = cfg->max_inflight;
    s->by_slot.resize((size_t)slots);
    s->active_pos.assign((size_t)slots, -1);
    s->active.reserve((size_t)slots);
    for (int i = slots - 1; i >= 0; --i) s->free_slots.push_back(i);
    cudaError_t e = cudaMalloc(&s->arena_base, (size_t)cfg->output_cap_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_reqs, sizeof(WalkConst) * (size_t)slots);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_done, 2 * sizeof(unsigned long long) * (size_t)slots);
    if (e == cudaSuccess)
        e = cudaHostAlloc(&s->h_steps, sizeof(unsigned long long) * (size_t)slots,
                          cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_chunks, sizeof(Chunk) * (size_t)cfg->max_chunks);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_ctl, sizeof(unsigned long long) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_exit, sizeof(int));
    if (e == cudaSuccess)
        e = cudaHostAlloc(&s->h_flags, sizeof(unsigned) * (size_t)slots, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&s->d_flags, s->h_flags, 0);
    if (e == cudaSuccess)
        e = cudaHostAlloc(&s->h_wc, sizeof(WalkConst) * (size_t)slots, cudaHostAllocDefault);
    if (e == cudaSuccess)
        e = cudaHostAlloc(&s->h_tail, sizeof(unsigned long long) * (size_t)slots,
                          cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(&s->h_misc, sizeof(unsigned long long) * 4, 0);
    if (e == cudaSuccess) std::memset(s->h_misc, 0, sizeof(unsigned long long) * 4);
    if (e == cudaSuccess) e = cudaHostAlloc(&s->h_starts, kStartsStage, cudaHostAllocDefault);
    if (e == cudaSuccess) {
        s->h_chunks_cap = (size_t)std::min<int64_t>(cfg->max_chunks, kChunkStage);
        e = cudaHostAlloc(&s->h_chunks, sizeof(Chunk) * s->h_chunks_cap, cudaHostAllocDefault);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->ctl, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->kernel_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemset(s->d_ctl, 0, sizeof(unsigned long long) * 4);
    if (e == cudaSuccess) e = cudaMemset(s->d_exit, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        grape_walk_server_destroy(s);
        return cuda_status(e);
    }
    std::memset(s->h_flags, 0, sizeof(unsigned) * (size_t)slots);
    s->driver = std::thread([s] { s->run(); });
    *out = s;
    return GRAPE_OK;
}

grape_status_t grape_walk_server_submit(grape_server_t* s, const grape_walk_request_t* r,
                                        uint64_t* ticket) {
    if (!s || !r || !ticket) return GRAPE_ERR_INVALID_ARG;
    WalkConst probe;
    grape_status_t st = make_walk_const(s->g, r->starts, r->num_starts, r->walk_len,
                                        r->walks_per_node, r->p, r->q, r->seed,
                                        reinterpret_cast<int32_t*>(alignof(int4)), &probe);
    if (st != GRAPE_OK) return st;
    auto q = std::make_shared<Req>();
    q->r = *r;
    q->host_out = r->out;
    q->num_walks = probe.num_walks;
    q->out_bytes = (int64_t)sizeof(int32_t) * probe.num_walks * r->walk_len;
    q->starts_bytes = r->starts ? (int64_t)sizeof(int32_t) * r->num_starts : 0;
    q->alloc_bytes = Arena::round(q->out_bytes) + Arena::round(q->starts_bytes);
    if (q->alloc_bytes > s->cfg.output_cap_bytes) return GRAPE_ERR_NOMEM;
    if (r->starts) q->starts.assign(r->starts, r->starts + r->num_starts);
    q->r.starts = nullptr;
    q->t_submit = now_ns();
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->accepting) return GRAPE_ERR_CANCELLED;
    if ((int64_t)s->pending.size() >= 4LL * s->cfg.max_inflight + 1024) return GRAPE_ERR_BUSY;
    q->ticket = s->next_ticket++;
    s->pending.push_back(q);
    s->live[q->ticket] = q;
    s->stats.submitted++;
    *ticket = q->ticket;
    s->cv.notify_all();
    return GRAPE_OK;
}

static bool terminal(St st) {
    return st == St::Done || st == St::Cancelled || st == St::Failed;
}

static grape_status_t retire_locked(grape_server* s, const std::shared_ptr<Req>& q,
                                    int32_t* host_out, std::unique_lock<std::mutex>& lk) {
    grape_status_t res = q->result;
    if (q->st == St::Done && q->arena_off >= 0) {
        // rows held in the arena: hand them over now
        if (!host_out) {
            res = GRAPE_ERR_INVALID_ARG;
        } else {
            const void* src = s->arena_base + q->arena_off;
            lk.unlock();
            cudaError_t e = cudaMemcpy(host_out, src, (size_t)q->out_bytes, cudaMemcpyDeviceToHost);
            lk.lock();
            res = cuda_status(e);
        }
        if (q->arena_off >= 0) {
            s->arena->release(q->arena_off, q->alloc_bytes);
            q->arena_off = -1;
        }
        s->release_slot_locked(*q);
        s->stats.bytes_reserved = s->arena->used();
        s->cv.notify_all();
    }
    q->retired = true;
    s->live.erase(q->ticket);
    return res;
}

grape_status_t grape_walk_server_wait(grape_server_t* s, uint64_t ticket, int64_t timeout_ms,
                                      int32_t* host_out) {
    if (!s) return GRAPE_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->live.find(ticket);
    if (it == s->live.end()) return GRAPE_ERR_NOT_FOUND;
    auto q = it->second;
    auto ready = [&] { return terminal(q->st); };
    if (timeout_ms < 0) s->cv.wait(lk, ready);
    else if (!s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return GRAPE_ERR_TIMEOUT;
    return retire_locked(s, q, host_out, lk);
}

grape_status_t grape_walk_server_wait_any(grape_server_t* s, int64_t timeout_ms,
                                          uint64_t* ticket, int64_t* latency_ns,
                                          int32_t* host_out) {
    if (!s || !ticket) return GRAPE_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] {
        while (!s->finished.empty() && !s->live.count(s->finished.front())) s->finished.pop_front();
        return !s->finished.empty();
    };
    if (timeout_ms < 0) s->cv.wait(lk, ready);
    else if (!s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return GRAPE_ERR_TIMEOUT;
    const uint64_t t = s->finished.front();
    s->finished.pop_front();
    auto q = s->live[t];
    *ticket = t;
    if (latency_ns) *latency_ns = q->t_done - q->t_submit;
    return retire_locked(s, q, host_out, lk);
}

grape_status_t grape_walk_server_cancel(grape_server_t* s, uint64_t ticket) {
    if (!s) return GRAPE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->live.find(ticket);
    if (it == s->live.end()) return GRAPE_ERR_NOT_FOUND;
    it->second->cancel = true;
    s->cv.notify_all();
    return GRAPE_OK;
}

grape_status_t grape_walk_server_inject_fault(grape_server_t* s, uint32_t faults) {
    if (!s || (faults & ~GRAPE_FAULT_NO_HEARTBEAT) != 0u) return GRAPE_ERR_INVALID_ARG;
    s->no_heartbeat.store((faults & GRAPE_FAULT_NO_HEARTBEAT) != 0u);
    return GRAPE_OK;
}

grape_status_t grape_walk_server_stats(grape_server_t* s, grape_server_stats_t* out) {
    if (!s || !out) return GRAPE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    return GRAPE_OK;
}

void grape_walk_server_destroy(grape_server_t* s) {
    if (!s) return;
    if (s->driver.joinable()) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->accepting = false;
            for (auto& q : s->pending) q->cancel = true;
            s->cv.notify_all();
            // admitted work gets a bounded time to finish
            s->cv.wait_for(lk, std::chrono::seconds(60), [&] { return s->stats.inflight == 0; });
            s->stop = true;
            s->cv.notify_all();
        }
        int* one = reinterpret_cast<int*>(s->h_misc + 3);
        *one = 1;
        cudaMemcpyAsync(s->d_exit, one, sizeof(int), cudaMemcpyHostToDevice, s->ctl);
        cudaStreamSynchronize(s->ctl);
        s->driver.join();
    }
    if (s->compute) cudaStreamSynchronize(s->compute);
    if (s->copy) cudaStreamSynchronize(s->copy);
    for (auto& kv : s->live)
        if (kv.second->copied) cudaEventDestroy(kv.second->copied);
    if (s->kernel_done) cudaEventDestroy(s->kernel_done);
    if (s->compute) cudaStreamDestroy(s->compute);
    if (s->copy) cudaStreamDestroy(s->copy);
    if (s->ctl) cudaStreamDestroy(s->ctl);
    if (s->h_flags) cudaFreeHost(s->h_flags);
    if (s->h_steps) cudaFreeHost(s->h_steps);
    if (s->h_wc) cudaFreeHost(s->h_wc);
    if (s->h_tail) cudaFreeHost(s->h_tail);
    if (s->h_misc) cudaFreeHost(s->h_misc);
    if (s->h_chunks) cudaFreeHost(s->h_chunks);
    if (s->h_starts) cudaFreeHost(s->h_starts);
    cudaFree(s->arena_base);
    cudaFree(s->d_reqs);
    cudaFree(s->d_done);
    cudaFree(s->d_chunks);
    cudaFree(s->d_ctl);
    cudaFree(s->d_exit);
    delete s;
}

}  // extern "C"
