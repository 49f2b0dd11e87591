// vc_server.cu - serving with continuous batching (include/vc_server.h).
//
// Requests are served by size class.  Each class is a "lane": one persistent traversal launch
// (traverse_kernel with Params::serving = 1) that works on every admitted request of the class at
// once: idle workers claim new requests from the lane's submission ring, run their greedy bound and
// then search them through the lane's worklist, whose entries carry the request's slot.
//   lane 0  graphs of at most 128 vertices: one-warp bit-row workers (node in registers)
//   lane 1  larger graphs: CSR-walk workers sized for the server's max_n
// (Lane 0 only when asked for, bit_rows > 0; lane 1 alone by default; lane 0 alone when
// max_n <= 128 and bit rows are asked for.)  The two
// launches run side by side on their own streams, lane 1 with three quarters of every SM's thread
// slots and lane 0 with the rest, and never wait on one another.  Stacks and worklist of a lane are sized for its largest graph.
//
// A host thread owned by the server, for every lane:
//   - admits queued requests while their bytes fit: each request reserves a slot and a range of
//     its lane's graph arena (CSR, cover mask and root entry);
//   - uploads the request on the lane's copy stream (CSR, slot record, ring entry, then the ring
//     tail, all ordered on that stream) while the launch keeps running;
//   - harvests completion records that the device writes into host-mapped memory;
//   - relaunches the traversal when requests arrive after an idle launch closed.
// Addresses are never reused within one launch (no L1 can hold stale graph data): slots and arena
// ranges are handed out in order within an "epoch"; when an epoch is used up, admission to that
// lane pauses until its requests in flight finish, its launch closes and the epoch restarts.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#ifdef __linux__
#include <sys/prctl.h>
#endif

#include "vc_internal.h"
#include "vc_tuning.h"
#include "vc_launch.h"
#include "../../include/vc_server.h"

namespace vc {
namespace {

constexpr int32_t kSlotStride = 128;  // bytes per problem record (one cache line, never shared)
constexpr size_t kAlign = 128;
constexpr int32_t kSmallN = 128;      // largest graph of the bit-row lane
constexpr int kSmallRowWords = 4;     // its bit rows: 4 words per vertex (n <= 128)
constexpr int kMaxLanes = 2;
constexpr int kThreadSlotsPerSm = 1024;  // threads an SM holds at the traversal's 64 registers

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}
size_t up(size_t b) { return (b + kAlign - 1) & ~(kAlign - 1); }

struct Request {
    uint64_t id = 0;
    int32_t kind = 0, k = 0, n = 0;
    int lane = 0;
    std::vector<int32_t> off, adj;
    int32_t slot = -1;
    int32_t tag = 0;
    int32_t state = 0;  // 0 queued, 1 in flight, 2 done
    int32_t answer = -1, status = VC_OK, greedy = -1;
    int64_t t_submit = 0, t_admit = 0, t_done = 0;
    size_t bytes = 0;
};

// One size class: its variant, device memory, persistent launch and epoch.
struct Lane {
    // variant
    int32_t max_n = 0;  // largest graph of the class
    int nw = 0;         // bit-row words per vertex (0: CSR walks)
    int wt = 0, width = 16, smem = 0, workers = 0, eb = 0, depth = 0, cap = 0, threshold = 0;
    int32_t csr_words = 0;
    int32_t slots = 0;  // problem slots per epoch (power of two, also the ring capacity)
    size_t arena_bytes = 0;
    // device memory (one allocation carved into these regions)
    void *mem = nullptr;
    Control *ctrl = nullptr;
    uint8_t *problems = nullptr;
    uint8_t *arena = nullptr;
    uint8_t *stacks = nullptr, *wl_slots = nullptr;
    uint32_t *wl_seq = nullptr, *sub_ring = nullptr, *sub_tail = nullptr, *rows = nullptr;
    unsigned long long *claim_state = nullptr, *sm_nodes = nullptr;
    int32_t *close_now = nullptr;
    // host memory
    int32_t *completion_h = nullptr, *completion_d = nullptr;  // mapped, 4 ints per slot
    uint8_t *stage_h = nullptr;  // pinned: slot records, ring entries, tail values, flags
    cudaStream_t kstream = nullptr, cstream = nullptr;
    cudaEvent_t kdone = nullptr;
    bool running = false;
    // epoch
    int32_t next_slot = 0;
    size_t arena_used = 0;
    uint32_t published = 0;
    bool draining = false;
    bool close_sent = false;
    // requests
    std::deque<Request *> pending;
    std::vector<Request *> in_flight;
    // counters
    unsigned long long nodes = 0;
    int64_t launches = 0, epochs = 0;
    int32_t last_status = VC_OK;
};

}  // namespace
}  // namespace vc

using namespace vc;

struct vc_server {
    vc_config cfg;
    int device = 0;
    int32_t max_n = 0;
    size_t budget = 0;
    Lane lane[kMaxLanes];
    int nlanes = 0;
    // requests
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::unordered_map<uint64_t, Request *> all;
    uint64_t next_id = 1;
    int64_t outstanding = 0;
    bool stop = false;
    std::thread th;
    int64_t completed = 0;
};

namespace vc {
namespace {

Problem *stage_problem(Lane &L, int32_t slot) {
    return reinterpret_cast<Problem *>(L.stage_h + (size_t)slot * kSlotStride);
}
uint32_t *stage_ring(Lane &L) { return reinterpret_cast<uint32_t *>(L.stage_h + (size_t)L.slots * kSlotStride); }
uint32_t *stage_tail(Lane &L) { return stage_ring(L) + L.slots; }
int32_t *stage_flags(Lane &L) { return reinterpret_cast<int32_t *>(stage_tail(L) + L.slots + 1); }
// Pinned zeros (the size of the control block) that the lane copies over the words it resets.
// Resets are copies rather than memsets: a memset may run a kernel the driver loads on first use,
// and loading code can wait for every running launch, such as the other lane's persistent one.
const void *stage_zeros(Lane &L) { return L.stage_h + (size_t)L.slots * kSlotStride + sizeof(uint32_t) * (2 * (size_t)L.slots + 1) + 64; }

Params serve_params(const vc_server *s, const Lane &L) {
    Params P;
    std::memset(&P, 0, sizeof(P));
    P.offsets = reinterpret_cast<const int32_t *>(L.arena);
    P.neighbors = reinterpret_cast<const int32_t *>(L.arena);
    P.problems = reinterpret_cast<Problem *>(L.problems);
    P.num_problems = L.slots;
    P.n_max = L.max_n;
    P.entry_bytes = L.eb;
    P.stack_depth = L.depth;
    P.ctrl = L.ctrl;
    P.cover = reinterpret_cast<int32_t *>(L.arena);
    P.stacks = L.stacks;
    P.wl_slots = L.wl_slots;
    P.wl_seq = L.wl_seq;
    P.wl_capacity = L.cap;
    P.wl_threshold = L.threshold;
    P.csr_words = L.csr_words;
    P.rows = L.rows;  // bit-row lane: rows at cover_base * nw words, written by each request's greedy pass
    P.roots = L.arena;  // each request's root node, kept by its greedy pass, at its root_base
    P.idle_timeout_ns = s->cfg.idle_timeout_ns > 0 ? s->cfg.idle_timeout_ns : 20000000000ll;
    P.cancel = s->cfg.cancel;
    P.sm_nodes = L.sm_nodes;
    P.serving = 1;
    P.sub_mask = (uint32_t)L.slots - 1u;
    P.sub_ring = L.sub_ring;
    P.sub_tail = L.sub_tail;
    P.claim_state = L.claim_state;
    P.close_now = L.close_now;
    P.completion = L.completion_d;
    P.linger_ns = 2000000;  // an empty launch closes after 2 ms idle
    return P;
}

const Launchers &lane_launchers(const Lane &L) { return launchers(L.width, false, L.nw); }

// Launches the lane's persistent traversal (the server lock is held).
int launch(vc_server *s, Lane &L) {
    const Launchers &LL = lane_launchers(L);
    if (cudaMemcpyAsync(L.ctrl, stage_zeros(L), sizeof(Control), cudaMemcpyHostToDevice, L.kstream) != cudaSuccess)
        return VC_ECUDA;
    if (cudaMemcpyAsync(L.close_now, stage_zeros(L), sizeof(int32_t), cudaMemcpyHostToDevice, L.kstream) != cudaSuccess)
        return VC_ECUDA;
    Params P = serve_params(s, L);
    if (int rc = launch_init_worklist(L.wl_seq, L.cap, L.ctrl, L.kstream, L.claim_state)) return rc;
    if (int rc = LL.traverse(L.wt, L.workers, L.smem, L.kstream, P)) return rc;
    if (cudaEventRecord(L.kdone, L.kstream) != cudaSuccess) return VC_ECUDA;
    L.running = true;
    L.close_sent = false;
    L.launches++;
    return VC_OK;
}

// Reads the statistics of a launch that has ended.
void collect(Lane &L) {
    Control c;
    if (cudaMemcpy(&c, L.ctrl, sizeof(Control), cudaMemcpyDeviceToHost) == cudaSuccess) {
        L.nodes += c.nodes;
        if (c.status != VC_OK) L.last_status = c.status;
    } else {
        cudaGetLastError();
    }
}

// Admits the lane's queued requests that fit its current epoch and publishes them (the server
// lock is held).
int admit(Lane &L) {
    uint32_t first = L.published;
    while (!L.pending.empty() && !L.draining) {
        Request *r = L.pending.front();
        if (L.next_slot >= L.slots || L.arena_used + r->bytes > L.arena_bytes) {
            L.draining = true;  // epoch used up: finish what is in flight, then restart
            break;
        }
        L.pending.pop_front();
        const int32_t slot = L.next_slot++;
        const size_t base = L.arena_used;
        L.arena_used += r->bytes;
        const size_t off_bytes = up(sizeof(int32_t) * ((size_t)r->n + 1));
        const size_t adj_bytes = up(sizeof(int32_t) * std::max<size_t>(r->adj.size(), 1));
        const size_t cover_bytes = up(sizeof(int32_t) * std::max<size_t>(r->n, 1));
        Problem *p = stage_problem(L, slot);
        std::memset(p, 0, sizeof(Problem));
        p->off_base = (int64_t)(base / 4);
        p->adj_base = (int64_t)((base + off_bytes) / 4);
        p->cover_base = (int64_t)((base + off_bytes + adj_bytes) / 4);
        p->root_base = (int64_t)(base + off_bytes + adj_bytes + cover_bytes);
        p->n = r->n;
        p->kind = r->kind;
        p->k = r->k;
        p->best = INT_MAX;
        p->cover_size = INT_MAX;
        r->slot = slot;
        r->tag = (int32_t)((r->id & 0x3fffffff) | 0x40000000);  // nonzero, and unlike any older tag
        p->tag = r->tag;
        L.completion_h[4 * slot] = 0;
        if (cudaMemcpyAsync(L.arena + base, r->off.data(), sizeof(int32_t) * r->off.size(), cudaMemcpyHostToDevice,
                            L.cstream) != cudaSuccess ||
            (!r->adj.empty() && cudaMemcpyAsync(L.arena + base + off_bytes, r->adj.data(),
                                                sizeof(int32_t) * r->adj.size(), cudaMemcpyHostToDevice,
                                                L.cstream) != cudaSuccess) ||
            cudaMemcpyAsync(L.problems + (size_t)slot * kSlotStride, p, sizeof(Problem), cudaMemcpyHostToDevice,
                            L.cstream) != cudaSuccess)
            return VC_ECUDA;
        uint32_t *ring = stage_ring(L);
        ring[L.published] = (uint32_t)slot;
        if (cudaMemcpyAsync(L.sub_ring + (L.published & (uint32_t)(L.slots - 1)), &ring[L.published],
                            sizeof(uint32_t), cudaMemcpyHostToDevice, L.cstream) != cudaSuccess)
            return VC_ECUDA;
        L.published++;
        r->state = 1;
        r->t_admit = now_ns();
        L.in_flight.push_back(r);
    }
    if (L.published != first) {
        // The tail goes last on the copy stream: every entry it covers is in place when it lands.
        uint32_t *tail = stage_tail(L);
        tail[L.published] = L.published;
        if (cudaMemcpyAsync(L.sub_tail, &tail[L.published], sizeof(uint32_t), cudaMemcpyHostToDevice, L.cstream) !=
            cudaSuccess)
            return VC_ECUDA;
    }
    return VC_OK;
}

// Harvests the lane's completion records (the server lock is held).  Returns how many finished.
int harvest(vc_server *s, Lane &L) {
    int done = 0;
    volatile int32_t *rec = L.completion_h;
    for (size_t i = 0; i < L.in_flight.size();) {
        Request *r = L.in_flight[i];
        if (rec[4 * r->slot] == r->tag) {
            std::atomic_thread_fence(std::memory_order_acquire);
            r->answer = rec[4 * r->slot + 1];
            r->status = rec[4 * r->slot + 2];
            r->greedy = rec[4 * r->slot + 3];
            r->t_done = now_ns();
            r->state = 2;
            r->off.clear();
            r->off.shrink_to_fit();
            r->adj.clear();
            r->adj.shrink_to_fit();
            L.in_flight[i] = L.in_flight.back();
            L.in_flight.pop_back();
            s->outstanding--;
            s->completed++;
            done++;
        } else {
            ++i;
        }
    }
    return done;
}

// Starts a new epoch of a lane (no launch running, nothing in flight; the server lock is held).
int reset_epoch(Lane &L) {
    L.next_slot = 0;
    L.arena_used = 0;
    L.published = 0;
    L.draining = false;
    L.epochs++;
    if (cudaMemcpyAsync(L.claim_state, stage_zeros(L), sizeof(unsigned long long), cudaMemcpyHostToDevice,
                        L.cstream) != cudaSuccess ||
        cudaMemcpyAsync(L.sub_tail, stage_zeros(L), sizeof(uint32_t), cudaMemcpyHostToDevice, L.cstream) != cudaSuccess ||
        cudaStreamSynchronize(L.cstream) != cudaSuccess)
        return VC_ECUDA;
    return VC_OK;
}

// Ends every open request of a lane with `code` (the server lock is held).
void fail_lane(vc_server *s, Lane &L, int32_t code) {
    for (Request *r : L.in_flight) {
        r->status = code;
        r->state = 2;
        r->t_done = now_ns();
        s->outstanding--;
    }
    L.in_flight.clear();
    for (Request *r : L.pending) {
        r->status = code;
        r->state = 2;
        r->t_done = now_ns();
        s->outstanding--;
    }
    L.pending.clear();
}

// The CSR rules of vc.h, checked on the host (the running launch must never see a bad graph).
bool csr_ok(const vc_graph *g) {
    const int32_t n = g->n;
    if (n == 0) return true;
    const int32_t *off = g->offsets, *adj = g->neighbors;
    if (off[0] != 0 || off[n] < 0 || (off[n] & 1) || (off[n] > 0 && !adj)) return false;
    // Every offset is checked before any list is read: the symmetry test below searches the
    // lists of later vertices.
    for (int32_t v = 0; v < n; ++v)
        if (off[v + 1] < off[v] || off[v + 1] > off[n]) return false;
    for (int32_t v = 0; v < n; ++v) {
        for (int32_t j = off[v]; j < off[v + 1]; ++j) {
            const int32_t x = adj[j];
            if (x < 0 || x >= n || x == v || (j > off[v] && adj[j - 1] >= x)) return false;
            if (!std::binary_search(adj + off[x], adj + off[x + 1], v)) return false;
        }
    }
    return true;
}

// One pass of the host thread over a lane (the server lock is held); returns whether anything
// moved.
bool step_lane(vc_server *s, Lane &L) {
    bool progress = false;
    if (harvest(s, L)) {
        progress = true;
        s->cv_done.notify_all();
    }
    if (L.running && cudaEventQuery(L.kdone) == cudaSuccess) {
        L.running = false;
        collect(L);
        progress = true;
        if (L.last_status != VC_OK) {  // the launch failed: report it on everything open
            harvest(s, L);
            fail_lane(s, L, L.last_status);
            L.last_status = VC_OK;
            s->cv_done.notify_all();
            if (L.draining || L.published) reset_epoch(L);
        }
    } else if (L.running) {
        cudaGetLastError();
    }
    if (!L.running && L.draining && L.in_flight.empty()) {
        if (reset_epoch(L) != VC_OK) {
            fail_lane(s, L, VC_ECUDA);
            s->cv_done.notify_all();
        }
        progress = true;
    }
    const uint32_t before = L.published;
    if (admit(L) != VC_OK) {
        fail_lane(s, L, VC_ECUDA);
        s->cv_done.notify_all();
    }
    if (L.published != before) progress = true;
    if (!L.running && !L.in_flight.empty()) {
        // Requests are published but no launch is running: start one once the uploads landed.
        if (cudaStreamSynchronize(L.cstream) != cudaSuccess || launch(s, L) != VC_OK) {
            cudaGetLastError();
            fail_lane(s, L, VC_ECUDA);
            s->cv_done.notify_all();
        }
        progress = true;
    }
    if (L.running && !L.close_sent && L.in_flight.empty() && (L.draining || s->stop)) {
        int32_t *flag = stage_flags(L);
        flag[0] = 1;
        cudaMemcpyAsync(L.close_now, flag, sizeof(int32_t), cudaMemcpyHostToDevice, L.cstream);
        L.close_sent = true;
    }
    return progress;
}

// The host thread's waits: 5 us while requests are in flight (their completion records are polled),
// 20 us while a launch runs without any, 2 ms when idle.  Its timer slack is set to 1 ns: Linux
// otherwise rounds each timed wait up by 50 us, which delayed every completion's harvest.  On the
// served stream (2000 req/s) both together cut the median latency from 0.333 to 0.305 ms and that of
// graphs with at most 128 vertices from 0.247 to 0.205 ms; busy polling without waits gained 3 us
// more and lost burst capacity to the server lock.
void loop(vc_server *s) {
    cudaSetDevice(s->device);
#ifdef __linux__
    prctl(PR_SET_TIMERSLACK, 1UL, 0UL, 0UL, 0UL);
#endif
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        bool progress = false, busy = false, idle = true, flying = false;
        for (int i = 0; i < s->nlanes; ++i) {
            Lane &L = s->lane[i];
            progress |= step_lane(s, L);
            busy |= L.running || !L.pending.empty();
            flying |= !L.in_flight.empty();
            idle &= L.pending.empty() && L.in_flight.empty() && !L.running;
        }
        if (s->stop && idle) break;
        if (!progress) s->cv_work.wait_for(lk, std::chrono::microseconds(flying ? 5 : busy ? 20 : 2000));
    }
}

// Sizes a lane's variant and memory for graphs of up to L.max_n vertices within `budget` bytes,
// with `share` of the worker slots the kernel's occupancy allows on each SM (the lanes' launches
// run side by side), then allocates it.
int make_lane(const vc_server *s, Lane &L, const cudaDeviceProp &prop, size_t budget, float share) {
    const vc_config &cfg = s->cfg;
    const LaunchDefaults tuned = tuned_defaults(L.max_n);
    if (L.nw > 0) {  // bit rows: one-warp workers, the tuned 32-bit entries, no CSR staging
        L.wt = 32;
        L.width = 32;
        L.csr_words = 0;
    } else {
        L.width = cfg.width ? cfg.width : tuned.width;
        if ((L.width != 16 && L.width != 32) || (L.width == 16 && L.max_n > 32768)) return VC_EINVAL;
        L.wt = cfg.worker_threads ? cfg.worker_threads : tuned.worker_threads;
        L.csr_words = default_csr_words(L.max_n, cfg.stage_csr);
    }
    L.smem = smem_bytes_for(L.max_n, L.width / 8, L.csr_words, L.nw);
    if (L.smem > (int)prop.sharedMemPerBlockOptin) return VC_EINVAL;
    // Loads and configures the lane's kernel now: a kernel loaded on its first launch may wait for
    // every running launch to finish, and the other lane's persistent launch could be one.
    int per_sm = 0;
    if (lane_launchers(L).serve_prepare(L.wt, L.smem, &per_sm) != VC_OK || per_sm <= 0) return VC_EINVAL;
    per_sm = std::max(1, (int)((float)per_sm * share));
    L.eb = entry_bytes_for(L.max_n, L.width / 8);
    L.depth = L.max_n + 3;  // MVC depth <= n + 1, PVC depth <= min(k, n) + 2
    L.slots = 16384;
    // Worklist: the batch default of the size class, limited to an eighth of the lane's budget.
    L.cap = default_worklist_capacity(L.eb, tuned.capacity);
    while (L.cap > 1024 && (size_t)L.cap * (size_t)L.eb > budget / 8) L.cap >>= 1;
    // Budget: half for the stacks (as many workers as fit), a quarter for the graph arena and, in
    // the bit-row lane, the rows (nw words for every cover word of the arena).
    const size_t per_worker = (size_t)L.depth * (size_t)L.eb;
    int64_t w = (L.nw == 0 && cfg.num_workers > 0) ? cfg.num_workers : (int64_t)prop.multiProcessorCount * per_sm;
    w = std::min<int64_t>(w, (int64_t)(budget / 2 / per_worker));
    if (w < 1) return VC_ENOMEM;
    L.workers = (int)w;
    const float frac = (cfg.donate_threshold > 0.f && L.nw == 0) ? cfg.donate_threshold : tuned.threshold;
    L.threshold = std::max(1, (int)(frac * L.cap));
    if (cfg.worklist_capacity > 0 && L.nw == 0) {
        int c = 1;
        while (c < cfg.worklist_capacity) c <<= 1;
        L.cap = c;
        L.threshold = std::max(1, (int)(frac * c));
    }
    L.arena_bytes = std::max<size_t>(budget / 4 / (size_t)(1 + L.nw), 64 << 10) & ~(size_t)(kAlign - 1);
    // One device allocation for everything.
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t at = off;
        off += up(b);
        return at;
    };
    const size_t o_ctrl = take(sizeof(Control));
    const size_t o_prob = take((size_t)L.slots * kSlotStride);
    const size_t o_ring = take(sizeof(uint32_t) * (size_t)L.slots);
    const size_t o_tail = take(sizeof(uint32_t));
    const size_t o_claim = take(sizeof(unsigned long long));
    const size_t o_close = take(sizeof(int32_t));
    const size_t o_smn = take(sizeof(unsigned long long) * kSmSlots);
    const size_t o_seq = take(sizeof(uint32_t) * (size_t)L.cap);
    const size_t o_wl = take((size_t)L.cap * (size_t)L.eb);
    const size_t o_arena = take(L.arena_bytes);
    const size_t o_rows = take(L.arena_bytes * (size_t)L.nw);
    const size_t o_stacks = take((size_t)L.workers * per_worker);
    if (cudaMalloc(&L.mem, off) != cudaSuccess) {
        cudaGetLastError();
        L.mem = nullptr;
        return VC_ENOMEM;
    }
    uint8_t *b = static_cast<uint8_t *>(L.mem);
    L.ctrl = reinterpret_cast<Control *>(b + o_ctrl);
    L.problems = b + o_prob;
    L.sub_ring = reinterpret_cast<uint32_t *>(b + o_ring);
    L.sub_tail = reinterpret_cast<uint32_t *>(b + o_tail);
    L.claim_state = reinterpret_cast<unsigned long long *>(b + o_claim);
    L.close_now = reinterpret_cast<int32_t *>(b + o_close);
    L.sm_nodes = reinterpret_cast<unsigned long long *>(b + o_smn);
    L.wl_seq = reinterpret_cast<uint32_t *>(b + o_seq);
    L.wl_slots = b + o_wl;
    L.arena = b + o_arena;
    L.rows = L.nw > 0 ? reinterpret_cast<uint32_t *>(b + o_rows) : nullptr;
    L.stacks = b + o_stacks;
    const size_t stage_bytes =
        (size_t)L.slots * kSlotStride + sizeof(uint32_t) * (2 * (size_t)L.slots + 1) + 64 + sizeof(Control);
    if (cudaMemset(L.mem, 0, o_arena) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void **>(&L.completion_h), sizeof(int32_t) * 4 * (size_t)L.slots,
                      cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(reinterpret_cast<void **>(&L.completion_d), L.completion_h, 0) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void **>(&L.stage_h), stage_bytes, cudaHostAllocDefault) != cudaSuccess ||
        cudaStreamCreateWithFlags(&L.kstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&L.cstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&L.kdone, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return VC_ENOMEM;
    }
    std::memset(L.completion_h, 0, sizeof(int32_t) * 4 * (size_t)L.slots);
    std::memset(L.stage_h, 0, stage_bytes);
    // The worklist initialiser too (it runs before every launch of the lane).
    if (launch_init_worklist(L.wl_seq, L.cap, L.ctrl, L.kstream, L.claim_state) != VC_OK ||
        cudaStreamSynchronize(L.kstream) != cudaSuccess) {
        cudaGetLastError();
        return VC_ECUDA;
    }
    return VC_OK;
}

void free_lane(Lane &L) {
    if (L.kstream) cudaStreamSynchronize(L.kstream);
    if (L.cstream) cudaStreamSynchronize(L.cstream);
    if (L.kdone) cudaEventDestroy(L.kdone);
    if (L.kstream) cudaStreamDestroy(L.kstream);
    if (L.cstream) cudaStreamDestroy(L.cstream);
    if (L.completion_h) cudaFreeHost(L.completion_h);
    if (L.stage_h) cudaFreeHost(L.stage_h);
    if (L.mem) cudaFree(L.mem);
    L.kdone = nullptr;
    L.kstream = L.cstream = nullptr;
    L.completion_h = nullptr;
    L.stage_h = nullptr;
    L.mem = nullptr;
}

}  // namespace
}  // namespace vc

extern "C" {

int vc_server_create(const vc_config *cfg, size_t device_bytes_budget, int32_t max_n, vc_server **out) {
    if (!out || max_n <= 0) return VC_EINVAL;
    *out = nullptr;
    vc_server *s = new vc_server();
    std::memset(&s->cfg, 0, sizeof(s->cfg));
    if (cfg) s->cfg = *cfg;
    // Nodes stay in shared memory or registers.
    if (s->cfg.node_in_global > 0) {
        delete s;
        return VC_EINVAL;
    }
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return VC_ECUDA;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, s->device) != cudaSuccess) {
        delete s;
        return VC_ECUDA;
    }
    s->max_n = max_n;
    s->budget = device_bytes_budget ? device_bytes_budget : (size_t(8) << 30);
    // Size classes: small graphs on bit-row workers when asked for (bit_rows > 0).  By default every
    // request runs on CSR walkers: on the served stream the bit-row class took a quarter of the SM
    // slots from them, and their large requests make the latency tail (p99 2.65 against 2.36 ms).
    const bool small = s->cfg.bit_rows > 0;
    const bool large = !small || max_n > kSmallN;
    const bool both = small && large;
    int rc = VC_OK;
    // With two classes the CSR-walk class takes cfg->num_workers workers if given (else three
    // quarters of every SM's thread slots) and the bit-row class the slots that remain.
    float small_share = both ? 0.25f : 1.f, large_share = both ? 0.75f : 1.f;
    if (both && s->cfg.num_workers > 0) {
        const int wt = s->cfg.worker_threads ? s->cfg.worker_threads : tuned_defaults(max_n).worker_threads;
        const int64_t per_sm = (s->cfg.num_workers + prop.multiProcessorCount - 1) / prop.multiProcessorCount;
        const float used = (float)(per_sm * wt) / (float)kThreadSlotsPerSm;
        if (used >= 1.f) {
            delete s;
            return VC_EINVAL;  // no room left for the bit-row class
        }
        large_share = 1.f;  // the worker count itself is the limit
        small_share = 1.f - used;
    }
    if (small) {
        Lane &L = s->lane[s->nlanes++];
        L.max_n = std::min(max_n, kSmallN);
        L.nw = kSmallRowWords;
        rc = make_lane(s, L, prop, both ? s->budget / 8 : s->budget, small_share);
    }
    if (rc == VC_OK && large) {
        Lane &L = s->lane[s->nlanes++];
        L.max_n = max_n;
        L.nw = 0;
        rc = make_lane(s, L, prop, both ? s->budget - s->budget / 8 : s->budget, large_share);
    }
    if (rc != VC_OK) {
        for (int i = 0; i < s->nlanes; ++i) free_lane(s->lane[i]);
        delete s;
        return rc;
    }
    s->th = std::thread(loop, s);
    *out = s;
    return VC_OK;
}

int vc_server_submit(vc_server *s, const vc_graph *g, int32_t kind, int32_t k, uint64_t *request_id) {
    if (!s || !g || !request_id || g->on_device || g->n < 0 || (kind != 0 && kind != 1)) return VC_EINVAL;
    if (g->n > s->max_n || (g->n > 0 && !g->offsets)) return VC_EINVAL;
    if (!csr_ok(g)) return VC_EINVAL;
    Request *r = new Request();
    r->kind = kind;
    r->k = k;
    r->n = g->n;
    r->lane = (s->nlanes > 1 && g->n > s->lane[0].max_n) ? 1 : 0;
    r->t_submit = now_ns();
    const int64_t len = g->n > 0 ? g->offsets[g->n] : 0;
    if (len < 0 || (len > 0 && !g->neighbors)) {
        delete r;
        return VC_EINVAL;
    }
    if (g->n == 0) r->off.assign(1, 0);  // offsets may be null for an empty graph
    else r->off.assign(g->offsets, g->offsets + g->n + 1);
    if (len > 0) r->adj.assign(g->neighbors, g->neighbors + len);
    r->bytes = up(sizeof(int32_t) * ((size_t)r->n + 1)) + up(sizeof(int32_t) * std::max<size_t>(len, 1)) +
               up(sizeof(int32_t) * std::max<size_t>(r->n, 1)) + up((size_t)s->lane[r->lane].eb);  // + root entry
    if (r->bytes > s->lane[r->lane].arena_bytes) {
        delete r;
        return VC_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
        delete r;
        return VC_EINVAL;
    }
    r->id = s->next_id++;
    s->all[r->id] = r;
    s->outstanding++;
    // Answers that need no search are given at once without a device round trip.
    if (kind == 1 && k < 0) {
        r->answer = 0;
        r->state = 2;
        r->t_done = r->t_admit = now_ns();
        s->outstanding--;
        s->completed++;
        r->off.clear();
        r->adj.clear();
    } else {
        s->lane[r->lane].pending.push_back(r);
        s->cv_work.notify_one();
    }
    *request_id = r->id;
    return VC_OK;
}

int vc_server_poll(vc_server *s, uint64_t request_id, vc_request_info *info) {
    if (!s || !info) return VC_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(request_id);
    if (it == s->all.end()) return VC_EINVAL;
    const Request *r = it->second;
    std::memset(info, 0, sizeof(*info));
    info->done = r->state == 2;
    info->answer = r->answer;
    info->status = r->status;
    info->greedy = r->greedy;
    info->submit_ns = r->t_submit;
    info->admit_ns = r->t_admit;
    info->done_ns = r->t_done;
    return VC_OK;
}

int vc_server_release(vc_server *s, uint64_t request_id) {
    if (!s) return VC_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(request_id);
    if (it == s->all.end() || it->second->state != 2) return VC_EINVAL;  // unknown, or not finished
    delete it->second;  // a finished request is in no queue: nothing else refers to it
    s->all.erase(it);
    return VC_OK;
}

int vc_server_drain(vc_server *s, int64_t timeout_ms) {
    if (!s) return VC_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_work.notify_one();
    auto pred = [&] { return s->outstanding == 0; };
    if (timeout_ms > 0) {
        if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) return VC_ETIMEOUT;
    } else {
        s->cv_done.wait(lk, pred);
    }
    return VC_OK;
}

int vc_server_stats(vc_server *s, vc_server_counters *out) {
    if (!s || !out) return VC_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->completed = s->completed;
    for (int i = 0; i < s->nlanes; ++i) {
        const Lane &L = s->lane[i];
        out->pending += (int64_t)L.pending.size();
        out->in_flight += (int64_t)L.in_flight.size();
        out->launches += L.launches;
        out->epochs += L.epochs;
        out->nodes_visited += (int64_t)L.nodes;
        out->workers += L.workers;
        out->slots_per_epoch += L.slots;
        out->arena_bytes += (int64_t)L.arena_bytes;
    }
    out->worker_threads = s->lane[s->nlanes - 1].wt;
    out->records = (int64_t)s->all.size();
    out->classes = s->nlanes;
    out->small_max_n = s->lane[0].nw > 0 ? s->lane[0].max_n : 0;
    out->small_workers = s->lane[0].nw > 0 ? s->lane[0].workers : 0;
    return VC_OK;
}

int vc_server_destroy(vc_server *s) {
    if (!s) return VC_EINVAL;
    if (s->th.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
            s->cv_work.notify_one();
        }
        s->th.join();
    }
    for (int i = 0; i < s->nlanes; ++i) free_lane(s->lane[i]);
    for (auto &kv : s->all) delete kv.second;
    delete s;
    return VC_OK;
}

}  // extern "C"
