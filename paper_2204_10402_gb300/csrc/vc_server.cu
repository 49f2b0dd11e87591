// vc_server.cu - serving with continuous batching (include/vc_server.h).
//
// One persistent traversal launch (traverse_kernel with Params::serving = 1) works on every
// admitted request at once: idle workers claim new requests from a submission ring, run their
// greedy bound and then search them through the shared worklist, whose entries carry the request's
// slot.  A host thread owned by the server
//   - admits queued requests while their bytes fit: each request reserves a slot and a range of
//     the graph arena (CSR + cover mask); stacks and worklist are sized once for the largest graph
//     the server accepts, so a request fits them whenever its n <= max_n;
//   - uploads the request on a copy stream (CSR, slot record, ring entry, then the ring tail, all
//     ordered on that stream) while the launch keeps running;
//   - harvests completion records that the device writes into host-mapped memory;
//   - relaunches the traversal when requests arrive after an idle launch closed.
// Addresses are never reused within one launch (no L1 can hold stale graph data): slots and arena
// ranges are handed out in order within an "epoch"; when an epoch is used up, admission pauses
// until the requests in flight finish, the launch closes and the epoch restarts.
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

#include "vc_internal.h"
#include "vc_tuning.h"
#include "vc_launch.h"
#include "../../include/vc_server.h"

namespace vc {
namespace {

constexpr int32_t kSlotStride = 128;  // bytes per problem record (one cache line, never shared)
constexpr size_t kAlign = 128;

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}
size_t up(size_t b) { return (b + kAlign - 1) & ~(kAlign - 1); }

struct Request {
    uint64_t id = 0;
    int32_t kind = 0, k = 0, n = 0;
    std::vector<int32_t> off, adj;
    int32_t slot = -1;
    int32_t tag = 0;
    int32_t state = 0;  // 0 queued, 1 in flight, 2 done
    int32_t answer = -1, status = VC_OK, greedy = -1;
    int64_t t_submit = 0, t_admit = 0, t_done = 0;
    size_t bytes = 0;
};

}  // namespace
}  // namespace vc

using namespace vc;

struct vc_server {
    vc_config cfg;
    int device = 0;
    int32_t max_n = 0;
    size_t budget = 0;
    // variant
    int wt = 0, width = 16, smem = 0, workers = 0, eb = 0, depth = 0, cap = 0, threshold = 0;
    int32_t csr_words = 0;
    int32_t slots = 0;          // problem slots per epoch (power of two, also the ring capacity)
    size_t arena_bytes = 0;
    // device memory
    void *mem = nullptr;        // one allocation carved into the regions below
    Control *ctrl = nullptr;
    uint8_t *problems = nullptr;
    uint8_t *arena = nullptr;
    uint8_t *stacks = nullptr, *wl_slots = nullptr;
    uint32_t *wl_seq = nullptr, *sub_ring = nullptr, *sub_tail = nullptr;
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
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;
    std::vector<Request *> in_flight;
    std::unordered_map<uint64_t, Request *> all;
    uint64_t next_id = 1;
    int64_t outstanding = 0;
    bool stop = false;
    std::thread th;
    // counters
    unsigned long long nodes = 0;
    int64_t launches = 0, epochs = 0, completed = 0;
    int32_t last_status = VC_OK;
};

namespace vc {
namespace {

Problem *stage_problem(vc_server *s, int32_t slot) {
    return reinterpret_cast<Problem *>(s->stage_h + (size_t)slot * kSlotStride);
}
uint32_t *stage_ring(vc_server *s) {
    return reinterpret_cast<uint32_t *>(s->stage_h + (size_t)s->slots * kSlotStride);
}
uint32_t *stage_tail(vc_server *s) { return stage_ring(s) + s->slots; }
int32_t *stage_flags(vc_server *s) { return reinterpret_cast<int32_t *>(stage_tail(s) + s->slots + 1); }

Params serve_params(vc_server *s) {
    Params P;
    std::memset(&P, 0, sizeof(P));
    P.offsets = reinterpret_cast<const int32_t *>(s->arena);
    P.neighbors = reinterpret_cast<const int32_t *>(s->arena);
    P.problems = reinterpret_cast<Problem *>(s->problems);
    P.num_problems = s->slots;
    P.n_max = s->max_n;
    P.entry_bytes = s->eb;
    P.stack_depth = s->depth;
    P.ctrl = s->ctrl;
    P.cover = reinterpret_cast<int32_t *>(s->arena);
    P.stacks = s->stacks;
    P.wl_slots = s->wl_slots;
    P.wl_seq = s->wl_seq;
    P.wl_capacity = s->cap;
    P.wl_threshold = s->threshold;
    P.csr_words = s->csr_words;
    P.idle_timeout_ns = s->cfg.idle_timeout_ns > 0 ? s->cfg.idle_timeout_ns : 20000000000ll;
    P.cancel = s->cfg.cancel;
    P.sm_nodes = s->sm_nodes;
    P.serving = 1;
    P.sub_mask = (uint32_t)s->slots - 1u;
    P.sub_ring = s->sub_ring;
    P.sub_tail = s->sub_tail;
    P.claim_state = s->claim_state;
    P.close_now = s->close_now;
    P.completion = s->completion_d;
    P.linger_ns = 2000000;  // an empty launch closes after 2 ms idle
    return P;
}

// Launches the persistent traversal (the server lock is held).
int launch(vc_server *s) {
    const Launchers &L = s->width == 16 ? launchers_w16() : launchers_w32();
    if (cudaMemsetAsync(s->ctrl, 0, sizeof(Control), s->kstream) != cudaSuccess) return VC_ECUDA;
    if (cudaMemsetAsync(s->close_now, 0, sizeof(int32_t), s->kstream) != cudaSuccess) return VC_ECUDA;
    Params P = serve_params(s);
    if (int rc = launch_init_worklist(s->wl_seq, s->cap, s->ctrl, s->kstream, s->claim_state)) return rc;
    if (int rc = L.traverse(s->wt, s->workers, s->smem, s->kstream, P)) return rc;
    if (cudaEventRecord(s->kdone, s->kstream) != cudaSuccess) return VC_ECUDA;
    s->running = true;
    s->close_sent = false;
    s->launches++;
    return VC_OK;
}

// Reads the statistics of a launch that has ended.
void collect(vc_server *s) {
    Control c;
    if (cudaMemcpy(&c, s->ctrl, sizeof(Control), cudaMemcpyDeviceToHost) == cudaSuccess) {
        s->nodes += c.nodes;
        if (c.status != VC_OK) s->last_status = c.status;
    } else {
        cudaGetLastError();
    }
}

// Admits queued requests that fit the current epoch and publishes them (the server lock is held).
int admit(vc_server *s) {
    uint32_t first = s->published;
    while (!s->pending.empty() && !s->draining) {
        Request *r = s->pending.front();
        if (s->next_slot >= s->slots || s->arena_used + r->bytes > s->arena_bytes) {
            s->draining = true;  // epoch used up: finish what is in flight, then restart
            break;
        }
        s->pending.pop_front();
        const int32_t slot = s->next_slot++;
        const size_t base = s->arena_used;
        s->arena_used += r->bytes;
        const size_t off_bytes = up(sizeof(int32_t) * ((size_t)r->n + 1));
        const size_t adj_bytes = up(sizeof(int32_t) * std::max<size_t>(r->adj.size(), 1));
        Problem *p = stage_problem(s, slot);
        std::memset(p, 0, sizeof(Problem));
        p->off_base = (int64_t)(base / 4);
        p->adj_base = (int64_t)((base + off_bytes) / 4);
        p->cover_base = (int64_t)((base + off_bytes + adj_bytes) / 4);
        p->n = r->n;
        p->kind = r->kind;
        p->k = r->k;
        p->best = INT_MAX;
        p->cover_size = INT_MAX;
        r->slot = slot;
        r->tag = (int32_t)((r->id & 0x3fffffff) | 0x40000000);  // nonzero, and unlike any older tag
        p->tag = r->tag;
        s->completion_h[4 * slot] = 0;
        if (cudaMemcpyAsync(s->arena + base, r->off.data(), sizeof(int32_t) * r->off.size(), cudaMemcpyHostToDevice,
                            s->cstream) != cudaSuccess ||
            (!r->adj.empty() && cudaMemcpyAsync(s->arena + base + off_bytes, r->adj.data(),
                                                sizeof(int32_t) * r->adj.size(), cudaMemcpyHostToDevice,
                                                s->cstream) != cudaSuccess) ||
            cudaMemcpyAsync(s->problems + (size_t)slot * kSlotStride, p, sizeof(Problem), cudaMemcpyHostToDevice,
                            s->cstream) != cudaSuccess)
            return VC_ECUDA;
        uint32_t *ring = stage_ring(s);
        ring[s->published] = (uint32_t)slot;
        if (cudaMemcpyAsync(s->sub_ring + (s->published & (uint32_t)(s->slots - 1)), &ring[s->published],
                            sizeof(uint32_t), cudaMemcpyHostToDevice, s->cstream) != cudaSuccess)
            return VC_ECUDA;
        s->published++;
        r->state = 1;
        r->t_admit = now_ns();
        s->in_flight.push_back(r);
    }
    if (s->published != first) {
        // The tail goes last on the copy stream: every entry it covers is in place when it lands.
        uint32_t *tail = stage_tail(s);
        tail[s->published] = s->published;
        if (cudaMemcpyAsync(s->sub_tail, &tail[s->published], sizeof(uint32_t), cudaMemcpyHostToDevice,
                            s->cstream) != cudaSuccess)
            return VC_ECUDA;
    }
    return VC_OK;
}

// Harvests completion records (the server lock is held).  Returns how many finished.
int harvest(vc_server *s) {
    int done = 0;
    volatile int32_t *rec = s->completion_h;
    for (size_t i = 0; i < s->in_flight.size();) {
        Request *r = s->in_flight[i];
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
            s->in_flight[i] = s->in_flight.back();
            s->in_flight.pop_back();
            s->outstanding--;
            s->completed++;
            done++;
        } else {
            ++i;
        }
    }
    return done;
}

// Starts a new epoch (no launch running, nothing in flight; the server lock is held).
int reset_epoch(vc_server *s) {
    s->next_slot = 0;
    s->arena_used = 0;
    s->published = 0;
    s->draining = false;
    s->epochs++;
    if (cudaMemsetAsync(s->claim_state, 0, sizeof(unsigned long long), s->cstream) != cudaSuccess ||
        cudaMemsetAsync(s->sub_tail, 0, sizeof(uint32_t), s->cstream) != cudaSuccess ||
        cudaStreamSynchronize(s->cstream) != cudaSuccess)
        return VC_ECUDA;
    return VC_OK;
}

void fail_all(vc_server *s, int32_t code) {
    for (Request *r : s->in_flight) {
        r->status = code;
        r->state = 2;
        r->t_done = now_ns();
        s->outstanding--;
    }
    s->in_flight.clear();
    for (Request *r : s->pending) {
        r->status = code;
        r->state = 2;
        r->t_done = now_ns();
        s->outstanding--;
    }
    s->pending.clear();
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

void loop(vc_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        bool progress = false;
        if (harvest(s)) {
            progress = true;
            s->cv_done.notify_all();
        }
        if (s->running && cudaEventQuery(s->kdone) == cudaSuccess) {
            s->running = false;
            collect(s);
            progress = true;
            if (s->last_status != VC_OK) {  // the launch failed: report it on everything open
                harvest(s);
                fail_all(s, s->last_status);
                s->last_status = VC_OK;
                s->cv_done.notify_all();
                if (s->draining || s->published) reset_epoch(s);
            }
        } else if (s->running) {
            cudaGetLastError();
        }
        if (s->stop && s->pending.empty() && s->in_flight.empty() && !s->running) break;
        if (!s->running && s->draining && s->in_flight.empty()) {
            if (reset_epoch(s) != VC_OK) {
                fail_all(s, VC_ECUDA);
                s->cv_done.notify_all();
            }
            progress = true;
        }
        const uint32_t before = s->published;
        if (admit(s) != VC_OK) {
            fail_all(s, VC_ECUDA);
            s->cv_done.notify_all();
        }
        if (s->published != before) progress = true;
        if (!s->running && !s->in_flight.empty()) {
            // Requests are published but no launch is running: start one once the uploads landed.
            if (cudaStreamSynchronize(s->cstream) != cudaSuccess || launch(s) != VC_OK) {
                cudaGetLastError();
                fail_all(s, VC_ECUDA);
                s->cv_done.notify_all();
            }
            progress = true;
        }
        if (s->running && !s->close_sent && s->in_flight.empty() && (s->draining || s->stop)) {
            int32_t *flag = stage_flags(s);
            flag[0] = 1;
            cudaMemcpyAsync(s->close_now, flag, sizeof(int32_t), cudaMemcpyHostToDevice, s->cstream);
            s->close_sent = true;
        }
        if (!progress) {
            const bool busy = s->running || !s->pending.empty();
            s->cv_work.wait_for(lk, std::chrono::microseconds(busy ? 20 : 2000));
        }
    }
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
    if (s->cfg.node_in_global > 0) {  // the server keeps the node in shared memory
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
    const LaunchDefaults tuned = tuned_defaults(max_n);
    s->width = s->cfg.width ? s->cfg.width : tuned.width;
    if ((s->width != 16 && s->width != 32) || (s->width == 16 && max_n > 32768)) {
        delete s;
        return VC_EINVAL;
    }
    s->wt = s->cfg.worker_threads ? s->cfg.worker_threads : tuned.worker_threads;
    s->csr_words = default_csr_words(max_n, s->cfg.stage_csr);
    s->smem = smem_bytes_for(max_n, s->width / 8, s->csr_words);
    if (s->smem > (int)prop.sharedMemPerBlockOptin) {
        delete s;
        return VC_EINVAL;
    }
    const Launchers &L = s->width == 16 ? launchers_w16() : launchers_w32();
    int per_sm = 0;
    if (L.occupancy(s->wt, s->smem, &per_sm) != VC_OK || per_sm <= 0) {
        delete s;
        return VC_EINVAL;
    }
    s->eb = entry_bytes_for(max_n, s->width / 8);
    s->depth = max_n + 3;  // MVC depth <= n + 1, PVC depth <= min(k, n) + 2
    s->slots = 4096;
    // Worklist: the batch default, limited to an eighth of the budget.
    s->cap = default_worklist_capacity(s->eb);
    while (s->cap > 1024 && (size_t)s->cap * (size_t)s->eb > s->budget / 8) s->cap >>= 1;
    // Budget: half for the stacks (as many workers as fit), a quarter for the graph arena.
    const size_t per_worker = (size_t)s->depth * (size_t)s->eb;
    int64_t w = s->cfg.num_workers > 0 ? s->cfg.num_workers : (int64_t)prop.multiProcessorCount * per_sm;
    w = std::min<int64_t>(w, (int64_t)(s->budget / 2 / per_worker));
    if (w < 1) {
        delete s;
        return VC_ENOMEM;
    }
    s->workers = (int)w;
    float frac = s->cfg.donate_threshold > 0.f ? s->cfg.donate_threshold : tuned.threshold;
    s->threshold = std::max(1, (int)(frac * s->cap));
    if (s->cfg.worklist_capacity > 0) {
        int c = 1;
        while (c < s->cfg.worklist_capacity) c <<= 1;
        s->cap = c;
        s->threshold = std::max(1, (int)(frac * c));
    }
    s->arena_bytes = std::max<size_t>(s->budget / 4, 64 << 10);
    // One device allocation for everything.
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t at = off;
        off += up(b);
        return at;
    };
    const size_t o_ctrl = take(sizeof(Control));
    const size_t o_prob = take((size_t)s->slots * kSlotStride);
    const size_t o_ring = take(sizeof(uint32_t) * (size_t)s->slots);
    const size_t o_tail = take(sizeof(uint32_t));
    const size_t o_claim = take(sizeof(unsigned long long));
    const size_t o_close = take(sizeof(int32_t));
    const size_t o_smn = take(sizeof(unsigned long long) * kSmSlots);
    const size_t o_seq = take(sizeof(uint32_t) * (size_t)s->cap);
    const size_t o_wl = take((size_t)s->cap * (size_t)s->eb);
    const size_t o_arena = take(s->arena_bytes);
    const size_t o_stacks = take((size_t)s->workers * per_worker);
    if (cudaMalloc(&s->mem, off) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return VC_ENOMEM;
    }
    uint8_t *b = static_cast<uint8_t *>(s->mem);
    s->ctrl = reinterpret_cast<Control *>(b + o_ctrl);
    s->problems = b + o_prob;
    s->sub_ring = reinterpret_cast<uint32_t *>(b + o_ring);
    s->sub_tail = reinterpret_cast<uint32_t *>(b + o_tail);
    s->claim_state = reinterpret_cast<unsigned long long *>(b + o_claim);
    s->close_now = reinterpret_cast<int32_t *>(b + o_close);
    s->sm_nodes = reinterpret_cast<unsigned long long *>(b + o_smn);
    s->wl_seq = reinterpret_cast<uint32_t *>(b + o_seq);
    s->wl_slots = b + o_wl;
    s->arena = b + o_arena;
    s->stacks = b + o_stacks;
    const size_t stage_bytes = (size_t)s->slots * kSlotStride + sizeof(uint32_t) * (2 * (size_t)s->slots + 1) + 64;
    if (cudaMemset(s->mem, 0, o_arena) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void **>(&s->completion_h), sizeof(int32_t) * 4 * (size_t)s->slots,
                      cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(reinterpret_cast<void **>(&s->completion_d), s->completion_h, 0) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void **>(&s->stage_h), stage_bytes, cudaHostAllocDefault) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->kstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->cstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->kdone, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        vc_server_destroy(s);
        return VC_ENOMEM;
    }
    std::memset(s->completion_h, 0, sizeof(int32_t) * 4 * (size_t)s->slots);
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
               up(sizeof(int32_t) * std::max<size_t>(r->n, 1));
    if (r->bytes > s->arena_bytes) {
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
        s->pending.push_back(r);
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
    out->pending = (int64_t)s->pending.size();
    out->in_flight = (int64_t)s->in_flight.size();
    out->launches = s->launches;
    out->epochs = s->epochs;
    out->nodes_visited = (int64_t)s->nodes;
    out->workers = s->workers;
    out->worker_threads = s->wt;
    out->slots_per_epoch = s->slots;
    out->arena_bytes = (int64_t)s->arena_bytes;
    out->records = (int64_t)s->all.size();
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
    if (s->kstream) cudaStreamSynchronize(s->kstream);
    if (s->cstream) cudaStreamSynchronize(s->cstream);
    if (s->kdone) cudaEventDestroy(s->kdone);
    if (s->kstream) cudaStreamDestroy(s->kstream);
    if (s->cstream) cudaStreamDestroy(s->cstream);
    if (s->completion_h) cudaFreeHost(s->completion_h);
    if (s->stage_h) cudaFreeHost(s->stage_h);
    if (s->mem) cudaFree(s->mem);
    for (auto &kv : s->all) delete kv.second;
    delete s;
    return VC_OK;
}

}  // extern "C"
