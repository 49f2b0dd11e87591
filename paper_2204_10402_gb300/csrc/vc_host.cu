// vc_host.cu - the C ABI of libvc (include/vc.h): argument checks, the cached per-device
// workspace, variant selection, and the launch sequence
//   validate -> worklist init -> greedy -> traverse -> copy results back
// on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <climits>
#include <cstring>
#include <mutex>
#include <vector>

#include "vc_internal.h"
#include "vc_tuning.h"
#include "vc_launch.h"

namespace vc {
namespace {

constexpr int kMaxDevices = 64;
constexpr size_t kStackBudget = size_t(8) << 30;  // stacks beyond this size trigger a tighter depth
constexpr size_t kBounceBytes = size_t(256) << 10;  // host arrays up to this size bounce through pinned memory
constexpr int64_t kMinCappedDepth = 256;           // smallest per-worker depth worth a capped launch
constexpr int64_t kDefaultIdleTimeoutNs = 20000000000ll;

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

struct Workspace {
    bool ready = false;
    int device = -1;
    int sms = 0;
    int smem_optin = 0;
    DevBuf csr_off, csr_adj, problems, adj_len, ctrl, cover, stacks, wl_slots, wl_seq, gstate, rows, roots;
    DevBuf meta;  // run(): problem records, lengths, control block and per-SM counts, laid out as in `pinned`
    void *pinned = nullptr;
    size_t pinned_cap = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<long long> last_sm_nodes;
};

std::mutex g_mu;
Workspace g_ws[kMaxDevices];

#define VC_CK(call)                                  \
    do {                                             \
        if ((call) != cudaSuccess) {                 \
            cudaGetLastError();                      \
            return VC_ECUDA;                         \
        }                                            \
    } while (0)

#define VC_RC(expr)                  \
    do {                             \
        int rc_ = (expr);            \
        if (rc_ != VC_OK) return rc_; \
    } while (0)

int grow(DevBuf &b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.cap >= bytes) return VC_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    size_t nb = bytes + bytes / 4;
    if (cudaMalloc(&b.p, nb) != cudaSuccess) {
        cudaGetLastError();
        nb = bytes;
        if (cudaMalloc(&b.p, nb) != cudaSuccess) {
            cudaGetLastError();
            b.p = nullptr;
            return VC_ENOMEM;
        }
    }
    b.cap = nb;
    return VC_OK;
}

int grow_pinned(Workspace &ws, size_t bytes) {
    if (ws.pinned_cap >= bytes) return VC_OK;
    if (ws.pinned) cudaFreeHost(ws.pinned);
    ws.pinned = nullptr;
    ws.pinned_cap = 0;
    const size_t nb = std::max<size_t>(bytes + bytes / 4, 4096);
    if (cudaMallocHost(&ws.pinned, nb) != cudaSuccess) {
        cudaGetLastError();
        ws.pinned = nullptr;
        return VC_ENOMEM;
    }
    ws.pinned_cap = nb;
    return VC_OK;
}

int workspace(Workspace **out) {
    int dev = 0;
    VC_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return VC_EINVAL;
    Workspace &ws = g_ws[dev];
    if (!ws.ready) {
        cudaDeviceProp prop;
        VC_CK(cudaGetDeviceProperties(&prop, dev));
        ws.device = dev;
        ws.sms = prop.multiProcessorCount;
        ws.smem_optin = (int)prop.sharedMemPerBlockOptin;
        VC_CK(cudaEventCreate(&ws.ev0));
        VC_CK(cudaEventCreate(&ws.ev1));
        ws.ready = true;
    }
    *out = &ws;
    return VC_OK;
}

void free_workspace(Workspace &ws) {
    DevBuf *bufs[] = {&ws.csr_off, &ws.csr_adj, &ws.problems, &ws.adj_len, &ws.ctrl, &ws.cover,
                      &ws.stacks, &ws.wl_slots, &ws.wl_seq, &ws.gstate, &ws.rows, &ws.roots,
                      &ws.meta};
    for (DevBuf *b : bufs) {
        if (b->p) cudaFree(b->p);
        b->p = nullptr;
        b->cap = 0;
    }
    if (ws.pinned) cudaFreeHost(ws.pinned);
    ws.pinned = nullptr;
    ws.pinned_cap = 0;
}

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }
int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Host description of one launch.
struct Spec {
    std::vector<Problem> probs;
    std::vector<int64_t> adj_len;   // expected offsets[n] per problem, -1 unknown
    const int32_t *offsets = nullptr;
    const int32_t *neighbors = nullptr;
    int on_device = 0;
    int64_t total_offsets = 0;      // entries of the packed offsets array (host inputs)
    int64_t total_adj = 0;          // entries of the packed neighbour array (host inputs)
    int64_t total_vertices = 0;
    int32_t n_max = 0;
    bool search = true;             // false: greedy only
};

struct Result {
    std::vector<Problem> probs;
    Control ctrl;
    float kernel_ms = 0.f;
    int workers = 0, wt = 0, width = 0, stack_depth = 0, nw = 0, eb = 0;
    bool csr_staged = false, gm = false;
};

constexpr int32_t kWideGreedyN = 400;  // single graphs above this size get the wide greedy block

Problem make_problem(int64_t off_base, int64_t adj_base, int64_t cover_base, int32_t n, int32_t kind, int32_t k) {
    Problem p;
    std::memset(&p, 0, sizeof(p));
    p.off_base = off_base;
    p.adj_base = adj_base;
    p.cover_base = cover_base;
    p.n = n;
    p.kind = kind;
    p.k = k;
    p.best = INT_MAX;
    p.cover_size = INT_MAX;
    return p;
}

// Waits for a call's queued work on every return, error paths included.  Declared after the
// workspace lock, it runs before the lock is released: the workspace is the next call's then, so
// nothing may still run on it.
struct StreamDrain {
    cudaStream_t s;
    ~StreamDrain() {
        if (cudaStreamSynchronize(s) != cudaSuccess) cudaGetLastError();
    }
};

// Runs one launch.  cover_out (may be null) receives Σ n cover entries, on the device or host.
int run(Workspace &ws, const Spec &spec, const vc_config *cfg_in, cudaStream_t s, int32_t *cover_out,
        int cover_on_device, Result &res) {
    StreamDrain drain{s};
    vc_config cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    if (cfg_in) cfg = *cfg_in;
    const int G = (int)spec.probs.size();
    const int n_max = std::max(spec.n_max, 1);

    // ---- variant: degree-array width and worker size ----
    const LaunchDefaults tuned = tuned_defaults(n_max);
    int width = cfg.width ? cfg.width : tuned.width;
    if (width != 16 && width != 32) return VC_EINVAL;
    if (width == 16 && n_max > 32768) return VC_EINVAL;
    const int wbytes = width / 8;
    int wt = cfg.worker_threads ? cfg.worker_threads : tuned.worker_threads;
    if (!is_pow2(wt) || wt < 32 || wt > 512) return VC_EINVAL;
    // CSR staging in shared memory: when every graph's CSR size is known and small enough, each
    // worker keeps a copy of its current graph's CSR next to the degree array.
    int64_t csr_need = 0;
    bool known = true;
    for (size_t i = 0; i < spec.probs.size(); ++i) {
        if (spec.adj_len[i] < 0) known = false;
        else csr_need = std::max<int64_t>(csr_need, (int64_t)spec.probs[i].n + 1 + spec.adj_len[i]);
    }
    // Default: stage only the offsets (n+1 ints) of graphs up to kOffsetStageN vertices; with
    // stage_csr = 1 stage the neighbour lists too; with stage_csr = -1 stage nothing.
    int32_t csr_words = 0;
    if (known && cfg.stage_csr > 0 && csr_need > 0 && csr_need * 4 <= (int64_t)ws.smem_optin)
        csr_words = (int32_t)csr_need;
    else
        csr_words = default_csr_words(n_max, cfg.stage_csr);
    int smem = smem_bytes_for(n_max, wbytes, csr_words);
    if (smem > ws.smem_optin && csr_words) {
        csr_words = 0;
        smem = smem_bytes_for(n_max, wbytes, 0);
    }
    // Node placement (Sec. IV-E): shared memory when it fits, else the global-memory version.
    const bool gm = cfg.node_in_global > 0 || (cfg.node_in_global == 0 && smem > ws.smem_optin);
    if (gm) {
        csr_words = default_csr_words(n_max, cfg.stage_csr);
        if (known && cfg.stage_csr > 0 && csr_need > 0 && smem_bytes_gm((int32_t)csr_need) <= ws.smem_optin)
            csr_words = (int32_t)csr_need;
        smem = smem_bytes_gm(csr_words);
    }
    if (smem > ws.smem_optin) return VC_EINVAL;  // graph too large for a shared-memory degree array
    // Bit-row workers: one warp per worker, node in registers, n_max <= 256.
    int nw = 0;
    if (cfg.bit_rows >= 0 && !gm && wt == 32) nw = rows_words_for(n_max);
    if (cfg.bit_rows > 0 && nw == 0) return VC_EINVAL;
    if (nw > 0 && smem_bytes_for(n_max, wbytes, csr_words, nw) <= ws.smem_optin)
        smem = smem_bytes_for(n_max, wbytes, csr_words, nw);
    else nw = 0;
    const Launchers &L = launchers(width, gm, nw);
    int per_sm = 0;
    VC_RC(L.occupancy(wt, smem, &per_sm));
    if (per_sm <= 0) return VC_EINVAL;
    int workers = cfg.num_workers > 0 ? cfg.num_workers : ws.sms * per_sm;
    const int32_t eb = entry_bytes_for(n_max, wbytes);

    // ---- worklist sizing (Sec. V-A explores 128K-512K entries, threshold 0.25-1.0 x size) ----
    int cap = cfg.worklist_capacity > 0 ? next_pow2(cfg.worklist_capacity) : default_worklist_capacity(eb, tuned.capacity);
    float frac = cfg.donate_threshold > 0.f ? cfg.donate_threshold : tuned.threshold;
    int threshold = (int)std::max<double>(0.0, std::min<double>(cap, (double)frac * cap));
    if (cfg.donate_threshold < 0.f) threshold = 0;  // never donate (stress setting)

    // ---- stack depth: every branch adds >= 1 vertex to S, and S stays below best (MVC) or at
    //      most k (PVC), so depth <= greedy bound (MVC) or k + 1 (PVC) (Sec. IV-E) ----
    int64_t depth = 2;
    for (const Problem &p : spec.probs) {
        const int64_t dp = p.kind == kMVC ? (int64_t)p.n + 2 : (int64_t)std::min(p.k, p.n) + 3;
        depth = std::max(depth, dp);
    }

    // ---- device buffers ----
    VC_RC(grow(ws.cover, sizeof(int32_t) * (size_t)std::max<int64_t>(spec.total_vertices, 1)));
    // The problem records, their adjacency lengths, the control block and the per-SM counts share
    // one device buffer laid out like their pinned staging: one upload sets them all (the control
    // block and the counts as zeros) and one download reads them back, instead of two copies and
    // two memsets before the launch and three copies after it.
    const size_t adj_len_at = sizeof(Problem) * (size_t)G;
    const size_t ctrl_at = (adj_len_at + sizeof(int64_t) * (size_t)G + 127) & ~size_t(127);
    const size_t smn_at = (ctrl_at + sizeof(Control) + 127) & ~size_t(127);
    // Small host arrays (a single request's CSR and cover) bounce through the same pinned region:
    // a copy from or to pageable memory would be staged by the driver and synchronise by itself.
    const size_t in_bytes = sizeof(int32_t) * (size_t)(spec.total_offsets + std::max<int64_t>(spec.total_adj, 0));
    const size_t out_bytes = sizeof(int32_t) * (size_t)std::max<int64_t>(spec.total_vertices, 0);
    const bool bounce_in = !spec.on_device && in_bytes <= kBounceBytes;
    const bool bounce_out = cover_out && !cover_on_device && out_bytes > 0 && out_bytes <= kBounceBytes;
    const size_t in_at = (smn_at + sizeof(unsigned long long) * (size_t)kSmSlots + 127) & ~size_t(127);
    const size_t out_at = (in_at + (bounce_in ? in_bytes : 0) + 127) & ~size_t(127);
    const size_t meta_bytes = smn_at + sizeof(unsigned long long) * (size_t)kSmSlots;
    VC_RC(grow(ws.meta, meta_bytes));
    VC_RC(grow_pinned(ws, out_at + (bounce_out ? out_bytes : 0)));
    Problem *h_probs = reinterpret_cast<Problem *>(ws.pinned);
    int64_t *h_adj_len = reinterpret_cast<int64_t *>(static_cast<uint8_t *>(ws.pinned) + adj_len_at);
    Control *h_ctrl = reinterpret_cast<Control *>(static_cast<uint8_t *>(ws.pinned) + ctrl_at);
    // per-SM node counts of the launch (vc_last_sm_nodes), staged in pinned memory like the rest
    unsigned long long *smn = reinterpret_cast<unsigned long long *>(static_cast<uint8_t *>(ws.pinned) + smn_at);
    std::memcpy(h_probs, spec.probs.data(), sizeof(Problem) * (size_t)G);
    for (int g = 0; g < G; ++g) h_probs[g].root_base = (int64_t)g * eb;  // one root entry per problem
    std::memcpy(h_adj_len, spec.adj_len.data(), sizeof(int64_t) * (size_t)G);
    std::memset(h_ctrl, 0, sizeof(Control));
    std::memset(smn, 0, sizeof(unsigned long long) * (size_t)kSmSlots);

    const int32_t *d_off = spec.offsets, *d_adj = spec.neighbors;
    if (!spec.on_device) {
        VC_RC(grow(ws.csr_off, sizeof(int32_t) * (size_t)std::max<int64_t>(spec.total_offsets, 1)));
        VC_RC(grow(ws.csr_adj, sizeof(int32_t) * (size_t)std::max<int64_t>(spec.total_adj, 1)));
        const int32_t *src_off = spec.offsets, *src_adj = spec.neighbors;
        if (bounce_in) {
            int32_t *b = reinterpret_cast<int32_t *>(static_cast<uint8_t *>(ws.pinned) + in_at);
            std::memcpy(b, spec.offsets, sizeof(int32_t) * (size_t)spec.total_offsets);
            if (spec.total_adj > 0) std::memcpy(b + spec.total_offsets, spec.neighbors, sizeof(int32_t) * (size_t)spec.total_adj);
            src_off = b;
            src_adj = b + spec.total_offsets;
        }
        VC_CK(cudaMemcpyAsync(ws.csr_off.p, src_off, sizeof(int32_t) * spec.total_offsets,
                              cudaMemcpyHostToDevice, s));
        if (spec.total_adj > 0)
            VC_CK(cudaMemcpyAsync(ws.csr_adj.p, src_adj, sizeof(int32_t) * spec.total_adj,
                                  cudaMemcpyHostToDevice, s));
        d_off = static_cast<const int32_t *>(ws.csr_off.p);
        d_adj = static_cast<const int32_t *>(ws.csr_adj.p);
    }
    uint8_t *dm = static_cast<uint8_t *>(ws.meta.p);
    Problem *d_probs = reinterpret_cast<Problem *>(dm);
    const int64_t *d_adj_len = reinterpret_cast<const int64_t *>(dm + adj_len_at);
    Control *d_ctrl = reinterpret_cast<Control *>(dm + ctrl_at);
    VC_CK(cudaMemcpyAsync(dm, ws.pinned, meta_bytes, cudaMemcpyHostToDevice, s));

    Params P;
    std::memset(&P, 0, sizeof(P));
    P.offsets = d_off;
    P.neighbors = d_adj;
    P.problems = d_probs;
    P.num_problems = G;
    P.n_max = n_max;
    P.entry_bytes = eb;
    P.ctrl = d_ctrl;
    // A device cover_out is written by the kernels themselves (the greedy pass writes every entry
    // before any search records a better cover), which saves the copy at the end.
    const bool direct_cover = cover_out && cover_on_device && spec.total_vertices > 0;
    P.cover = direct_cover ? cover_out : static_cast<int32_t *>(ws.cover.p);
    P.wl_capacity = cap;
    P.wl_threshold = threshold;
    P.csr_words = csr_words;
    P.idle_timeout_ns = cfg.idle_timeout_ns > 0 ? cfg.idle_timeout_ns : kDefaultIdleTimeoutNs;
    P.cancel = cfg.cancel;
    P.sm_nodes = reinterpret_cast<unsigned long long *>(dm + smn_at);
    if (gm) {
        P.gstate_bytes = gstate_bytes_for(n_max, wbytes);
        VC_RC(grow(ws.gstate, (size_t)workers * (size_t)P.gstate_bytes));
        P.gstate = static_cast<uint8_t *>(ws.gstate.p);
    }
    if (nw > 0) {  // the greedy pass writes each graph's bit rows here; the traversal copies them
        VC_RC(grow(ws.rows, sizeof(uint32_t) * (size_t)nw * (size_t)std::max<int64_t>(spec.total_vertices, 1)));
        P.rows = static_cast<uint32_t *>(ws.rows.p);
    }
    // The greedy pass keeps each problem's first fixpoint here as its root node.
    VC_RC(grow(ws.roots, (size_t)G * (size_t)eb));
    P.roots = static_cast<uint8_t *>(ws.roots.p);

    if (!cfg.skip_validation)
        VC_RC(launch_validate(d_off, d_adj, d_probs, d_adj_len, G, spec.total_vertices, d_ctrl, s));
    // A single large graph's greedy pass is one worker's sequential rounds: it runs on a 512-thread
    // block whatever the traversal's worker size (Chung-Lu graphs of 1,000-3,000 vertices: 40 %
    // less greedy time than with their 128- or 256-thread workers).
    const int greedy_wt = (G == 1 && nw == 0 && n_max > kWideGreedyN) ? std::max(wt, 512) : wt;
    VC_RC(L.greedy(greedy_wt, std::min(G, workers), smem, s, P));

    if (spec.search) {
        // Tighten the depth with the greedy bound when the generic bound would need too much memory.
        if ((size_t)workers * (size_t)depth * (size_t)eb > kStackBudget) {
            VC_CK(cudaMemcpyAsync(h_probs, d_probs, sizeof(Problem) * (size_t)G, cudaMemcpyDeviceToHost, s));
            VC_CK(cudaStreamSynchronize(s));
            int64_t d2 = 2;
            for (int i = 0; i < G; ++i) {
                const Problem &p = h_probs[i];
                d2 = std::max<int64_t>(d2, p.kind == kMVC ? (int64_t)p.greedy + 2 : (int64_t)std::min(p.k, p.n) + 3);
            }
            depth = std::min(depth, d2);
            // Still over the budget (large graphs): halve the workers while each would get fewer
            // than kMinCappedDepth entries, then cap the depth to what fits; a search that goes
            // deeper than the cap stops with VC_ESTACK.
            auto fit = [&] { return (int64_t)(kStackBudget / ((size_t)workers * (size_t)eb)); };
            while (workers > ws.sms && depth > fit() && fit() < kMinCappedDepth) workers /= 2;
            if (depth > fit()) depth = std::max<int64_t>(fit(), 2);
        }
        P.stack_depth = (int32_t)depth;
        VC_RC(grow(ws.stacks, (size_t)workers * (size_t)depth * (size_t)eb));
        VC_RC(grow(ws.wl_slots, (size_t)cap * (size_t)eb));
        VC_RC(grow(ws.wl_seq, sizeof(uint32_t) * (size_t)cap));
        P.stacks = static_cast<uint8_t *>(ws.stacks.p);
        P.wl_slots = static_cast<uint8_t *>(ws.wl_slots.p);
        P.wl_seq = static_cast<uint32_t *>(ws.wl_seq.p);
        VC_RC(launch_init_worklist(P.wl_seq, cap, d_ctrl, s));
        VC_CK(cudaEventRecord(ws.ev0, s));
        VC_RC(L.traverse(wt, workers, smem, s, P));
        VC_CK(cudaEventRecord(ws.ev1, s));
    }

    VC_CK(cudaMemcpyAsync(ws.pinned, dm, meta_bytes, cudaMemcpyDeviceToHost, s));
    int32_t *cover_bounce = bounce_out ? reinterpret_cast<int32_t *>(static_cast<uint8_t *>(ws.pinned) + out_at) : nullptr;
    if (cover_out && spec.total_vertices > 0 && !direct_cover)
        VC_CK(cudaMemcpyAsync(cover_bounce ? cover_bounce : cover_out, ws.cover.p, sizeof(int32_t) * spec.total_vertices,
                              cudaMemcpyDeviceToHost, s));
    VC_CK(cudaStreamSynchronize(s));
    if (cover_bounce) std::memcpy(cover_out, cover_bounce, out_bytes);
    if (spec.search) {
        int used = ws.sms;
        for (int i = 0; i < kSmSlots; ++i)
            if (smn[i]) used = std::max(used, i + 1);
        ws.last_sm_nodes.assign(smn, smn + used);
    }

    res.probs.assign(h_probs, h_probs + G);
    res.ctrl = *h_ctrl;
#ifdef VC_DEBUG_CHECKS
    if (h_ctrl->dbg_site) fprintf(stderr, "vc debug check failed: site %d value %d\n", h_ctrl->dbg_site, h_ctrl->dbg_value);
#endif
    res.kernel_ms = 0.f;
    if (spec.search) VC_CK(cudaEventElapsedTime(&res.kernel_ms, ws.ev0, ws.ev1));
    res.workers = workers;
    res.wt = wt;
    res.width = width;
    res.csr_staged = nw == 0 && csr_words > 0;  // bit-row workers stage no CSR
    res.gm = gm;
    res.nw = nw;
    res.eb = eb;
    res.stack_depth = spec.search ? (int)depth : 0;
    return h_ctrl->status;
}

void fill_stats(vc_stats *st, const Result &r, double total_ms, int32_t greedy) {
    if (!st) return;
    std::memset(st, 0, sizeof(*st));
    st->nodes_visited = (int64_t)r.ctrl.nodes;
    st->stack_pushes = (int64_t)r.ctrl.stack_pushes;
    st->stack_pops = (int64_t)r.ctrl.stack_pops;
    st->donations = (int64_t)r.ctrl.donations;
    st->worklist_pops = (int64_t)r.ctrl.worklist_pops;
    st->rule_passes = (int64_t)r.ctrl.rule_passes;
    st->csr_words = (int64_t)r.ctrl.csr_words;
    // every pop, push, donation and dequeue copies one entry
    st->entry_bytes_moved = (int64_t)r.eb * (int64_t)(r.ctrl.stack_pops + r.ctrl.stack_pushes + r.ctrl.donations +
                                                       r.ctrl.worklist_pops);
    for (int i = 0; i < 4; ++i) st->trace_ns[i] = (int64_t)r.ctrl.trace_ns[i];
    st->idle_polls = (int64_t)r.ctrl.idle_polls;
    for (int i = 0; i < 16; ++i) st->trace_cycles[i] = (int64_t)r.ctrl.trace_cycles[i];
    st->max_depth = r.ctrl.max_depth;
    st->greedy_ub = greedy;
    st->workers = r.workers;
    st->worker_threads = r.wt;
    st->width = r.width;
    st->csr_staged = r.csr_staged ? 1 : 0;
    st->node_in_global = r.gm ? 1 : 0;
    st->bit_rows = r.nw;
    st->stack_depth = r.stack_depth;
    st->status = r.ctrl.status;
    st->kernel_ms = r.kernel_ms;
    st->total_ms = (float)total_ms;
}

// Host-side shape checks that need no access to the CSR contents.
int check_graph(const vc_graph *g) {
    if (!g || g->n < 0) return VC_EINVAL;
    if (g->n > 0 && (!g->offsets)) return VC_EINVAL;
    return VC_OK;
}

double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// Builds the one-problem spec of a single-graph call.
int single_spec(const vc_graph *g, int32_t kind, int32_t k, bool search, Spec &spec) {
    spec.probs.push_back(make_problem(0, 0, 0, g->n, kind, k));
    spec.offsets = g->offsets;
    spec.neighbors = g->neighbors;
    spec.on_device = g->on_device ? 1 : 0;
    spec.total_offsets = (int64_t)g->n + 1;
    spec.total_vertices = g->n;
    spec.n_max = g->n;
    spec.search = search;
    if (!g->on_device) {
        const int64_t len = g->offsets[g->n];
        if (len < 0 || (len > 0 && !g->neighbors)) return VC_EINVAL;
        spec.total_adj = len;
        spec.adj_len.push_back(len);
    } else {
        spec.adj_len.push_back(-1);
    }
    return VC_OK;
}

}  // namespace
}  // namespace vc

using namespace vc;

extern "C" {

int vc_version(void) { return 100; }

const char *vc_strerror(int code) {
    switch (code) {
        case VC_OK: return "VC_OK";
        case VC_EINVAL: return "VC_EINVAL";
        case VC_ENOMEM: return "VC_ENOMEM";
        case VC_ETIMEOUT: return "VC_ETIMEOUT";
        case VC_ESTACK: return "VC_ESTACK";
        case VC_ECUDA: return "VC_ECUDA";
        case VC_ECANCELLED: return "VC_ECANCELLED";
        default: return "VC_UNKNOWN";
    }
}

int vc_mvc(const vc_graph *g, const vc_config *cfg, void *stream, int32_t *cover_out, int32_t *cover_size_out,
           vc_stats *stats) {
    const auto t0 = std::chrono::steady_clock::now();
    if (check_graph(g) || !cover_size_out) return VC_EINVAL;
    if (g->n == 0) {
        *cover_size_out = 0;
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return VC_OK;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    Workspace *ws;
    VC_RC(workspace(&ws));
    Spec spec;
    VC_RC(single_spec(g, kMVC, 0, true, spec));
    Result r;
    const int rc = run(*ws, spec, cfg, (cudaStream_t)stream, cover_out, g->on_device, r);
    if (rc != VC_OK) return rc;
    *cover_size_out = r.probs[0].best;
    fill_stats(stats, r, ms_since(t0), r.probs[0].greedy);
    return VC_OK;
}

int vc_pvc(const vc_graph *g, int32_t k, const vc_config *cfg, void *stream, int32_t *found_out,
           int32_t *cover_out, int32_t *cover_size_out, vc_stats *stats) {
    const auto t0 = std::chrono::steady_clock::now();
    if (check_graph(g) || !found_out) return VC_EINVAL;
    if (k < 0 || g->n == 0) {
        *found_out = k >= 0;
        if (cover_size_out) *cover_size_out = k >= 0 ? 0 : -1;
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return VC_OK;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    Workspace *ws;
    VC_RC(workspace(&ws));
    Spec spec;
    VC_RC(single_spec(g, kPVC, k, true, spec));
    Result r;
    const int rc = run(*ws, spec, cfg, (cudaStream_t)stream, cover_out, g->on_device, r);
    if (rc != VC_OK) return rc;
    *found_out = r.probs[0].found ? 1 : 0;
    if (cover_size_out) *cover_size_out = r.probs[0].found ? r.probs[0].cover_size : -1;
    fill_stats(stats, r, ms_since(t0), r.probs[0].greedy);
    return VC_OK;
}

int vc_mvc_batch(int32_t num_graphs, const int32_t *graph_vtx_offsets, const int32_t *graph_edge_offsets,
                 const int32_t *packed_offsets, const int32_t *packed_neighbors, int32_t on_device,
                 const vc_config *cfg, void *stream, int32_t *sizes_out, int32_t *covers_out, vc_stats *stats) {
    const auto t0 = std::chrono::steady_clock::now();
    if (num_graphs < 0 || !sizes_out || (num_graphs > 0 && (!graph_vtx_offsets || !graph_edge_offsets)))
        return VC_EINVAL;
    if (num_graphs == 0) {
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return VC_OK;
    }
    if (graph_vtx_offsets[0] != 0 || graph_edge_offsets[0] != 0) return VC_EINVAL;
    Spec spec;
    spec.offsets = packed_offsets;
    spec.neighbors = packed_neighbors;
    spec.on_device = on_device ? 1 : 0;
    for (int g = 0; g < num_graphs; ++g) {
        const int32_t n = graph_vtx_offsets[g + 1] - graph_vtx_offsets[g];
        const int64_t len = (int64_t)graph_edge_offsets[g + 1] - graph_edge_offsets[g];
        if (n < 0 || len < 0) return VC_EINVAL;
        spec.probs.push_back(make_problem((int64_t)graph_vtx_offsets[g] + g, graph_edge_offsets[g],
                                          graph_vtx_offsets[g], n, kMVC, 0));
        spec.adj_len.push_back(len);
        spec.n_max = std::max(spec.n_max, n);
    }
    spec.total_vertices = graph_vtx_offsets[num_graphs];
    spec.total_offsets = (int64_t)graph_vtx_offsets[num_graphs] + num_graphs;
    spec.total_adj = graph_edge_offsets[num_graphs];
    if (!packed_offsets || (spec.total_adj > 0 && !packed_neighbors)) return VC_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    Workspace *ws;
    VC_RC(workspace(&ws));
    Result r;
    const int rc = run(*ws, spec, cfg, (cudaStream_t)stream, covers_out, on_device, r);
    if (rc != VC_OK) return rc;
    int64_t gsum = 0;
    for (int g = 0; g < num_graphs; ++g) {
        sizes_out[g] = r.probs[g].n == 0 ? 0 : r.probs[g].best;
        gsum += r.probs[g].greedy;
    }
    fill_stats(stats, r, ms_since(t0), (int32_t)std::min<int64_t>(gsum, INT_MAX));
    return VC_OK;
}

int vc_greedy(const vc_graph *g, const vc_config *cfg, void *stream, int32_t *cover_out, int32_t *size_out) {
    if (check_graph(g) || !size_out) return VC_EINVAL;
    if (g->n == 0) {
        *size_out = 0;
        return VC_OK;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    Workspace *ws;
    VC_RC(workspace(&ws));
    Spec spec;
    VC_RC(single_spec(g, kMVC, 0, false, spec));
    Result r;
    const int rc = run(*ws, spec, cfg, (cudaStream_t)stream, cover_out, g->on_device, r);
    if (rc != VC_OK) return rc;
    *size_out = r.probs[0].greedy;
    return VC_OK;
}

int vc_reduce_node(const vc_graph *g, int32_t *deg, int32_t *S, int32_t *m, int32_t problem, int32_t bound,
                   int32_t rules, int32_t branch, const vc_config *cfg, void *stream, int32_t *pruned_out) {
    if (check_graph(g) || !deg || !S || !m || !pruned_out || (problem != kMVC && problem != kPVC) ||
        (rules & ~kRuleAll))
        return VC_EINVAL;
    if (branch >= g->n || (branch <= -2 && -2 - branch >= g->n)) return VC_EINVAL;
    if (g->n == 0) {
        const int64_t t = problem == kMVC ? (int64_t)bound - *S - 1 : (int64_t)bound - *S;
        *pruned_out = (problem == kMVC ? *S >= bound : *S > bound) || (int64_t)*m > t * t;
        return VC_OK;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    Workspace *ws;
    VC_RC(workspace(&ws));
    vc_config c;
    std::memset(&c, 0, sizeof(c));
    if (cfg) c = *cfg;
    const LaunchDefaults tuned = tuned_defaults(g->n);
    const int width = c.width ? c.width : tuned.width;
    if ((width != 16 && width != 32) || (width == 16 && g->n > 32768)) return VC_EINVAL;
    const int wt = c.worker_threads ? c.worker_threads : tuned.worker_threads;
    int smem = smem_bytes_for(g->n, width / 8);
    const bool gm = c.node_in_global > 0 || (c.node_in_global == 0 && smem > ws->smem_optin);
    if (gm) smem = smem_bytes_gm(0);
    if (smem > ws->smem_optin) return VC_EINVAL;
    int nw = (c.bit_rows >= 0 && !gm && wt == 32) ? rows_words_for(g->n) : 0;
    if (c.bit_rows > 0 && nw == 0) return VC_EINVAL;
    if (nw > 0) smem = smem_bytes_for(g->n, width / 8, 0, nw);
    cudaStream_t s = (cudaStream_t)stream;
    StreamDrain drain{s};
    const int64_t len = g->on_device ? -1 : g->offsets[g->n];
    // device copies: graph (if host), degree array, io words
    const size_t deg_bytes = sizeof(int32_t) * (size_t)g->n;
    const size_t io_off = (deg_bytes + 15) & ~size_t(15);
    VC_RC(grow(ws->cover, io_off + 16));
    VC_RC(grow(ws->ctrl, sizeof(Control)));
    const int32_t *d_off = g->offsets, *d_adj = g->neighbors;
    if (!g->on_device) {
        VC_RC(grow(ws->csr_off, sizeof(int32_t) * ((size_t)g->n + 1)));
        VC_RC(grow(ws->csr_adj, sizeof(int32_t) * (size_t)std::max<int64_t>(len, 1)));
        VC_CK(cudaMemcpyAsync(ws->csr_off.p, g->offsets, sizeof(int32_t) * ((size_t)g->n + 1), cudaMemcpyHostToDevice, s));
        if (len > 0) VC_CK(cudaMemcpyAsync(ws->csr_adj.p, g->neighbors, sizeof(int32_t) * len, cudaMemcpyHostToDevice, s));
        d_off = static_cast<const int32_t *>(ws->csr_off.p);
        d_adj = static_cast<const int32_t *>(ws->csr_adj.p);
    }
    // validate the graph first (one problem)
    Spec spec;
    VC_RC(single_spec(g, problem, bound, false, spec));
    VC_RC(grow(ws->problems, sizeof(Problem)));
    VC_RC(grow(ws->adj_len, sizeof(int64_t)));
    VC_RC(grow_pinned(*ws, sizeof(Control) + 64));
    VC_CK(cudaMemcpyAsync(ws->problems.p, spec.probs.data(), sizeof(Problem), cudaMemcpyHostToDevice, s));
    VC_CK(cudaMemcpyAsync(ws->adj_len.p, spec.adj_len.data(), sizeof(int64_t), cudaMemcpyHostToDevice, s));
    VC_CK(cudaMemsetAsync(ws->ctrl.p, 0, sizeof(Control), s));
    if (!c.skip_validation)
        VC_RC(launch_validate(d_off, d_adj, static_cast<const Problem *>(ws->problems.p),
                              static_cast<const int64_t *>(ws->adj_len.p), 1, g->n, static_cast<Control *>(ws->ctrl.p), s));
    Control *h_ctrl = static_cast<Control *>(ws->pinned);
    VC_CK(cudaMemcpyAsync(h_ctrl, ws->ctrl.p, sizeof(Control), cudaMemcpyDeviceToHost, s));
    VC_CK(cudaStreamSynchronize(s));
    if (h_ctrl->status != VC_OK) return h_ctrl->status;

    int32_t *d_deg = static_cast<int32_t *>(ws->cover.p);
    int32_t *d_io = reinterpret_cast<int32_t *>(static_cast<uint8_t *>(ws->cover.p) + io_off);
    int32_t *h_io = reinterpret_cast<int32_t *>(h_ctrl + 1);
    h_io[0] = *S;
    h_io[1] = *m;
    h_io[2] = 0;
    VC_CK(cudaMemcpyAsync(d_deg, deg, deg_bytes, g->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    VC_CK(cudaMemcpyAsync(d_io, h_io, 3 * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    ReduceParams R;
    R.offsets = d_off;
    R.neighbors = d_adj;
    R.n = g->n;
    R.problem = problem;
    R.bound = bound;
    R.rules = rules;
    R.branch = branch;
    R.deg = d_deg;
    R.io = d_io;
    R.gstate = nullptr;
    if (gm) {
        VC_RC(grow(ws->gstate, (size_t)gstate_bytes_for(g->n, width / 8)));
        R.gstate = static_cast<uint8_t *>(ws->gstate.p);
    }
    const Launchers &L = launchers(width, gm, nw);
    VC_RC(L.reduce(wt, smem, s, R));
    VC_CK(cudaMemcpyAsync(deg, d_deg, deg_bytes, g->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    VC_CK(cudaMemcpyAsync(h_io, d_io, 3 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    VC_CK(cudaStreamSynchronize(s));
    *S = h_io[0];
    *m = h_io[1];
    *pruned_out = h_io[2];
    return VC_OK;
}

int vc_last_sm_nodes(int64_t *counts_out, int32_t capacity) {
    if (!counts_out || capacity < 0) return VC_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    Workspace *ws;
    VC_RC(workspace(&ws));
    const int n = std::min<int>(capacity, (int)ws->last_sm_nodes.size());
    for (int i = 0; i < n; ++i) counts_out[i] = ws->last_sm_nodes[i];
    return (int)ws->last_sm_nodes.size();
}

int vc_release(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return VC_ECUDA;
    }
    if (dev >= 0 && dev < kMaxDevices) free_workspace(g_ws[dev]);
    return VC_OK;
}

}  // extern "C"
