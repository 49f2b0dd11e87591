// vc_noalloc.cu - vc_mvc_noalloc: minimum vertex cover of one small device-resident graph without
// any memory allocation by the library.
//
// Some callers cannot let a library allocate: code running under a memory pool or arena that owns
// all device memory, processes whose allocator is locked after start-up, or deployments that
// forbid allocation (and the implicit synchronisation of cudaMalloc/cudaFree) on the request path.
// This entry point serves them: every scratch byte the search needs (control block, problem
// record, cover mask, local stacks, worklist) lives in one file-scope __device__ array of fixed
// size that is part of the loaded library image, so the call itself allocates nothing.
//
// The array is reached from host code only through its device address, which cudaGetSymbolAddress
// returns; the first call on each device looks that address up (with the device current) and
// caches it.  Every call reuses the same array: the parts that must start at zero or at a known
// value are reset at the start of each call, and two calls whose work overlaps on the GPU (for
// example from two streams or two host threads without ordering) would corrupt each other.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>

#include "vc_internal.h"
#include "vc_tuning.h"
#include "vc_launch.h"

namespace vc {
namespace {

constexpr int kNoAllocMaxN = VC_NOALLOC_MAX_N;
constexpr size_t kNoAllocBytes = VC_NOALLOC_SCRATCH_BYTES;
constexpr int kNoAllocWorklist = 1024;  // worklist entries (a power of two)
constexpr int kMaxDevs = 64;

// The scratch array: one copy per device that loads the library, held until the process exits.
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
uint8_t *g_scratch_addr[kMaxDevs] = {};
int g_sms[kMaxDevs] = {};

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

// Looks up the device address of the scratch array for the current device (once per device).
int scratch_for_current_device(uint8_t **addr, int *sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return VC_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevs) return VC_EINVAL;
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return VC_ECUDA;
        }
        int count = 0;
        if (cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return VC_ECUDA;
        }
        g_scratch_addr[dev] = static_cast<uint8_t *>(p);
        g_sms[dev] = count;
    }
    *addr = g_scratch_addr[dev];
    *sms = g_sms[dev];
    return VC_OK;
}

}  // namespace
}  // namespace vc

using namespace vc;

extern "C" int vc_mvc_noalloc(const vc_graph *g, const vc_config *cfg_in, void *stream, int32_t *cover_out,
                              int32_t *cover_size_out, vc_stats *stats) {
    if (!g || !cover_size_out || g->n < 0 || !g->on_device) return VC_EINVAL;
    if (g->n > kNoAllocMaxN) return VC_EINVAL;  // larger than the fixed scratch array supports
    if (g->n > 0 && (!g->offsets || !g->neighbors)) return VC_EINVAL;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (g->n == 0) {
        *cover_size_out = 0;
        return VC_OK;
    }
    vc_config cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    if (cfg_in) cfg = *cfg_in;
    // Settings this entry point cannot honour are errors, not silently replaced: the node stays in
    // shared memory, entries are 16-bit, the workers walk the CSR with at most its offsets staged,
    // and the worklist is the array's fixed ring.
    if (cfg.node_in_global > 0 || (cfg.width != 0 && cfg.width != 16) || cfg.bit_rows > 0 || cfg.stage_csr > 0 ||
        (cfg.worklist_capacity != 0 && cfg.worklist_capacity != kNoAllocWorklist))
        return VC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;

    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    // Every return, error paths included, waits for this call's GPU work before the lock is
    // released (declared after the lock, so it runs first): the next call never overlaps it.
    struct DrainOnExit {
        cudaStream_t s;
        ~DrainOnExit() {
            if (cudaStreamSynchronize(s) != cudaSuccess) cudaGetLastError();
        }
    } drain{s};
    uint8_t *base = nullptr;
    int sms = 0;
    if (int rc = scratch_for_current_device(&base, &sms)) return rc;

    // ---- variant (16-bit degree arrays; n <= 512 always fits) ----
    const int n = g->n;
    const int wt = cfg.worker_threads ? cfg.worker_threads : tuned_defaults(n).worker_threads;
    const int wbytes = 2;
    const int32_t csr_words = default_csr_words(n, cfg.stage_csr);
    const int smem = smem_bytes_for(n, wbytes, csr_words);
    const Launchers &L = launchers_w16();
    int per_sm = 0;
    if (int rc = L.occupancy(wt, smem, &per_sm)) return rc;
    if (per_sm <= 0) return VC_EINVAL;
    const int32_t eb = entry_bytes_for(n, wbytes);

    // ---- carve the scratch array ----
    size_t off = 0;
    Control *d_ctrl = reinterpret_cast<Control *>(base + off);
    off += up256(sizeof(Control));
    Problem *d_prob = reinterpret_cast<Problem *>(base + off);
    off += up256(sizeof(Problem));
    int64_t *d_adj_len = reinterpret_cast<int64_t *>(base + off);
    off += up256(sizeof(int64_t));
    int32_t *d_cover = reinterpret_cast<int32_t *>(base + off);
    off += up256(sizeof(int32_t) * (size_t)kNoAllocMaxN);
    unsigned long long *d_sm = reinterpret_cast<unsigned long long *>(base + off);
    off += up256(sizeof(unsigned long long) * (size_t)kSmSlots);
    uint32_t *d_seq = reinterpret_cast<uint32_t *>(base + off);
    off += up256(sizeof(uint32_t) * (size_t)kNoAllocWorklist);
    uint8_t *d_slots = base + off;
    off += up256((size_t)kNoAllocWorklist * (size_t)eb);
    uint8_t *d_stacks = base + off;
    const size_t stack_bytes = kNoAllocBytes - off;

    // ---- problem record (host copy on the stack: no allocation) ----
    Problem h_prob;
    std::memset(&h_prob, 0, sizeof(h_prob));
    h_prob.n = n;
    h_prob.kind = kMVC;
    h_prob.best = INT_MAX;
    h_prob.cover_size = INT_MAX;
    const int64_t h_adj_len = -1;  // the CSR length is read on the device
    if (cudaMemsetAsync(d_ctrl, 0, sizeof(Control), s) != cudaSuccess ||
        cudaMemcpyAsync(d_prob, &h_prob, sizeof(Problem), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(d_adj_len, &h_adj_len, sizeof(int64_t), cudaMemcpyHostToDevice, s) != cudaSuccess) {
        cudaGetLastError();
        return VC_ECUDA;
    }

    Params P;
    std::memset(&P, 0, sizeof(P));
    P.offsets = g->offsets;
    P.neighbors = g->neighbors;
    P.problems = d_prob;
    P.num_problems = 1;
    P.n_max = n;
    P.entry_bytes = eb;
    P.ctrl = d_ctrl;
    P.cover = d_cover;
    P.wl_capacity = kNoAllocWorklist;
    // Donation threshold as in vc_mvc: a fraction of the ring (0: one half), negative = never donate.
    const float frac = cfg.donate_threshold > 0.f ? std::min(cfg.donate_threshold, 1.f) : 0.5f;
    P.wl_threshold = cfg.donate_threshold < 0.f ? 0 : std::max(1, (int)(frac * (float)kNoAllocWorklist));
    P.csr_words = csr_words;
    P.idle_timeout_ns = cfg.idle_timeout_ns > 0 ? cfg.idle_timeout_ns : 20000000000ll;
    P.cancel = cfg.cancel;
    P.sm_nodes = d_sm;

    if (!cfg.skip_validation) {
        if (int rc = launch_validate(g->offsets, g->neighbors, d_prob, d_adj_len, 1, n, d_ctrl, s)) return rc;
    }
    if (int rc = L.greedy(wt, 1, smem, s, P)) return rc;

    // The greedy bound caps the stack depth (every branch adds a vertex to S below best).
    Problem h_after;
    int32_t status = VC_OK;
    if (cudaMemcpyAsync(&h_after, d_prob, sizeof(Problem), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&status, &d_ctrl->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return VC_ECUDA;
    }
    if (status != VC_OK) return status;
    const int64_t depth = (int64_t)h_after.greedy + 2;
    const size_t per_worker = (size_t)depth * (size_t)eb;
    int64_t workers = cfg.num_workers > 0 ? cfg.num_workers : (int64_t)sms * per_sm;
    workers = std::min<int64_t>(workers, (int64_t)(stack_bytes / per_worker));
    if (workers < 1) return VC_EINVAL;
    P.stack_depth = (int32_t)depth;
    P.stacks = d_stacks;
    P.wl_slots = d_slots;
    P.wl_seq = d_seq;

    if (int rc = launch_init_worklist(d_seq, kNoAllocWorklist, d_ctrl, s)) return rc;
    if (cudaMemsetAsync(d_sm, 0, sizeof(unsigned long long) * (size_t)kSmSlots, s) != cudaSuccess) {
        cudaGetLastError();
        return VC_ECUDA;
    }
    if (int rc = L.traverse(wt, (int)workers, smem, s, P)) return rc;

    Control h_ctrl;
    Problem h_res;
    if (cudaMemcpyAsync(&h_ctrl, d_ctrl, sizeof(Control), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&h_res, d_prob, sizeof(Problem), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        (cover_out && cudaMemcpyAsync(cover_out, d_cover, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice,
                                      s) != cudaSuccess) ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return VC_ECUDA;
    }
    if (h_ctrl.status != VC_OK) return h_ctrl.status;
    *cover_size_out = h_res.best;
    if (stats) {
        stats->nodes_visited = (int64_t)h_ctrl.nodes;
        stats->stack_pushes = (int64_t)h_ctrl.stack_pushes;
        stats->stack_pops = (int64_t)h_ctrl.stack_pops;
        stats->donations = (int64_t)h_ctrl.donations;
        stats->worklist_pops = (int64_t)h_ctrl.worklist_pops;
        stats->rule_passes = (int64_t)h_ctrl.rule_passes;
        stats->csr_words = (int64_t)h_ctrl.csr_words;
        stats->entry_bytes_moved = (int64_t)eb * (int64_t)(h_ctrl.stack_pops + h_ctrl.stack_pushes + h_ctrl.donations +
                                                            h_ctrl.worklist_pops);
        stats->max_depth = h_ctrl.max_depth;
        stats->greedy_ub = h_res.greedy;
        stats->workers = (int32_t)workers;
        stats->worker_threads = wt;
        stats->width = 16;
        stats->csr_staged = csr_words > 0 ? 1 : 0;
        stats->stack_depth = (int32_t)depth;
        stats->status = h_ctrl.status;
    }
    return VC_OK;
}
