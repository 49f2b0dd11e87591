// vc_plan.cu - batched MVC as a reusable plan whose whole launch sequence is one CUDA graph
// (include/vc_plan.h).
//
// Creating a plan copies the packed graphs into plan-owned device memory, checks them once, picks
// the launch variant, allocates stacks / worklist / counters, and captures
//   problem-table reset -> control reset -> worklist init -> greedy -> traversal -> gather answers
// into a CUDA graph.  vc_plan_launch replays that graph on any stream without a host
// synchronisation, so a step of many thousand graphs is a single graph launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "vc_internal.h"
#include "vc_tuning.h"
#include "vc_launch.h"
#include "../../include/vc_plan.h"

namespace vc {
namespace {

__global__ void gather_sizes_kernel(const Problem *probs, int32_t num, int32_t *sizes) {
    const int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < num) sizes[g] = probs[g].n == 0 ? 0 : probs[g].best;
}

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace
}  // namespace vc

using namespace vc;

struct vc_plan {
    int32_t G = 0;
    int64_t total_vertices = 0;
    int width = 16, wt = 32, smem = 0, workers = 0, eb = 0, cap = 0, nw = 0;
    void *mem = nullptr;
    Problem *pristine = nullptr, *probs = nullptr;
    Control *ctrl = nullptr;
    int32_t *sizes = nullptr, *cover = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int64_t greedy_sum = 0;
};

extern "C" {

int vc_plan_create_mvc_batch(int32_t G, const int32_t *vtx, const int32_t *edge, const int32_t *packed_offsets,
                             const int32_t *packed_neighbors, int32_t on_device, const vc_config *cfg_in,
                             vc_plan **out) {
    if (!out || G <= 0 || !vtx || !edge || !packed_offsets || vtx[0] != 0 || edge[0] != 0) return VC_EINVAL;
    *out = nullptr;
    vc_config cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    if (cfg_in) cfg = *cfg_in;
    if (cfg.node_in_global > 0) return VC_EINVAL;  // plans keep the node in shared memory
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return VC_ECUDA;

    // ---- problems ----
    std::vector<Problem> probs(G);
    std::vector<int64_t> adj_len(G);
    int32_t n_max = 1;
    for (int g = 0; g < G; ++g) {
        const int32_t n = vtx[g + 1] - vtx[g];
        const int64_t len = (int64_t)edge[g + 1] - edge[g];
        if (n < 0 || len < 0) return VC_EINVAL;
        Problem &p = probs[g];
        std::memset(&p, 0, sizeof(p));
        p.off_base = (int64_t)vtx[g] + g;
        p.adj_base = edge[g];
        p.cover_base = vtx[g];
        p.n = n;
        p.kind = kMVC;
        p.best = INT_MAX;
        p.cover_size = INT_MAX;
        adj_len[g] = len;
        n_max = std::max(n_max, n);
    }
    const int64_t total_off = (int64_t)vtx[G] + G, total_adj = edge[G], total_v = vtx[G];
    if (total_adj > 0 && !packed_neighbors) return VC_EINVAL;

    // ---- variant (as for vc_mvc_batch) ----
    vc_plan *pl = new vc_plan();
    pl->G = G;
    pl->total_vertices = total_v;
    const LaunchDefaults tuned = tuned_defaults(n_max);
    pl->width = cfg.width ? cfg.width : tuned.width;
    if ((pl->width != 16 && pl->width != 32) || (pl->width == 16 && n_max > 32768)) {
        delete pl;
        return VC_EINVAL;
    }
    pl->wt = cfg.worker_threads ? cfg.worker_threads : tuned.worker_threads;
    const int32_t csr_words = default_csr_words(n_max, cfg.stage_csr);
    pl->smem = smem_bytes_for(n_max, pl->width / 8, csr_words);
    // Bit-row workers as in vc_mvc_batch: one warp per worker and n_max <= 256.
    pl->nw = (cfg.bit_rows >= 0 && pl->wt == 32) ? rows_words_for(n_max) : 0;
    if (cfg.bit_rows > 0 && pl->nw == 0) {
        delete pl;
        return VC_EINVAL;
    }
    if (pl->nw > 0) pl->smem = smem_bytes_for(n_max, pl->width / 8, csr_words, pl->nw);
    const Launchers &L = launchers(pl->width, false, pl->nw);
    int per_sm = 0;
    if (pl->smem > (int)prop.sharedMemPerBlockOptin || L.occupancy(pl->wt, pl->smem, &per_sm) != VC_OK || per_sm <= 0) {
        delete pl;
        return VC_EINVAL;
    }
    pl->workers = cfg.num_workers > 0 ? cfg.num_workers : prop.multiProcessorCount * per_sm;
    pl->eb = entry_bytes_for(n_max, pl->width / 8);
    int cap = 1;
    if (cfg.worklist_capacity > 0)
        while (cap < cfg.worklist_capacity) cap <<= 1;
    else
        cap = default_worklist_capacity(pl->eb, tuned.capacity);
    pl->cap = cap;
    const float frac = cfg.donate_threshold > 0.f ? cfg.donate_threshold : tuned.threshold;
    const int threshold = cfg.donate_threshold < 0.f ? 0 : std::max(0, std::min(cap, (int)(frac * cap)));
    const int64_t depth = (int64_t)n_max + 2;

    // ---- one allocation ----
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t at = off;
        off += up256(std::max<size_t>(b, 16));
        return at;
    };
    const size_t o_off = take(sizeof(int32_t) * total_off);
    const size_t o_adj = take(sizeof(int32_t) * std::max<int64_t>(total_adj, 1));
    const size_t o_pris = take(sizeof(Problem) * G);
    const size_t o_prob = take(sizeof(Problem) * G);
    const size_t o_len = take(sizeof(int64_t) * G);
    const size_t o_ctrl = take(sizeof(Control));
    const size_t o_sizes = take(sizeof(int32_t) * G);
    const size_t o_cover = take(sizeof(int32_t) * std::max<int64_t>(total_v, 1));
    const size_t o_smn = take(sizeof(unsigned long long) * kSmSlots);
    const size_t o_seq = take(sizeof(uint32_t) * cap);
    const size_t o_wl = take((size_t)cap * pl->eb);
    const size_t o_stk = take((size_t)pl->workers * (size_t)depth * pl->eb);
    const size_t o_rows = take(sizeof(uint32_t) * (size_t)pl->nw * (size_t)std::max<int64_t>(total_v, 1));
    const size_t o_roots = take((size_t)G * pl->eb);  // each problem's root node, kept by the greedy pass
    for (int g = 0; g < G; ++g) probs[g].root_base = (int64_t)g * pl->eb;
    if (cudaMalloc(&pl->mem, off) != cudaSuccess) {
        cudaGetLastError();
        delete pl;
        return VC_ENOMEM;
    }
    uint8_t *b = static_cast<uint8_t *>(pl->mem);
    int32_t *d_off = reinterpret_cast<int32_t *>(b + o_off);
    int32_t *d_adj = reinterpret_cast<int32_t *>(b + o_adj);
    pl->pristine = reinterpret_cast<Problem *>(b + o_pris);
    pl->probs = reinterpret_cast<Problem *>(b + o_prob);
    int64_t *d_len = reinterpret_cast<int64_t *>(b + o_len);
    pl->ctrl = reinterpret_cast<Control *>(b + o_ctrl);
    pl->sizes = reinterpret_cast<int32_t *>(b + o_sizes);
    pl->cover = reinterpret_cast<int32_t *>(b + o_cover);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaStream_t cs = nullptr;
    int rc = VC_OK;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMemcpyAsync(d_off, packed_offsets, sizeof(int32_t) * total_off, kind, cs) != cudaSuccess ||
        (total_adj > 0 && cudaMemcpyAsync(d_adj, packed_neighbors, sizeof(int32_t) * total_adj, kind, cs) != cudaSuccess) ||
        cudaMemcpyAsync(pl->pristine, probs.data(), sizeof(Problem) * G, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
        cudaMemcpyAsync(d_len, adj_len.data(), sizeof(int64_t) * G, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
        cudaMemsetAsync(pl->ctrl, 0, sizeof(Control), cs) != cudaSuccess)
        rc = VC_ECUDA;
    // ---- check the graphs once ----
    if (rc == VC_OK && !cfg.skip_validation) rc = launch_validate(d_off, d_adj, pl->pristine, d_len, G, total_v, pl->ctrl, cs);
    int32_t status = VC_OK;
    if (rc == VC_OK && (cudaMemcpyAsync(&status, &pl->ctrl->status, sizeof(int32_t), cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
                        cudaStreamSynchronize(cs) != cudaSuccess))
        rc = VC_ECUDA;
    if (rc == VC_OK && status != VC_OK) rc = status;

    // ---- capture the launch sequence ----
    Params P;
    std::memset(&P, 0, sizeof(P));
    P.offsets = d_off;
    P.neighbors = d_adj;
    P.problems = pl->probs;
    P.num_problems = G;
    P.n_max = n_max;
    P.entry_bytes = pl->eb;
    P.stack_depth = (int32_t)depth;
    P.ctrl = pl->ctrl;
    P.cover = pl->cover;
    P.stacks = b + o_stk;
    P.wl_slots = b + o_wl;
    P.wl_seq = reinterpret_cast<uint32_t *>(b + o_seq);
    P.wl_capacity = cap;
    P.wl_threshold = threshold;
    P.csr_words = csr_words;
    P.idle_timeout_ns = cfg.idle_timeout_ns > 0 ? cfg.idle_timeout_ns : 20000000000ll;
    P.cancel = cfg.cancel;
    P.sm_nodes = reinterpret_cast<unsigned long long *>(b + o_smn);
    P.rows = pl->nw > 0 ? reinterpret_cast<uint32_t *>(b + o_rows) : nullptr;
    P.roots = b + o_roots;
    if (rc == VC_OK && (cudaEventCreate(&pl->ev0) != cudaSuccess || cudaEventCreate(&pl->ev1) != cudaSuccess)) rc = VC_ECUDA;
    if (rc == VC_OK && cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = VC_ECUDA;
    if (rc == VC_OK) {
        int r2 = VC_OK;
        if (cudaMemcpyAsync(pl->probs, pl->pristine, sizeof(Problem) * G, cudaMemcpyDeviceToDevice, cs) != cudaSuccess ||
            cudaMemsetAsync(pl->ctrl, 0, sizeof(Control), cs) != cudaSuccess ||
            cudaMemsetAsync(P.sm_nodes, 0, sizeof(unsigned long long) * kSmSlots, cs) != cudaSuccess)
            r2 = VC_ECUDA;
        if (r2 == VC_OK) r2 = launch_init_worklist(P.wl_seq, cap, pl->ctrl, cs);
        if (r2 == VC_OK) r2 = L.greedy(pl->wt, std::min(G, pl->workers), pl->smem, cs, P);
        if (r2 == VC_OK && cudaEventRecordWithFlags(pl->ev0, cs, cudaEventRecordExternal) != cudaSuccess) r2 = VC_ECUDA;
        if (r2 == VC_OK) r2 = L.traverse(pl->wt, pl->workers, pl->smem, cs, P);
        if (r2 == VC_OK && cudaEventRecordWithFlags(pl->ev1, cs, cudaEventRecordExternal) != cudaSuccess) r2 = VC_ECUDA;
        if (r2 == VC_OK) {
            gather_sizes_kernel<<<(G + 255) / 256, 256, 0, cs>>>(pl->probs, G, pl->sizes);
            if (cudaPeekAtLastError() != cudaSuccess) r2 = VC_ECUDA;
        }
        const cudaError_t e = cudaStreamEndCapture(cs, &pl->graph);
        if (r2 == VC_OK && e != cudaSuccess) r2 = VC_ECUDA;
        if (r2 == VC_OK && cudaGraphInstantiate(&pl->exec, pl->graph, 0) != cudaSuccess) r2 = VC_ECUDA;
        rc = r2;
    }
    if (cs) cudaStreamDestroy(cs);
    if (rc != VC_OK) {
        cudaGetLastError();
        vc_plan_destroy(pl);
        return rc;
    }
    *out = pl;
    return VC_OK;
}

int vc_plan_launch(vc_plan *pl, void *stream) {
    if (!pl || !pl->exec) return VC_EINVAL;
    return cudaGraphLaunch(pl->exec, (cudaStream_t)stream) == cudaSuccess ? VC_OK : VC_ECUDA;
}

int vc_plan_results(vc_plan *pl, void *stream, int32_t *sizes_out, int32_t *covers_out, int32_t covers_on_device,
                    vc_stats *stats) {
    if (!pl || !sizes_out) return VC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Control c;
    if (cudaMemcpyAsync(sizes_out, pl->sizes, sizeof(int32_t) * pl->G, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&c, pl->ctrl, sizeof(Control), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        (covers_out && cudaMemcpyAsync(covers_out, pl->cover, sizeof(int32_t) * pl->total_vertices,
                                       covers_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return VC_ECUDA;
    }
    if (c.status != VC_OK) return c.status;
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->nodes_visited = (int64_t)c.nodes;
        stats->stack_pushes = (int64_t)c.stack_pushes;
        stats->stack_pops = (int64_t)c.stack_pops;
        stats->donations = (int64_t)c.donations;
        stats->worklist_pops = (int64_t)c.worklist_pops;
        stats->rule_passes = (int64_t)c.rule_passes;
        stats->csr_words = (int64_t)c.csr_words;
        stats->entry_bytes_moved = (int64_t)pl->eb * (int64_t)(c.stack_pops + c.stack_pushes + c.donations + c.worklist_pops);
        for (int i = 0; i < 4; ++i) stats->trace_ns[i] = (int64_t)c.trace_ns[i];
        stats->idle_polls = (int64_t)c.idle_polls;
        for (int i = 0; i < 16; ++i) stats->trace_cycles[i] = (int64_t)c.trace_cycles[i];
        stats->max_depth = c.max_depth;
        stats->workers = pl->workers;
        stats->worker_threads = pl->wt;
        stats->width = pl->width;
        stats->bit_rows = pl->nw;
        stats->status = c.status;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pl->ev0, pl->ev1) == cudaSuccess) stats->kernel_ms = ms;
        else cudaGetLastError();
    }
    return VC_OK;
}

int vc_plan_completion_ns(vc_plan *pl, void *stream, int64_t *done_ns_out) {
    if (!pl || !done_ns_out) return VC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<Problem> probs((size_t)pl->G);
    Control c;
    if (cudaMemcpyAsync(probs.data(), pl->probs, sizeof(Problem) * (size_t)pl->G, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&c, pl->ctrl, sizeof(Control), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return VC_ECUDA;
    }
    if (c.status != VC_OK) return c.status;
    for (int32_t g = 0; g < pl->G; ++g) {
        const int64_t t = probs[(size_t)g].t_done_ns;
        done_ns_out[g] = t > 0 && (uint64_t)t >= c.t_launch_ns ? t - (int64_t)c.t_launch_ns : 0;
    }
    return VC_OK;
}

int vc_plan_destroy(vc_plan *pl) {
    if (!pl) return VC_EINVAL;
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->ev0) cudaEventDestroy(pl->ev0);
    if (pl->ev1) cudaEventDestroy(pl->ev1);
    if (pl->mem) cudaFree(pl->mem);
    delete pl;
    return VC_OK;
}

}  // extern "C"
