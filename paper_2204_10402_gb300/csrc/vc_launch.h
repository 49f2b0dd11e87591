// vc_launch.h - host-side entry points into the templated kernels, one set per degree-array
// width and node placement (vc_kern_w16.cu, vc_kern_w32.cu: node in shared memory;
// vc_kern_w16_gm.cu, vc_kern_w32_gm.cu: node in global memory; vc_kern_w16_rows.cu,
// vc_kern_w32_rows.cu: bit-row workers for graphs of at most 256 vertices).
#pragma once

#include <cuda_runtime.h>

#include "vc_internal.h"

namespace vc {

struct Launchers {
    int (*greedy)(int wt, int grid, int smem, cudaStream_t s, const Params &P);
    int (*traverse)(int wt, int grid, int smem, cudaStream_t s, const Params &P);
    int (*reduce)(int wt, int smem, cudaStream_t s, const ReduceParams &R);
    // Resident blocks per SM of the traversal kernel at this worker size and shared memory.
    int (*occupancy)(int wt, int smem, int *blocks_per_sm);
    // The same for the serving instance, which this also loads and configures (so that its first
    // launch loads no code while another persistent launch is running).
    int (*serve_prepare)(int wt, int smem, int *blocks_per_sm);
};

const Launchers &launchers_w16();
const Launchers &launchers_w32();
const Launchers &launchers_w16_gm();
const Launchers &launchers_w32_gm();
const Launchers &launchers_w16_rows(int nw);  // nw = 1, 2, 4 or 8; one-warp workers only
const Launchers &launchers_w32_rows(int nw);
inline const Launchers &launchers(int width, bool gm, int nw = 0) {
    if (nw > 0) return width == 16 ? launchers_w16_rows(nw) : launchers_w32_rows(nw);
    if (gm) return width == 16 ? launchers_w16_gm() : launchers_w32_gm();
    return width == 16 ? launchers_w16() : launchers_w32();
}

// Non-templated kernels (vc_common.cu).
int launch_validate(const int32_t *offsets, const int32_t *neighbors, const Problem *probs,
                    const int64_t *adj_len, int32_t num_problems, int64_t total_vertices, Control *ctrl,
                    cudaStream_t s);
int launch_init_worklist(uint32_t *seq, int32_t capacity, Control *ctrl, cudaStream_t s,
                         unsigned long long *claim_state = nullptr);

}  // namespace vc
