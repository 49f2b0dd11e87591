// vc_launch_impl.cuh - instantiates the kernels of one degree-array width W, one node placement
// (GM: shared or global memory) and one bit-row size (NW: 0 = CSR walks, else words per row) for
// every supported worker size, behind a Launchers table.
#pragma once

#include "vc_kernels.cuh"
#include "vc_launch.h"

namespace vc {

template <typename Kernel>
static int prepare(Kernel k, int smem) {
    if (smem > 48 * 1024) {
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
            return VC_ECUDA;
    }
    return VC_OK;
}

// The server's launches (one per size class) run side by side on the same SMs.  An SM changes its
// shared-memory / L1 split only while idle, so both instances ask for the same split -- all of the
// configurable memory as shared memory -- and the blocks of one never wait for the other's to leave
// an SM that was configured with a smaller shared-memory share.
template <typename Kernel>
static int prepare_serving(Kernel k, int smem) {
    if (int rc = prepare(k, smem)) return rc;
    if (cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
        cudaSuccess)
        return VC_ECUDA;
    return VC_OK;
}

static inline int launch_status() { return cudaPeekAtLastError() == cudaSuccess ? VC_OK : VC_ECUDA; }

// Runs the statement with constexpr WT bound to the worker size; bit-row kernels exist for
// one-warp workers only.
#define VC_WT_SWITCH(wt, ...)                                          \
    if constexpr (NW > 0) {                                            \
        if ((wt) != 32) return VC_EINVAL;                              \
        { constexpr int WT = 32; __VA_ARGS__; }                        \
    } else {                                                           \
        switch (wt) {                                                  \
            case 32: { constexpr int WT = 32; __VA_ARGS__; } break;    \
            case 64: { constexpr int WT = 64; __VA_ARGS__; } break;    \
            case 128: { constexpr int WT = 128; __VA_ARGS__; } break;  \
            case 256: { constexpr int WT = 256; __VA_ARGS__; } break;  \
            case 512: { constexpr int WT = 512; __VA_ARGS__; } break;  \
            default: return VC_EINVAL;                                 \
        }                                                              \
    }

template <typename W, bool GM, int NW>
struct LaunchImpl {
    static int greedy(int wt, int grid, int smem, cudaStream_t s, const Params &P) {
        VC_WT_SWITCH(wt, {
            if (int rc = prepare(greedy_kernel<W, WT, GM, NW>, smem)) return rc;
            greedy_kernel<W, WT, GM, NW><<<grid, WT, smem, s>>>(P);
        });
        return launch_status();
    }
    static int traverse(int wt, int grid, int smem, cudaStream_t s, const Params &P) {
        if (P.serving) {  // the server's launches: CSR walks, or 4-word bit rows (graphs of <= 128 vertices)
            if constexpr (GM || (NW != 0 && NW != 4)) {
                return VC_EINVAL;
            } else {
                VC_WT_SWITCH(wt, {
                    if (int rc = prepare_serving(traverse_kernel<W, WT, GM, NW, true>, smem)) return rc;
                    traverse_kernel<W, WT, GM, NW, true><<<grid, WT, smem, s>>>(P);
                });
                return launch_status();
            }
        }
        VC_WT_SWITCH(wt, {
            if (int rc = prepare(traverse_kernel<W, WT, GM, NW, false>, smem)) return rc;
            traverse_kernel<W, WT, GM, NW, false><<<grid, WT, smem, s>>>(P);
        });
        return launch_status();
    }
    static int reduce(int wt, int smem, cudaStream_t s, const ReduceParams &R) {
        VC_WT_SWITCH(wt, {
            if (int rc = prepare(reduce_node_kernel<W, WT, GM, NW>, smem)) return rc;
            reduce_node_kernel<W, WT, GM, NW><<<1, WT, smem, s>>>(R);
        });
        return launch_status();
    }
    static int occupancy(int wt, int smem, int *blocks) {
        VC_WT_SWITCH(wt, {
            if (int rc = prepare(traverse_kernel<W, WT, GM, NW, false>, smem)) return rc;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, traverse_kernel<W, WT, GM, NW, false>, WT, smem) !=
                cudaSuccess)
                return VC_ECUDA;
        });
        return VC_OK;
    }
    static int serve_prepare(int wt, int smem, int *blocks) {
        if constexpr (GM || (NW != 0 && NW != 4)) {
            return VC_EINVAL;
        } else {
            VC_WT_SWITCH(wt, {
                if (int rc = prepare_serving(traverse_kernel<W, WT, GM, NW, true>, smem)) return rc;
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, traverse_kernel<W, WT, GM, NW, true>, WT, smem) !=
                    cudaSuccess)
                    return VC_ECUDA;
            });
            return VC_OK;
        }
    }
    static const Launchers &table() {
        static const Launchers L = {&greedy, &traverse, &reduce, &occupancy, &serve_prepare};
        return L;
    }
};

}  // namespace vc
