// vc_common.cu - kernels that do not depend on the degree-array width: CSR validation and
// worklist initialisation.
#include "vc_kernels.cuh"
#include "vc_launch.h"

namespace vc {

// Binary search for `key` in the sorted list a[lo, hi).
__device__ __forceinline__ bool sorted_contains(const int32_t *a, int32_t lo, int32_t hi, int32_t key) {
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        const int32_t x = __ldg(a + mid);
        if (x == key) return true;
        if (x < key) lo = mid + 1;
        else hi = mid;
    }
    return false;
}

__global__ void validate_kernel(const int32_t *offsets, const int32_t *neighbors, const Problem *probs,
                                const int64_t *adj_len, int32_t num_problems, int64_t total_vertices,
                                Control *ctrl) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t gv = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gv < total_vertices; gv += stride) {
        // The problem owning global vertex gv: the last one whose first vertex is <= gv.
        int lo = 0, hi = num_problems - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (probs[mid].cover_base <= gv) lo = mid;
            else hi = mid - 1;
        }
        const Problem &pr = probs[lo];
        const int32_t n = pr.n;
        const int32_t v = (int32_t)(gv - pr.cover_base);
        const int32_t *off = offsets + pr.off_base;
        const int32_t *adj = neighbors + pr.adj_base;
        const int32_t end = __ldg(off + n);
        const int32_t b = __ldg(off + v), e = __ldg(off + v + 1);
        // With a known neighbour count (host inputs, batches) nothing past it is ever read.
        const bool known = adj_len && adj_len[lo] >= 0;
        bool bad = b < 0 || b > e || e > end || (end & 1) || (v == 0 && b != 0) ||
                   (known && (int64_t)end != adj_len[lo]);
        for (int32_t j = b; !bad && j < e; ++j) {
            const int32_t x = __ldg(adj + j);
            if (x < 0 || x >= n || x == v || (j > b && __ldg(adj + j - 1) >= x)) {
                bad = true;
                break;
            }
            const int32_t xb = __ldg(off + x), xe = __ldg(off + x + 1);
            if (xb < 0 || xb > xe || xe > end || !sorted_contains(adj, xb, xe, v)) bad = true;
        }
        if (bad) raise_status(ctrl, VC_EINVAL);
    }
}

__global__ void init_worklist_kernel(uint32_t *seq, int32_t capacity, Control *ctrl,
                                     unsigned long long *claim_state) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < capacity) seq[i] = (uint32_t)i;
    if (i == 0) {
        ctrl->wl_space = capacity;
        if (claim_state) *claim_state &= 0xffffffffull;  // a new serving launch is open again
    }
}

int launch_validate(const int32_t *offsets, const int32_t *neighbors, const Problem *probs,
                    const int64_t *adj_len, int32_t num_problems, int64_t total_vertices, Control *ctrl,
                    cudaStream_t s) {
    if (total_vertices <= 0) return VC_OK;
    const int threads = 256;
    const int64_t want = (total_vertices + threads - 1) / threads;
    const int blocks = (int)(want < 4096 ? want : 4096);
    validate_kernel<<<blocks, threads, 0, s>>>(offsets, neighbors, probs, adj_len, num_problems,
                                               total_vertices, ctrl);
    return cudaPeekAtLastError() == cudaSuccess ? VC_OK : VC_ECUDA;
}

int launch_init_worklist(uint32_t *seq, int32_t capacity, Control *ctrl, cudaStream_t s,
                         unsigned long long *claim_state) {
    init_worklist_kernel<<<(capacity + 255) / 256, 256, 0, s>>>(seq, capacity, ctrl, claim_state);
    return cudaPeekAtLastError() == cudaSuccess ? VC_OK : VC_ECUDA;
}

}  // namespace vc
