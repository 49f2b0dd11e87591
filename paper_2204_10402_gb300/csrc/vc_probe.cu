// vc_probe.cu - L2 bandwidth probe for the roofline of the traversal kernel, whose working set
// (degree arrays, stacks, worklist) is meant to stay in L2: one launch copies an L2-sized buffer
// onto another `passes` times, through L2 only (.cg), so that no launch gap and no L1 hit enters
// the measurement.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vc.h"

namespace {

__global__ void l2_copy_kernel(int4 *dst, const int4 *src, size_t n16, int32_t passes) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int32_t p = 0; p < passes; ++p) {
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
            int4 v = __ldcg(src + i);
            v.x ^= p;  // every pass stores something different, so none can be folded away
            __stcg(dst + i, v);
        }
    }
}

}  // namespace

extern "C" int vc_l2_copy_probe(void *dst, const void *src, size_t bytes, int32_t passes, void *stream) {
    if (!dst || !src || bytes == 0 || (bytes & 15) || passes < 1 || ((uintptr_t)dst & 15) || ((uintptr_t)src & 15))
        return VC_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return VC_ECUDA;
    const size_t n16 = bytes / 16;
    const int threads = 512;
    size_t blocks = (size_t)sms * 4;
    const size_t need = (n16 + threads - 1) / threads;
    if (blocks > need) blocks = need;
    l2_copy_kernel<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(static_cast<int4 *>(dst),
                                                                          static_cast<const int4 *>(src), n16, passes);
    return cudaPeekAtLastError() == cudaSuccess ? VC_OK : VC_ECUDA;
}
