// 16-bit degree-array instances of the kernels, node in global memory (Sec. IV-E's second
// kernel version: graphs whose node state does not fit in shared memory).
#include "vc_launch_impl.cuh"

namespace vc {
const Launchers &launchers_w16_gm() { return LaunchImpl<int16_t, true, 0>::table(); }
}  // namespace vc
