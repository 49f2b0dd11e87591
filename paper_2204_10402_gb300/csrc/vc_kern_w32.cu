// 32-bit degree-array instances of the kernels, node in shared memory.
#include "vc_launch_impl.cuh"

namespace vc {
const Launchers &launchers_w32() { return LaunchImpl<int32_t, false, 0>::table(); }
}  // namespace vc
