// 16-bit degree-array instances of the kernels, node in shared memory (graphs with n <= 32768).
#include "vc_launch_impl.cuh"

namespace vc {
const Launchers &launchers_w16() { return LaunchImpl<int16_t, false, 0>::table(); }
}  // namespace vc
