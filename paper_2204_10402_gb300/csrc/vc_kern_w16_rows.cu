// 16-bit degree-array instances of the bit-row kernels: one-warp workers, node in shared
// memory, adjacency as 1-, 2-, 4- or 8-word bit rows (graphs with n <= 32, 64, 128, 256).
#include "vc_launch_impl.cuh"

namespace vc {
const Launchers &launchers_w16_rows(int nw) {
    if (nw == 1) return LaunchImpl<int16_t, false, 1>::table();
    if (nw == 2) return LaunchImpl<int16_t, false, 2>::table();
    if (nw == 4) return LaunchImpl<int16_t, false, 4>::table();
    return LaunchImpl<int16_t, false, 8>::table();
}
}  // namespace vc
