// 16-bit degree-array instances of the kernels (graphs with n <= 32768).
#include "vc_launch_impl.cuh"

namespace vc {
const Launchers &launchers_w16() {
    static const Launchers L = {&LaunchImpl<int16_t>::greedy, &LaunchImpl<int16_t>::traverse,
                                &LaunchImpl<int16_t>::reduce, &LaunchImpl<int16_t>::occupancy};
    return L;
}
}  // namespace vc
