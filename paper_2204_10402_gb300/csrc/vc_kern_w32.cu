// 32-bit degree-array instances of the kernels.
#include "vc_launch_impl.cuh"

namespace vc {
const Launchers &launchers_w32() {
    static const Launchers L = {&LaunchImpl<int32_t>::greedy, &LaunchImpl<int32_t>::traverse,
                                &LaunchImpl<int32_t>::reduce, &LaunchImpl<int32_t>::occupancy};
    return L;
}
}  // namespace vc
