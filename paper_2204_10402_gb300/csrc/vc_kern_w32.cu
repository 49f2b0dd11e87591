// 32-bit degree-array instances of the kernels, node in shared memory.
#include "vc_launch_impl.cuh"

namespace vc {
const Launchers &launchers_w32() {
    using I = LaunchImpl<int32_t, false>;
    static const Launchers L = {&I::greedy, &I::traverse, &I::reduce, &I::occupancy};
    return L;
}
}  // namespace vc
