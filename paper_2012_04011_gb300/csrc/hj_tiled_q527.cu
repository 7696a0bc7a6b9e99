// Q5.27 fixed-point variants of the tiled step kernel (both modes).
#include "hj_tiled_kernel.cuh"

namespace hj_tiled {

KernelFn select_q527(bool padded, bool bcast, bool track, int nc)
{
    if (track) {
        if (padded) return bcast ? by_bound<true, true, false, true, true>(nc) : by_bound<true, true, false, false, true>(nc);
        return bcast ? by_bound<true, false, false, true, true>(nc) : by_bound<true, false, false, false, true>(nc);
    }
    if (padded) return bcast ? by_bound<true, true, false, true, false>(nc) : by_bound<true, true, false, false, false>(nc);
    return bcast ? by_bound<true, false, false, true, false>(nc) : by_bound<true, false, false, false, false>(nc);
}

}  // namespace hj_tiled
