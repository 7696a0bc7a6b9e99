// FP32 variants of the tiled step kernel (fixed-horizon mode).
#include "hj_tiled_kernel.cuh"

namespace hj_tiled {

KernelFn select_f32(bool padded, bool usign, bool bcast, int nc, int rpt)
{
    if (rpt > 1 && !padded && usign && bcast)
        return rpt == 4 ? by_bound<false, false, true, true, false, 4>(nc) : by_bound<false, false, true, true, false, 2>(nc);
    if (padded) {
        if (usign) return bcast ? by_bound<false, true, true, true, false>(nc) : by_bound<false, true, true, false, false>(nc);
        return bcast ? by_bound<false, true, false, true, false>(nc) : by_bound<false, true, false, false, false>(nc);
    }
    if (usign) return bcast ? by_bound<false, false, true, true, false>(nc) : by_bound<false, false, true, false, false>(nc);
    return bcast ? by_bound<false, false, false, true, false>(nc) : by_bound<false, false, false, false, false>(nc);
}

}  // namespace hj_tiled
