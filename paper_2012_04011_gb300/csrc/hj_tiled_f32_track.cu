// FP32 variants of the tiled step kernel in convergence mode (they also
// reduce max |V_{n+1} - V_n|).
#include "hj_tiled_kernel.cuh"

namespace hj_tiled {

KernelFn select_f32_track(bool padded, bool usign, bool bcast, int nc, int rpt)
{
    if (rpt > 1 && !padded && usign && bcast)
        return rpt == 4 ? by_bound<false, false, true, true, true, 4>(nc) : by_bound<false, false, true, true, true, 2>(nc);
    if (padded) {
        if (usign) return bcast ? by_bound<false, true, true, true, true>(nc) : by_bound<false, true, true, false, true>(nc);
        return bcast ? by_bound<false, true, false, true, true>(nc) : by_bound<false, true, false, false, true>(nc);
    }
    if (usign) return bcast ? by_bound<false, false, true, true, true>(nc) : by_bound<false, false, true, false, true>(nc);
    return bcast ? by_bound<false, false, false, true, true>(nc) : by_bound<false, false, false, false, true>(nc);
}

}  // namespace hj_tiled
