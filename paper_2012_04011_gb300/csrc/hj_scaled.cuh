// Step epilogue of the kernels whose coefficient tables carry dt (the FP64
// dt-scaled table and the Q5.27 fixed-point weights): as hj_step_epilogue
// (alpha^max partials, last-CTA finaliser), and the last CTA also rescales
// the table when the next dt differs from the one it holds, which happens
// after the first step of a call and before the cut last step.  Every other
// CTA has finished reading the table by then (it counted itself done after
// its last cell), and the next step kernel is ordered after this one on the
// stream.
#pragma once

#include "hj_device.cuh"

__device__ __forceinline__ void hj_step_epilogue_scaled(HjDevState *st, const HjGeom &g, unsigned long long a1,
                                                        unsigned long long a2, unsigned long long d,
                                                        unsigned long long *scratch, HjScaledCoef *scaled,
                                                        int32_t *qw, const HjCoef<double> *coef, const double *k4)
{
    __shared__ int s_last;
    const bool last = hj_step_reduce(st, g, a1, a2, d, scratch);
    if (threadIdx.x == 0) s_last = last;
    __syncthreads();
    if (s_last) {
        const volatile HjDevState *vs = st;
        const double dtn = vs->dt;
        if (!vs->done && dtn != vs->dt_scaled) {
            if (scaled) hj_rescale_table(scaled, coef, k4, g.n3, g.n4, dtn);
            else hj_rescale_qweights(qw, coef, g.n3, g.n4, g.p4, g.k3, k4, dtn);
            __syncthreads();
            if (threadIdx.x == 0) {
                st->dt_scaled = dtn;
                __threadfence();
            }
        }
    }
}
