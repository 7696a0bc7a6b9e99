// Device helpers shared by the step kernels of libhj: order-preserving
// min/max, the fused alpha^max reduction, and the CFL/time-loop finaliser
// that the last CTA of every step runs.
#pragma once

#include <cuda_runtime.h>

#include "hj_internal.h"

// ---------------------------------------------------------------- min / max
// FP64 min/max are slow on this GPU (they run on the FP64 unit).  For finite
// doubles, flipping the magnitude bits of negative values gives an integer
// key with the same order, so min/max become integer compares plus a select.
__device__ __forceinline__ long long hj_key(double x)
{
    long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double hj_max(double a, double b) { return hj_key(a) >= hj_key(b) ? a : b; }
__device__ __forceinline__ double hj_min(double a, double b) { return hj_key(a) <= hj_key(b) ? a : b; }
__device__ __forceinline__ float hj_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ float hj_min(float a, float b) { return fminf(a, b); }

// Non-negative doubles order like their bit patterns read as unsigned.
__device__ __forceinline__ unsigned long long hj_abits(double a) { return (unsigned long long)__double_as_longlong(a); }

__device__ __forceinline__ unsigned long long hj_warp_max_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = v > w ? v : w;
    }
    return v;
}

// ---------------------------------------------------------------- time loop

// dt for the next step from alpha^max (Algorithm 1: dt = CFL / sum_d
// alpha_d^max / dx_d), cut so that t lands on the horizon.  Same operation
// order as the oracle's FP64 arithmetic, with explicit round-to-nearest
// intrinsics so that no contraction can change a bit.
__device__ __forceinline__ void hj_next_dt(HjDevState *st, const HjGeom &g, const double a[4], double t)
{
    double T = st->T;
    if (!(t < T)) {
        st->done = 1;
        st->last = 0;
        return;
    }
    double S = 0.0;
#pragma unroll
    for (int d = 0; d < 4; ++d)
        S = __dadd_rn(S, __ddiv_rn(a[d], g.h[d]));
    double dt = (S == 0.0) ? 0.0 : __ddiv_rn(st->cfl, S);
    if (!(dt >= 0.0) || isinf(dt)) {
        st->status = HJ_ERR_UNSTABLE;
        st->done = 1;
        return;
    }
    int last = (dt == 0.0) || (__dadd_rn(t, dt) >= T);
    if (last) dt = __dadd_rn(T, -t);
    st->dt = dt;
    st->last = last;
    st->done = 0;
}

// The finaliser's arithmetic, given the step's alpha_1^max, alpha_2^max
// (|xdot_1|, |xdot_2| maxima) and largest change eps: publish alpha^max,
// advance t and n, run the convergence test, compute the next dt.
__device__ __forceinline__ void hj_finalise_values(HjDevState *st, const HjGeom &g, double a1, double a2, double eps)
{
    double a[4];
    a[0] = a1;
    a[1] = a2;
    a[2] = g.alpha3;  // |a_opt| = a_max at every cell (bang-bang), |c3| for constant dynamics
    a[3] = g.alpha4;
#pragma unroll
    for (int d = 0; d < 4; ++d) st->alpha_prev[d] = a[d];
    double t = st->t, dt = st->dt;
    double tn = st->last ? st->T : __dadd_rn(t, dt);
    st->dt_prev = dt;
    st->t = tn;
    st->n = st->n + 1;
    if (st->track) {  // Algorithm 2's convergence test on the step just taken
        st->delta_last = eps;
        if (eps < st->threshold) st->converged = 1;
    }
    if (st->status == HJ_OK)
        hj_next_dt(st, g, a, tn);
    else
        st->done = 1;
    if (st->converged) st->done = 1;
}

// Run by one thread of the last CTA to finish a step: read the grid-wide
// maxima, finalise, reset the per-step accumulators.
__device__ __forceinline__ void hj_finalise(HjDevState *st, const HjGeom &g)
{
    __threadfence();
    const double a1 = __longlong_as_double((long long)atomicAdd(&st->alpha_bits[0], 0ull));
    const double a2 = __longlong_as_double((long long)atomicAdd(&st->alpha_bits[1], 0ull));
    const double eps = st->track ? __longlong_as_double((long long)atomicAdd(&st->delta_bits, 0ull)) : 0.0;
    hj_finalise_values(st, g, a1, a2, eps);
    st->alpha_bits[0] = 0ull;
    st->alpha_bits[1] = 0ull;
    st->delta_bits = 0ull;
    st->blocks_done = 0u;
    __threadfence();
}

// Start of a solve call, run by one block: horizon, Courant number and the
// dt of the first step.  Right after V0 is set (n == 0), or after new
// dynamics, alpha^max is reduced over the (v, theta) coefficient table, which
// holds |xdot_1|, |xdot_2| of every cell (the car's velocity depends only on
// v and theta).  scratch holds at least 64 values.
template <typename T>
__device__ __forceinline__ void hj_prologue_block(HjDevState *st, const HjGeom &g, const HjCoef<T> *__restrict__ coef,
                                                  int ncoef, double T_end, double cfl, double threshold,
                                                  unsigned long long *scratch)
{
    unsigned long long a1 = 0ull, a2 = 0ull;
    const bool fresh = st->n == 0 || st->alpha_stale;
    if (fresh)
        for (int i = threadIdx.x; i < ncoef; i += blockDim.x) {
            unsigned long long b1 = hj_abits(coef[i].a1), b2 = hj_abits(coef[i].a2);
            a1 = a1 > b1 ? a1 : b1;
            a2 = a2 > b2 ? a2 : b2;
        }
    a1 = hj_warp_max_u64(a1);
    a2 = hj_warp_max_u64(a2);
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        scratch[warp] = a1;
        scratch[32 + warp] = a2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            a1 = a1 > scratch[w] ? a1 : scratch[w];
            a2 = a2 > scratch[32 + w] ? a2 : scratch[32 + w];
        }
        st->T = T_end;
        st->cfl = cfl;
        // convergence mode (threshold > 0): the steps reduce max |V_{n+1} - V_n|
        st->track = threshold > 0.0 ? 1 : 0;
        st->threshold = threshold;
        st->converged = 0;
        st->delta_bits = 0ull;
        st->delta_last = 0.0;
        double a[4];
        if (fresh) {
            a[0] = __longlong_as_double((long long)a1);
            a[1] = __longlong_as_double((long long)a2);
            a[2] = g.alpha3;
            a[3] = g.alpha4;
            for (int d = 0; d < 4; ++d) st->alpha_prev[d] = a[d];
            st->alpha_stale = 0;
        } else {
            for (int d = 0; d < 4; ++d) a[d] = st->alpha_prev[d];
        }
        st->alpha_bits[0] = 0ull;
        st->alpha_bits[1] = 0ull;
        st->blocks_done = 0u;
        if (st->status == HJ_OK)
            hj_next_dt(st, g, a, st->t);
        else
            st->done = 1;
    }
}

// Block-wide max of the CTA's |xdot_1|, |xdot_2| partials and of its largest
// change |V_{n+1} - V_n| (bit patterns of non-negative doubles; the change
// is 0 outside the convergence mode).  Every thread of the block must call
// it; thread 0 returns the CTA's maxima in a1, a2, d.  `scratch` holds at
// least 3 * 32 unsigned long long.
__device__ __forceinline__ void hj_block_max3(unsigned long long &a1, unsigned long long &a2, unsigned long long &d,
                                              unsigned long long *scratch)
{
    a1 = hj_warp_max_u64(a1);
    a2 = hj_warp_max_u64(a2);
    d = hj_warp_max_u64(d);
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = (blockDim.x + 31) >> 5;
    if (lane == 0) {
        scratch[warp] = a1;
        scratch[32 + warp] = a2;
        scratch[64 + warp] = d;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nwarp; ++w) {
            a1 = a1 > scratch[w] ? a1 : scratch[w];
            a2 = a2 > scratch[32 + w] ? a2 : scratch[32 + w];
            d = d > scratch[64 + w] ? d : scratch[64 + w];
        }
    }
}

// The CTA's maxima (hj_block_max3), then the grid-wide atomic max and the
// last-CTA finaliser.  Every thread of the block must call it.  Thread 0
// returns whether its CTA was the last one.
__device__ __forceinline__ bool hj_step_reduce(HjDevState *st, const HjGeom &g, unsigned long long a1,
                                               unsigned long long a2, unsigned long long d,
                                               unsigned long long *scratch)
{
    hj_block_max3(a1, a2, d, scratch);
    bool last = false;
    if (threadIdx.x == 0) {
        atomicMax(&st->alpha_bits[0], a1);
        atomicMax(&st->alpha_bits[1], a2);
        if (d) atomicMax(&st->delta_bits, d);
        __threadfence();
        unsigned int prev = atomicAdd(&st->blocks_done, 1u);
        last = prev == gridDim.x - 1;
        if (last) hj_finalise(st, g);
    }
    return last;
}

__device__ __forceinline__ void hj_step_epilogue(HjDevState *st, const HjGeom &g, unsigned long long a1,
                                                 unsigned long long a2, unsigned long long d,
                                                 unsigned long long *scratch)
{
    hj_step_reduce(st, g, a1, a2, d, scratch);
}

// Selects V after n steps' input and output buffers.
template <typename T>
__device__ __forceinline__ void hj_io_buffers(const T *v0, T *buf, long long nint, long long n, const T *&vin, T *&vout)
{
    vin = (n == 0) ? v0 : buf + ((n - 1) & 1) * nint;
    vout = buf + (n & 1) * nint;
}
