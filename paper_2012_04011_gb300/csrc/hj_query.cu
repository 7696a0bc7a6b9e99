// Value, gradient and optimal control of a grid's current V at arbitrary
// states: the controller side of the paper (Sec. IV-A: near the BRT
// boundary, Eq. closetoboundary, the car applies u_opt = argmax_u
// grad V^T f, Eq. uopt_max).
//
// V(z) is the multilinear interpolation of the grid values over the cell
// that contains z (theta wraps; the other axes clamp onto the grid), grad
// V(z) the gradient of that interpolant, and u_opt the bang-bang argmax with
// ties to the upper bound, as in the step kernels.  One thread per state,
// FP64 arithmetic; grid values are read in the grid's precision.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <type_traits>

#include "hj_internal.h"

namespace {

struct QueryGeom {
    int n[4];
    int p4;
    unsigned int periodic;
    double lo[4], h[4];
    int dyn;
    double p[3];
};

template <typename T>
__device__ __forceinline__ double value_at(const T *__restrict__ V, long long o)
{
    if constexpr (std::is_same<T, int32_t>::value) return hj_q527_to_f64(V[o]);
    else return (double)V[o];
}

// Cell index and fraction of coordinate z on axis d.
__device__ __forceinline__ void query_cell(const QueryGeom &q, int d, double z, int &i0, double &f)
{
    const int N = q.n[d];
    const double h = q.h[d], lo = q.lo[d];
    if ((q.periodic >> d) & 1u) {
        const double span = h * (double)N;
        double u = fmod(z - lo, span);
        if (u < 0.0) u += span;
        const double r = u / h;
        int i = (int)floor(r);
        if (i >= N) i = N - 1;
        i0 = i;
        f = r - (double)i;
        return;
    }
    const double r = (z - lo) / h;
    if (!(r > 0.0)) {  // also NaN: clamp to the lower end
        i0 = 0;
        f = 0.0;
        return;
    }
    if (r >= (double)(N - 1)) {
        i0 = N - 2;
        f = 1.0;
        return;
    }
    int i = (int)floor(r);
    if (i > N - 2) i = N - 2;
    i0 = i;
    f = r - (double)i;
}

template <typename T>
__global__ void query_kernel(const T *__restrict__ V, const QueryGeom q, const double *__restrict__ states, long long m,
                             double *__restrict__ value, double *__restrict__ grad, double *__restrict__ control)
{
    const long long stride3 = q.p4, stride2 = (long long)q.n[2] * q.p4, stride1 = (long long)q.n[1] * stride2;
    const long long strides[4] = {stride1, stride2, stride3, 1};
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < m;
         s += (long long)gridDim.x * blockDim.x) {
        int i0[4], i1[4];
        double f[4];
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            query_cell(q, d, states[4 * s + d], i0[d], f[d]);
            i1[d] = i0[d] + 1;
            if (i1[d] >= q.n[d]) i1[d] = ((q.periodic >> d) & 1u) ? 0 : q.n[d] - 1;
        }
        double val = 0.0, g[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
        for (int c = 0; c < 16; ++c) {
            long long off = 0;
            double w = 1.0;
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                const int hi = (c >> d) & 1;
                off += (long long)(hi ? i1[d] : i0[d]) * strides[d];
                w *= hi ? f[d] : 1.0 - f[d];
            }
            const double vv = value_at(V, off);
            val += w * vv;
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                double wd = ((c >> d) & 1) ? 1.0 : -1.0;
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (e != d) wd *= ((c >> e) & 1) ? f[e] : 1.0 - f[e];
                g[d] += wd * vv / q.h[d];
            }
        }
        value[s] = val;
        if (grad)
#pragma unroll
            for (int d = 0; d < 4; ++d) grad[4 * s + d] = g[d];
        if (control) {
            double a = 0.0, u = 0.0;
            if (q.dyn == HJ_DYN_CAR4D) {
                a = g[2] >= 0.0 ? q.p[0] : -q.p[0];
                u = g[3] >= 0.0 ? q.p[1] : -q.p[1];
            } else if (q.dyn == HJ_DYN_CAR4D_STEER) {
                a = g[2] >= 0.0 ? q.p[0] : -q.p[0];
                u = g[3] * states[4 * s + 2] >= 0.0 ? q.p[1] : -q.p[1];
            }
            control[2 * s] = a;
            control[2 * s + 1] = u;
        }
    }
}

QueryGeom make_geom(const hj_grid *g)
{
    QueryGeom q;
    memset(&q, 0, sizeof(q));
    for (int d = 0; d < 4; ++d) {
        q.n[d] = g->n[d];
        q.lo[d] = g->lo[d];
        q.h[d] = g->h[d];
    }
    q.p4 = g->p4;
    q.periodic = g->periodic;
    q.dyn = g->dyn;
    for (int i = 0; i < 3; ++i) q.p[i] = g->params[i];
    return q;
}

}  // namespace

cudaError_t hj_launch_query(const hj_grid *g, const void *V, const double *states, long long m, double *value,
                            double *grad, double *control)
{
    if (m <= 0) return cudaSuccess;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    long long blocks = (m + 255) / 256;
    const long long cap = (long long)(sms > 0 ? sms : 1) * 16;
    if (blocks > cap) blocks = cap;
    const QueryGeom q = make_geom(g);
    if (g->prec == HJ_FP64)
        query_kernel<double><<<(int)blocks, 256, 0, g->stream>>>((const double *)V, q, states, m, value, grad, control);
    else if (g->prec == HJ_FP32)
        query_kernel<float><<<(int)blocks, 256, 0, g->stream>>>((const float *)V, q, states, m, value, grad, control);
    else
        query_kernel<int32_t><<<(int)blocks, 256, 0, g->stream>>>((const int32_t *)V, q, states, m, value, grad,
                                                                  control);
    return cudaGetLastError();
}
