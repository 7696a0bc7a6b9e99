// Value, gradient and optimal control of a grid's current V at arbitrary
// states: the controller side of the paper (Sec. IV-A: near the BRT
// boundary, Eq. closetoboundary, the car applies u_opt = argmax_u
// grad V^T f, Eq. uopt_max).
//
// V(z) is the multilinear interpolation of the grid values over the cell
// that contains z (theta wraps; the other axes clamp onto the grid), grad
// V(z) the gradient of that interpolant, and u_opt the bang-bang argmax with
// ties to the upper bound, as in the step kernels.  One thread per state,
// FP64 arithmetic; grid values are read in the grid's precision.  The
// interpolant is evaluated as a tensor product, one axis at a time (15
// linear interpolations for the value, 11 more for the gradient, instead of
// 16 weighted corners per component).
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
    double lo[4], h[4], inv_h[4];
    double span[4], inv_span[4];  // periodic axes: N h and its inverse
    int dyn;
    double p[3];
};

template <typename T>
__device__ __forceinline__ double value_at(const T *__restrict__ V, long long o)
{
    if constexpr (std::is_same<T, int32_t>::value) return hj_q527_to_f64(V[o]);
    else return (double)V[o];
}

// Cell index and fraction of coordinate z on axis d.  The coordinate is
// scaled by the reciprocal spacing and a periodic axis is wrapped with one
// floor (no FP64 division or fmod: both are long FP64 sequences, and the FP64
// unit bounds this kernel); the fraction then differs from the quotient by a
// few ulps at most.
__device__ __forceinline__ void query_cell(const QueryGeom &q, int d, double z, int &i0, double &f)
{
    const int N = q.n[d];
    const double lo = q.lo[d];
    if ((q.periodic >> d) & 1u) {
        const double span = q.span[d];
        double u = z - lo;
        u = fma(-floor(u * q.inv_span[d]), span, u);
        if (u < 0.0) u += span;
        if (u >= span) u -= span;
        const double r = u * q.inv_h[d];
        int i = (int)floor(r);
        if (i >= N) i = N - 1;
        if (i < 0) i = 0;
        i0 = i;
        f = r - (double)i;
        return;
    }
    const double r = (z - lo) * q.inv_h[d];
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

// Linear interpolation a + f (b - a); the difference b - a is returned too.
__device__ __forceinline__ double lerp(double a, double b, double f, double &diff)
{
    diff = b - a;
    return fma(f, diff, a);
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
        // the 16 corner values, corner index ((a*2 + b)*2 + c)*2 + e for
        // (x, y, v, theta) = (i_a, j_b, k_c, l_e); all loads issued first
        double c16[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            long long off = 0;
#pragma unroll
            for (int d = 0; d < 4; ++d) off += (long long)(((c >> (3 - d)) & 1) ? i1[d] : i0[d]) * strides[d];
            c16[c] = value_at(V, off);
        }
        // the multilinear interpolant, contracted one axis at a time (theta,
        // v, y, x); the differences along each axis give the gradient
        double a8[8], d3[8], b4[4], d2[4], c2[2], d1[2], d0;
#pragma unroll
        for (int k = 0; k < 8; ++k) a8[k] = lerp(c16[2 * k], c16[2 * k + 1], f[3], d3[k]);
#pragma unroll
        for (int k = 0; k < 4; ++k) b4[k] = lerp(a8[2 * k], a8[2 * k + 1], f[2], d2[k]);
#pragma unroll
        for (int k = 0; k < 2; ++k) c2[k] = lerp(b4[2 * k], b4[2 * k + 1], f[1], d1[k]);
        value[s] = lerp(c2[0], c2[1], f[0], d0);
        double t;
        // dV/dx: d0; dV/dy: d1 interpolated along x; dV/dv: d2 along y, x;
        // dV/dtheta: d3 along v, y, x
        const double gy = lerp(d1[0], d1[1], f[0], t);
        const double e2a = lerp(d2[0], d2[1], f[1], t), e2b = lerp(d2[2], d2[3], f[1], t);
        const double gv = lerp(e2a, e2b, f[0], t);
        double e3[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) e3[k] = lerp(d3[2 * k], d3[2 * k + 1], f[2], t);
        const double e3a = lerp(e3[0], e3[1], f[1], t), e3b = lerp(e3[2], e3[3], f[1], t);
        const double gt = lerp(e3a, e3b, f[0], t);
        const double g0 = d0 * q.inv_h[0], g1 = gy * q.inv_h[1], g2 = gv * q.inv_h[2], g3 = gt * q.inv_h[3];
        if (grad) {
            grad[4 * s + 0] = g0;
            grad[4 * s + 1] = g1;
            grad[4 * s + 2] = g2;
            grad[4 * s + 3] = g3;
        }
        if (control) {
            double a = 0.0, u = 0.0;
            if (q.dyn == HJ_DYN_CAR4D) {
                a = g2 >= 0.0 ? q.p[0] : -q.p[0];
                u = g3 >= 0.0 ? q.p[1] : -q.p[1];
            } else if (q.dyn == HJ_DYN_CAR4D_STEER) {
                a = g2 >= 0.0 ? q.p[0] : -q.p[0];
                u = g3 * states[4 * s + 2] >= 0.0 ? q.p[1] : -q.p[1];
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
        q.inv_h[d] = 1.0 / g->h[d];
        q.span[d] = g->h[d] * (double)g->n[d];
        q.inv_span[d] = 1.0 / q.span[d];
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
