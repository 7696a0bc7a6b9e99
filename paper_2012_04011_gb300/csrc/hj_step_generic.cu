// Generic HJ step kernel: one thread per cell (grid-stride), neighbours read
// through L1/L2.  Supports every grid, both precisions and any periodic
// mask.  It is the FP64 path (which is bound by the FP64 ALU on this GPU,
// not by HBM) and the FP32 fallback for grids the tiled kernel rejects.
//
// Per cell it computes one step of Algorithm 2 (Sec. II-B of arxiv
// 2012.04011) in upwind form.  With the local dissipation alpha_d = |xdot_d|
// the Lax-Friedrichs rate of one axis,
//     xdot_d (D+ + D-)/2 + |xdot_d| (D+ - D-)/2,
// equals xdot_d D+ when xdot_d >= 0 and xdot_d D- otherwise, i.e.
//     (|xdot_d| / dx_d) (V_up - V_c)
// with V_up the neighbour on the side the flow comes from.  On a control
// axis the bang-bang u_opt takes the sign of the costate, so V_up is
// max(V+, V-).  Summing over axes:
//     V_new = min(V0, V_c + dt * (sum_d K_d V_up,d - K_sum V_c)),
// with K_d = |xdot_d| / dx_d.  The FP64 variant folds dt into a per-(v, theta)
// table (w0 = 1 - dt K_sum, w_d = dt K_d): 1 DMUL + 4 DFMA per cell, the
// table rescaled by the last CTA only when dt changes.  The FP32 variant
// keeps the differences (V_up - V_c) for accuracy.  The Q5.27 kernel
// (hj_step_q527_kernel) evaluates the same form in exact integer differences
// with fixed-point weights.
#include "hj_scaled.cuh"

namespace {

// Division of 32-bit unsigned integers by an invariant divisor d >= 1 with a
// multiply-high and shifts (Granlund and Montgomery, "Division by Invariant
// Integers using Multiplication", PLDI 1994, Sec. 4): with l = ceil(log2 d)
// and m = floor(2^32 (2^l - d) / d) + 1, q = (t + ((n - t) >> min(l, 1)))
// >> max(l - 1, 0) where t = mulhi(m, n), exact for every 32-bit n.  A
// runtime integer division is a long instruction sequence on this GPU (part
// of it on the FP64 unit, which the FP64 path needs for its arithmetic).
struct FastDiv {
    uint32_t d, m, s1, s2;
};

FastDiv make_fastdiv(uint32_t d)
{
    FastDiv f;
    int l = 0;
    while ((1ull << l) < d) ++l;
    f.d = d;
    f.m = (uint32_t)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
    f.s1 = l > 0 ? 1u : 0u;
    f.s2 = l > 0 ? (uint32_t)(l - 1) : 0u;
    return f;
}

__device__ __forceinline__ uint32_t fast_div(uint32_t n, const FastDiv &f)
{
    const uint32_t t = __umulhi(n, f.m);
    return (t + ((n - t) >> f.s1)) >> f.s2;
}

struct Divisors {
    FastDiv n4, n3, n2;
};

// Sign and magnitude of a coefficient without the FP64 unit: the sign bit
// is in the high word.
__device__ __forceinline__ bool nonneg(double x) { return __double2hiint(x) >= 0; }
__device__ __forceinline__ bool nonneg(float x) { return __float_as_int(x) >= 0; }

template <typename T>
struct Neigh {
    T m, p;  // values at index - 1 and + 1 along one axis (ghosts already applied)
};

// Neighbours along one axis of a cell at offset o with index i of N and
// stride s.  Ends: periodic wrap, or linear extrapolation
// V_{-1} = 2 V_0 - V_1, V_N = 2 V_{N-1} - V_{N-2} (the "extrapolated points"
// of Sec. II-B).
template <typename T>
__device__ __forceinline__ Neigh<T> axis_neighbours(const T *__restrict__ v, long long o, int i, int N, long long s,
                                                    bool periodic, T vc)
{
    Neigh<T> r;
    if (i > 0)
        r.m = v[o - s];
    else
        r.m = periodic ? v[o + (long long)(N - 1) * s] : T(2) * vc - v[o + s];
    if (i < N - 1)
        r.p = v[o + s];
    else
        r.p = periodic ? v[o - (long long)(N - 1) * s] : T(2) * vc - v[o - s];
    return r;
}

template <typename T>
__device__ __forceinline__ T upwind_value(const Neigh<T> &nb, int mode)
{
    if (mode == HJ_AXIS_CONTROL) return hj_max(nb.p, nb.m);
    return mode == HJ_AXIS_PLUS ? nb.p : nb.m;
}

// Magnitude without the FP64 unit: clear the sign bit.
__device__ __forceinline__ double mag(double x)
{
    return __longlong_as_double(__double_as_longlong(x) & 0x7fffffffffffffffLL);
}

// Q5.27 neighbour differences along one axis: V(i-1) - V_c and V(i+1) - V_c
// in exact integers (ghosts: periodic wrap or the linear extrapolation, whose
// difference is minus the one on the other side).
struct QDiff {
    long long dm, dp;
};

__device__ __forceinline__ QDiff q_axis(const int32_t *__restrict__ v, long long o, int i, int N, long long s,
                                        bool periodic, int32_t vc)
{
    long long m = 0, p = 0;
    const bool gm = i == 0 && !periodic, gp = i == N - 1 && !periodic;
    if (i > 0) m = v[o - s];
    else if (periodic) m = v[o + (long long)(N - 1) * s];
    if (i < N - 1) p = v[o + s];
    else if (periodic) p = v[o - (long long)(N - 1) * s];
    QDiff d;
    d.dm = gm ? (long long)vc - p : m - vc;
    d.dp = gp ? (long long)vc - m : p - vc;
    return d;
}

__device__ __forceinline__ long long q_upwind(const QDiff &d, int mode)
{
    if (mode == HJ_AXIS_CONTROL) return d.dp > d.dm ? d.dp : d.dm;
    return mode == HJ_AXIS_PLUS ? d.dp : d.dm;
}

// One step in Q5.27 for every grid (the tiled kernel covers the car grids it
// supports): V_c + round_half_up(sum_d W_d (V_up,d - V_c) / 2^30), BRT min,
// saturation (hj_q527_update).  alpha^max comes from the FP64 table, so the dt
// sequence is the FP64 one.
template <bool FAST32, bool TRACK>
__global__ void __launch_bounds__(256) hj_step_q527_kernel(const int32_t *__restrict__ v0, int32_t *__restrict__ buf,
                                                            const HjCoef<double> *__restrict__ coef, int32_t *qw,
                                                            const double *__restrict__ k4tab, HjDevState *st,
                                                            const HjGeom g, long long nint, const Divisors dv)
{
    __shared__ unsigned long long scratch[96];
    if (st->done) return;
    const long long n = st->n;
    const int32_t *vin;
    int32_t *vout;
    hj_io_buffers<int32_t>(v0, buf, nint, n, vin, vout);

    const unsigned int N1 = g.n1, N2 = g.n2, N3 = g.n3, N4 = g.n4;
    const long long s3 = g.p4, s2 = (long long)N3 * g.p4, s1 = (long long)N2 * s2;
    const unsigned long long ncell = (unsigned long long)N1 * N2 * N3 * N4;
    const int tot = (int)N3 * g.p4;
    const int32_t w3 = qw[2 * tot];
    const int32_t *w4tab = qw + 2 * tot + HJ_QW_TAIL;  // theta weight per speed
    unsigned long long am1 = 0ull, am2 = 0ull, dq = 0ull;

    for (unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; c < ncell;
         c += (unsigned long long)gridDim.x * blockDim.x) {
        unsigned long long row;
        int l, k, i, j;
        if (FAST32) {
            const uint32_t c32 = (uint32_t)c, row32 = fast_div(c32, dv.n4);
            const uint32_t r2 = fast_div(row32, dv.n3);
            const uint32_t i32 = fast_div(r2, dv.n2);
            row = row32;
            l = (int)(c32 - row32 * N4);
            k = (int)(row32 - r2 * N3);
            i = (int)i32;
            j = (int)(r2 - i32 * N2);
        } else {
            row = c / N4;
            l = (int)(c - row * N4);
            const unsigned long long r2 = row / N3;
            k = (int)(row - r2 * N3);
            i = (int)(r2 / N2);
            j = (int)(r2 - (unsigned long long)i * N2);
        }
        const long long o = (long long)row * g.p4 + l;
        const int32_t vc = vin[o];
        const QDiff dx = q_axis(vin, o, i, N1, s1, g.periodic & 1, vc);
        const QDiff dy = q_axis(vin, o, j, N2, s2, (g.periodic >> 1) & 1, vc);
        const QDiff dv3 = q_axis(vin, o, k, N3, s3, (g.periodic >> 2) & 1, vc);
        const QDiff dv4 = q_axis(vin, o, l, N4, 1, (g.periodic >> 3) & 1, vc);
        const int32_t w1 = qw[k * g.p4 + l], w2 = qw[tot + k * g.p4 + l];
        const long long d1 = w1 >= 0 ? dx.dp : dx.dm;
        const long long d2 = w2 >= 0 ? dy.dp : dy.dm;
        const int32_t vn = hj_q527_update(vc, v0[o], d1, d2, q_upwind(dv3, g.mode3), q_upwind(dv4, g.mode4), abs(w1),
                                          abs(w2), w3, w4tab[k]);
        vout[o] = vn;
        if constexpr (TRACK) {  // convergence mode: largest change of V
            const long long dd = (long long)vn - vc;
            const unsigned long long ad = (unsigned long long)(dd < 0 ? -dd : dd);
            dq = dq > ad ? dq : ad;
        }
        const HjCoef<double> cf = coef[k * N4 + l];
        const unsigned long long b1 = hj_abits(cf.a1), b2 = hj_abits(cf.a2);
        am1 = am1 > b1 ? am1 : b1;
        am2 = am2 > b2 ? am2 : b2;
    }
    // the largest change in codes, as the FP64 value it stands for (exact)
    hj_step_epilogue_scaled(st, g, am1, am2, hj_abits((double)dq * (1.0 / HJ_Q527_SCALE)), scratch, nullptr, qw, coef,
                            k4tab);
}

template <typename T, bool FAST32, bool TRACK>
__global__ void __launch_bounds__(256) hj_step_generic_kernel(const T *__restrict__ v0, T *__restrict__ buf,
                                                               const HjCoef<T> *__restrict__ coef,
                                                               HjScaledCoef *scaled, const void *__restrict__ k4tab,
                                                               HjDevState *st, const HjGeom g, long long nint,
                                                               const Divisors dv)
{
    __shared__ unsigned long long scratch[96];
    if (st->done) return;  // uniform: written by the previous kernel on this stream
    const long long n = st->n;
    const T dt = (T)st->dt;
    const T *vin;
    T *vout;
    hj_io_buffers<T>(v0, buf, nint, n, vin, vout);

    const unsigned int N1 = g.n1, N2 = g.n2, N3 = g.n3, N4 = g.n4;
    const long long s3 = g.p4, s2 = (long long)N3 * g.p4, s1 = (long long)N2 * s2;
    const unsigned long long ncell = (unsigned long long)N1 * N2 * N3 * N4;
    const T k3 = (T)g.k3;
    // FP64: dt is folded into the per-(v, theta) table; the v weight needs it
    // once per thread
    const double k3dt = g.k3 * st->dt;
    unsigned long long am1 = 0ull, am2 = 0ull, dbits = 0ull;
    float am1f = 0.f, am2f = 0.f, dmf = 0.f;

    for (unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; c < ncell;
         c += (unsigned long long)gridDim.x * blockDim.x) {
        unsigned long long row;
        int l, k, i, j;
        if (FAST32) {  // the grid has fewer than 2^32 cells
            const uint32_t c32 = (uint32_t)c, row32 = fast_div(c32, dv.n4);
            const uint32_t r2 = fast_div(row32, dv.n3);
            const uint32_t i32 = fast_div(r2, dv.n2);
            row = row32;
            l = (int)(c32 - row32 * N4);
            k = (int)(row32 - r2 * N3);
            i = (int)i32;
            j = (int)(r2 - i32 * N2);
        } else {
            row = c / N4;
            l = (int)(c - row * N4);
            const unsigned long long r2 = row / N3;
            k = (int)(row - r2 * N3);
            i = (int)(r2 / N2);
            j = (int)(r2 - (unsigned long long)i * N2);
        }
        const long long o = (long long)row * g.p4 + l;

        const T vc = vin[o];
        const Neigh<T> nx = axis_neighbours<T>(vin, o, i, N1, s1, g.periodic & 1, vc);
        const Neigh<T> ny = axis_neighbours<T>(vin, o, j, N2, s2, (g.periodic >> 1) & 1, vc);
        const Neigh<T> nv = axis_neighbours<T>(vin, o, k, N3, s3, (g.periodic >> 2) & 1, vc);
        const Neigh<T> nt = axis_neighbours<T>(vin, o, l, N4, 1, (g.periodic >> 3) & 1, vc);

        const HjCoef<T> cf = coef[k * N4 + l];
        const T u3 = upwind_value<T>(nv, g.mode3);
        const T u4 = upwind_value<T>(nt, g.mode4);
        T vn;
        if constexpr (sizeof(T) == 8) {
            // V_new = w0 V_c + |w1| V_up1 + |w2| V_up2 + dt k3 V_up3 + dt k4 V_up4:
            // 1 DMUL + 4 DFMA; signs and magnitudes by integer operations
            const HjScaledCoef sc = scaled[k * N4 + l];
            const T u1 = nonneg(sc.w1) ? nx.p : nx.m;
            const T u2 = nonneg(sc.w2) ? ny.p : ny.m;
            T r = sc.w0 * vc;
            r = fma(mag(sc.w1), u1, r);
            r = fma(mag(sc.w2), u2, r);
            r = fma(k3dt, u3, r);
            vn = fma(sc.w4, u4, r);
        } else {
            const T u1 = nonneg(cf.c1) ? nx.p : nx.m;
            const T u2 = nonneg(cf.c2) ? ny.p : ny.m;
            const T K1 = fabs(cf.c1), K2 = fabs(cf.c2);
            T r = K1 * (u1 - vc);
            r = fmaf(K2, u2 - vc, r);
            r = fmaf(k3, u3 - vc, r);
            r = fmaf(((const float2 *)k4tab)[k].x, u4 - vc, r);  // theta coefficient of this speed
            vn = fmaf(dt, r, vc);
        }
        vn = hj_min(v0[o], vn);  // BRT min with the target (Algorithm 2)
        vout[o] = vn;
        if constexpr (TRACK) {  // convergence mode: largest change of V (Algorithm 2's epsilon)
            if constexpr (sizeof(T) == 8) {
                const unsigned long long b = hj_abits(mag(vn - vc));
                dbits = dbits > b ? dbits : b;
            } else {
                dmf = fmaxf(dmf, fabsf(vn - vc));
            }
        }

        // alpha_d^max: the largest |xdot_d| among the cells this thread updated
        // (FP64: integer max of the bit patterns; FP32: float max, widened once)
        if constexpr (sizeof(T) == 8) {
            const unsigned long long b1 = hj_abits((double)cf.a1), b2 = hj_abits((double)cf.a2);
            am1 = am1 > b1 ? am1 : b1;
            am2 = am2 > b2 ? am2 : b2;
        } else {
            am1f = fmaxf(am1f, (float)cf.a1);
            am2f = fmaxf(am2f, (float)cf.a2);
        }
    }
    if constexpr (sizeof(T) == 4) {
        am1 = hj_abits((double)am1f);
        am2 = hj_abits((double)am2f);
        hj_step_epilogue(st, g, am1, am2, hj_abits((double)dmf), scratch);
    } else {
        hj_step_epilogue_scaled(st, g, am1, am2, dbits, scratch, scaled, nullptr, (const HjCoef<double> *)coef,
                                (const double *)k4tab);
    }
}

}  // namespace

cudaError_t hj_launch_step_generic(hj_grid *g)
{
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    const int threads = 256;
    long long want = (g->ncell + threads - 1) / threads;
    long long cap = (long long)(sms > 0 ? sms : 1) * 8;
    int blocks = (int)(want < cap ? want : cap);
    if (blocks < 1) blocks = 1;
    Divisors dv;
    dv.n4 = make_fastdiv((uint32_t)g->n[3]);
    dv.n3 = make_fastdiv((uint32_t)g->n[2]);
    dv.n2 = make_fastdiv((uint32_t)g->n[1]);
    const bool fast = g->ncell < (1LL << 32);
#define HJ_LAUNCH_Q(F, K)                                                                                     \
    hj_step_q527_kernel<F, K><<<blocks, threads, 0, g->stream>>>(                                          \
        (const int32_t *)g->v0, (int32_t *)g->buf, (const HjCoef<double> *)g->coef, g->qw,                  \
        (const double *)g->k4tab, g->dstate, g->geom, g->nint, dv)
#define HJ_LAUNCH(T, F, K)                                                                                    \
    hj_step_generic_kernel<T, F, K><<<blocks, threads, 0, g->stream>>>(                                    \
        (const T *)g->v0, (T *)g->buf, (const HjCoef<T> *)g->coef, g->scaled, g->k4tab, g->dstate, g->geom, \
        g->nint, dv)
#define HJ_LAUNCH2(T, F)          \
    do {                          \
        if (g->track)             \
            HJ_LAUNCH(T, F, true);  \
        else                      \
            HJ_LAUNCH(T, F, false); \
    } while (0)
    if (g->prec == HJ_Q527) {
        if (fast) {
            if (g->track) HJ_LAUNCH_Q(true, true);
            else HJ_LAUNCH_Q(true, false);
        } else {
            if (g->track) HJ_LAUNCH_Q(false, true);
            else HJ_LAUNCH_Q(false, false);
        }
    } else if (g->prec == HJ_FP64) {
        if (fast) HJ_LAUNCH2(double, true);
        else HJ_LAUNCH2(double, false);
    } else {
        if (fast) HJ_LAUNCH2(float, true);
        else HJ_LAUNCH2(float, false);
    }
#undef HJ_LAUNCH_Q
#undef HJ_LAUNCH
#undef HJ_LAUNCH2
    return cudaGetLastError();
}
