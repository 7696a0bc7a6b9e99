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
//
// The same per-cell updates also run in a resident form
// (hj_step_resident_kernel): one cooperative launch takes many steps, with a
// bounded grid barrier between them instead of a kernel boundary, for grids
// so small that launching a step costs more than computing it.
#include <type_traits>

#include "hj_resident.cuh"
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

// ---------------------------------------------------------- one cell's update
// The resident kernel's FP32 / FP64 update and the Q5.27 update of both
// forms.  hj_step_generic_kernel writes the same FP32 / FP64 expressions, in
// the same order, inline (its FP64 build is 2 % faster that way), so the
// resident and per-step kernels give the same result bit for bit (tested).

// FP32: V_c + dt (K1 (V_up1 - V_c) + K2 (V_up2 - V_c) + k3 (V_up3 - V_c) +
// k4 (V_up4 - V_c)), the Euler update before the BRT min with V0 (the caller
// applies it).  c1, c2 are the signed xdot_d / dx_d of the cell's (v, theta).
__device__ __forceinline__ float cell_value(const float vc, const Neigh<float> &nx, const Neigh<float> &ny,
                                            const Neigh<float> &nv, const Neigh<float> &nt, float c1, float c2,
                                            float k3, float k4, float dt, int mode3, int mode4)
{
    const float u3 = upwind_value<float>(nv, mode3);
    const float u4 = upwind_value<float>(nt, mode4);
    const float u1 = nonneg(c1) ? nx.p : nx.m;
    const float u2 = nonneg(c2) ? ny.p : ny.m;
    const float K1 = fabsf(c1), K2 = fabsf(c2);
    float r = K1 * (u1 - vc);
    r = fmaf(K2, u2 - vc, r);
    r = fmaf(k3, u3 - vc, r);
    r = fmaf(k4, u4 - vc, r);
    return fmaf(dt, r, vc);
}

// FP64: w0 V_c + |w1| V_up1 + |w2| V_up2 + dt k3 V_up3 + w4 V_up4 (1 DMUL +
// 4 DFMA; signs and magnitudes by integer operations), before the BRT min.
__device__ __forceinline__ double cell_value(const double vc, const Neigh<double> &nx, const Neigh<double> &ny,
                                             const Neigh<double> &nv, const Neigh<double> &nt,
                                             const HjScaledCoef &sc, double k3dt, int mode3, int mode4)
{
    const double u3 = upwind_value<double>(nv, mode3);
    const double u4 = upwind_value<double>(nt, mode4);
    const double u1 = nonneg(sc.w1) ? nx.p : nx.m;
    const double u2 = nonneg(sc.w2) ? ny.p : ny.m;
    double r = sc.w0 * vc;
    r = fma(mag(sc.w1), u1, r);
    r = fma(mag(sc.w2), u2, r);
    r = fma(k3dt, u3, r);
    return fma(sc.w4, u4, r);
}

// Q5.27: V_c + round_half_up(sum_d W_d (V_up,d - V_c) / 2^30), BRT min,
// saturation (hj_q527_update); w1, w2 signed (the sign picks the side).
__device__ __forceinline__ int32_t q_cell_value(int32_t vc, int32_t v0c, const QDiff &dx, const QDiff &dy,
                                                const QDiff &dv3, const QDiff &dv4, int32_t w1, int32_t w2,
                                                int32_t w3, int32_t w4, int mode3, int mode4)
{
    const long long d1 = w1 >= 0 ? dx.dp : dx.dm;
    const long long d2 = w2 >= 0 ? dy.dp : dy.dm;
    return hj_q527_update(vc, v0c, d1, d2, q_upwind(dv3, mode3), q_upwind(dv4, mode4), abs(w1), abs(w2), w3, w4);
}

// A cell's indices (i, j, k, l) and its offset in the padded layout, from
// its linear index c over the n1 x n2 x n3 x n4 cells.
struct Cell {
    long long o;
    int i, j, k, l;
};

template <bool FAST32>
__device__ __forceinline__ Cell cell_at(unsigned long long c, const Divisors &dv, const HjGeom &g)
{
    const unsigned int N2 = g.n2, N3 = g.n3, N4 = g.n4;
    unsigned long long row;
    Cell r;
    if (FAST32) {  // the grid has fewer than 2^32 cells
        const uint32_t c32 = (uint32_t)c, row32 = fast_div(c32, dv.n4);
        const uint32_t r2 = fast_div(row32, dv.n3);
        const uint32_t i32 = fast_div(r2, dv.n2);
        row = row32;
        r.l = (int)(c32 - row32 * N4);
        r.k = (int)(row32 - r2 * N3);
        r.i = (int)i32;
        r.j = (int)(r2 - i32 * N2);
    } else {
        row = c / N4;
        r.l = (int)(c - row * N4);
        const unsigned long long r2 = row / N3;
        r.k = (int)(row - r2 * N3);
        r.i = (int)(r2 / N2);
        r.j = (int)(r2 - (unsigned long long)r.i * N2);
    }
    r.o = (long long)row * g.p4 + r.l;
    return r;
}

// Per-thread maxima of a step: |xdot_1|, |xdot_2| and the change of V.
struct StepMax {
    unsigned long long a1 = 0ull, a2 = 0ull, d = 0ull;  // FP64 bit patterns (Q5.27: d in codes)
    float df = 0.f;                                     // FP32 kernels: the change of V
};

// The maxima as bit patterns of non-negative doubles.
template <typename T>
__device__ __forceinline__ void step_max_bits(const StepMax &m, unsigned long long &a1, unsigned long long &a2,
                                              unsigned long long &d)
{
    if constexpr (std::is_same<T, float>::value) {
        a1 = m.a1;
        a2 = m.a2;
        d = hj_abits((double)m.df);
    } else if constexpr (std::is_same<T, double>::value) {
        a1 = m.a1;
        a2 = m.a2;
        d = m.d;
    } else {  // the largest change in codes, as the FP64 value it stands for (exact)
        a1 = m.a1;
        a2 = m.a2;
        d = hj_abits((double)m.d * (1.0 / HJ_Q527_SCALE));
    }
}

// Largest change of V, per precision (convergence mode).
__device__ __forceinline__ void track_change(StepMax &m, float vn, float vc) { m.df = fmaxf(m.df, fabsf(vn - vc)); }
__device__ __forceinline__ void track_change(StepMax &m, double vn, double vc)
{
    const unsigned long long b = hj_abits(mag(vn - vc));
    m.d = m.d > b ? m.d : b;
}
__device__ __forceinline__ void track_change(StepMax &m, int32_t vn, int32_t vc)
{
    const long long dd = (long long)vn - vc;
    const unsigned long long ad = (unsigned long long)(dd < 0 ? -dd : dd);
    m.d = m.d > ad ? m.d : ad;
}

// One step in Q5.27 for every grid (the tiled kernel covers the car grids it
// supports).  alpha^max comes from the FP64 table, so the dt sequence is the
// FP64 one.
template <bool FAST32, bool TRACK>
__global__ void __launch_bounds__(256) hj_step_q527_kernel(const int32_t *__restrict__ v0, int32_t *__restrict__ buf,
                                                            const HjCoef<double> *__restrict__ coef, int32_t *qw,
                                                            const double *__restrict__ k4tab, HjDevState *st,
                                                            const HjGeom g, long long nint, const Divisors dv)
{
    __shared__ unsigned long long scratch[96];
    // a programmatic dependent of the previous step: wait for its grid (its
    // V_n and finalised state), then let the next step be scheduled
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (st->done) return;
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const long long n = st->n;
    const int32_t *vin;
    int32_t *vout;
    hj_io_buffers<int32_t>(v0, buf, nint, n, vin, vout);

    const long long s2 = (long long)g.n3 * g.p4, s1 = (long long)g.n2 * s2;
    const unsigned long long ncell = (unsigned long long)g.n1 * g.n2 * g.n3 * g.n4;
    const int tot = g.n3 * g.p4;
    const int32_t w3 = qw[2 * tot];
    const int32_t *w4tab = qw + 2 * tot + HJ_QW_TAIL;  // theta weight per speed
    StepMax m;
    for (unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; c < ncell;
         c += (unsigned long long)gridDim.x * blockDim.x) {
        const Cell cl = cell_at<FAST32>(c, dv, g);
        const long long o = cl.o;
        const int32_t vc = vin[o];
        const QDiff dx = q_axis(vin, o, cl.i, g.n1, s1, g.periodic & 1, vc);
        const QDiff dy = q_axis(vin, o, cl.j, g.n2, s2, (g.periodic >> 1) & 1, vc);
        const QDiff dv3 = q_axis(vin, o, cl.k, g.n3, g.p4, (g.periodic >> 2) & 1, vc);
        const QDiff dv4 = q_axis(vin, o, cl.l, g.n4, 1, (g.periodic >> 3) & 1, vc);
        const int32_t vn = q_cell_value(vc, v0[o], dx, dy, dv3, dv4, qw[cl.k * g.p4 + cl.l],
                                        qw[tot + cl.k * g.p4 + cl.l], w3, w4tab[cl.k], g.mode3, g.mode4);
        vout[o] = vn;
        if constexpr (TRACK) track_change(m, vn, vc);  // convergence mode: largest change of V
        const HjCoef<double> cf = coef[cl.k * g.n4 + cl.l];
        const unsigned long long b1 = hj_abits(cf.a1), b2 = hj_abits(cf.a2);
        m.a1 = m.a1 > b1 ? m.a1 : b1;
        m.a2 = m.a2 > b2 ? m.a2 : b2;
    }
    unsigned long long a1, a2, d;
    step_max_bits<int32_t>(m, a1, a2, d);
    hj_step_epilogue_scaled(st, g, a1, a2, d, scratch, nullptr, qw, coef, k4tab);
}

template <typename T, bool FAST32, bool TRACK>
__global__ void __launch_bounds__(256) hj_step_generic_kernel(const T *__restrict__ v0, T *__restrict__ buf,
                                                               const HjCoef<T> *__restrict__ coef,
                                                               HjScaledCoef *scaled, const void *__restrict__ k4tab,
                                                               HjDevState *st, const HjGeom g, long long nint,
                                                               const Divisors dv)
{
    __shared__ unsigned long long scratch[96];
    // a programmatic dependent of the previous step: wait for its grid (its
    // V_n and finalised state), then let the next step be scheduled
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (st->done) return;  // uniform: written by the previous kernel on this stream
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
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
    float dmf = 0.f;

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
        // (integer max of the FP64 bit patterns, in both precisions)
        {
            const unsigned long long b1 = hj_abits(cf.a1), b2 = hj_abits(cf.a2);
            am1 = am1 > b1 ? am1 : b1;
            am2 = am2 > b2 ? am2 : b2;
        }
    }
    if constexpr (sizeof(T) == 4) {
        hj_step_epilogue(st, g, am1, am2, hj_abits((double)dmf), scratch);
    } else {
        hj_step_epilogue_scaled(st, g, am1, am2, dbits, scratch, scaled, nullptr, (const HjCoef<double> *)coef,
                                (const double *)k4tab);
    }
}

// ------------------------------------------------------------ resident form
//
// Up to ksteps steps of the time loop in one cooperative launch.  Each thread
// updates theta quads (4 consecutive cells of a row: one 16- or 32-byte load
// per neighbour row instead of four) with the per-cell functions above, so
// the results equal the per-step kernels' bit for bit.  Per CTA, in shared
// memory: the loop state and the per-(v, theta) coefficients of the current
// dt (rebuilt by the CTA itself when dt changes).  alpha^max does not depend
// on V, so every CTA reduces it once from the coefficient table (the same
// maximum as over the grid's cells); each step then needs one grid barrier
// (plus a max-reduction of the change of V in convergence mode), after which
// every CTA runs the finaliser on its copy of the state (identical inputs,
// identical dt).  The state goes back to global memory at the end; a barrier
// that times out records HJ_ERR_TIMEOUT and ends the launch.

constexpr int RES_THREADS = 256;
constexpr int RES_MAX_PER_SM = 4;
constexpr unsigned long long RES_WAIT_NS = 2000000000ull;  // 2 s per barrier wait
constexpr size_t RES_MAX_TABLE = 160 * 1024;                // shared-memory coefficient table

struct QuadDivisors {
    FastDiv q4, n3, n2;
};

template <typename T>
struct Quad {
    T v[4];
};

// Four consecutive values (16-byte aligned) through L2 only: other CTAs
// wrote them earlier in the same launch, and L1 is not coherent across SMs.
__device__ __forceinline__ Quad<float> ld_quad(const float *p)
{
    const float4 a = __ldcg((const float4 *)p);
    return {{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ Quad<int32_t> ld_quad(const int32_t *p)
{
    const int4 a = __ldcg((const int4 *)p);
    return {{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ Quad<double> ld_quad(const double *p)
{
    const double2 a = __ldcg((const double2 *)p), b = __ldcg((const double2 *)p + 1);
    return {{a.x, a.y, b.x, b.y}};
}
// V0 does not change during the launch: the read-only path.
__device__ __forceinline__ Quad<float> ld_quad_ro(const float *p)
{
    const float4 a = __ldg((const float4 *)p);
    return {{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ Quad<int32_t> ld_quad_ro(const int32_t *p)
{
    const int4 a = __ldg((const int4 *)p);
    return {{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ Quad<double> ld_quad_ro(const double *p)
{
    const double2 a = __ldg((const double2 *)p), b = __ldg((const double2 *)p + 1);
    return {{a.x, a.y, b.x, b.y}};
}
// The first nv values of a quad (nv < 4 only at the end of a row).
__device__ __forceinline__ void st_quad(float *p, const Quad<float> &q, int nv)
{
    if (nv == 4) {
        *(float4 *)p = make_float4(q.v[0], q.v[1], q.v[2], q.v[3]);
    } else {
#pragma unroll
        for (int L = 0; L < 4; ++L)
            if (L < nv) p[L] = q.v[L];
    }
}
__device__ __forceinline__ void st_quad(int32_t *p, const Quad<int32_t> &q, int nv)
{
    if (nv == 4) {
        *(int4 *)p = make_int4(q.v[0], q.v[1], q.v[2], q.v[3]);
    } else {
#pragma unroll
        for (int L = 0; L < 4; ++L)
            if (L < nv) p[L] = q.v[L];
    }
}
__device__ __forceinline__ void st_quad(double *p, const Quad<double> &q, int nv)
{
    if (nv == 4) {
        *(double2 *)p = make_double2(q.v[0], q.v[1]);
        *((double2 *)p + 1) = make_double2(q.v[2], q.v[3]);
    } else {
#pragma unroll
        for (int L = 0; L < 4; ++L)
            if (L < nv) p[L] = q.v[L];
    }
}

// The neighbour quads of a quad along one of the axes x, y, v (index i of N,
// stride s): periodic wrap applied; a side that is an extrapolated ghost is
// flagged and not loaded.
template <typename T>
struct QuadAxis {
    Quad<T> m, p;
    bool gm, gp;
};

template <typename T>
__device__ __forceinline__ QuadAxis<T> quad_axis(const T *pc, int i, int N, long long s, bool periodic)
{
    QuadAxis<T> a;
    a.gm = i == 0 && !periodic;
    a.gp = i == N - 1 && !periodic;
    a.m = {{T(0), T(0), T(0), T(0)}};
    a.p = a.m;
    if (i > 0) a.m = ld_quad(pc - s);
    else if (periodic) a.m = ld_quad(pc + (long long)(N - 1) * s);
    if (i < N - 1) a.p = ld_quad(pc + s);
    else if (periodic) a.p = ld_quad(pc - (long long)(N - 1) * s);
    return a;
}

// FP32 / FP64: replace an extrapolated side by the ghost of axis_neighbours,
// V_{-1} = 2 V_0 - V_1 or V_N = 2 V_{N-1} - V_{N-2}, once per quad (the flags
// are the same for its four lanes; N >= 3, so at most one side is a ghost).
template <typename T>
__device__ __forceinline__ void apply_ghosts(QuadAxis<T> &a, const Quad<T> &C)
{
    if (a.gm) {
#pragma unroll
        for (int L = 0; L < 4; ++L) a.m.v[L] = T(2) * C.v[L] - a.p.v[L];
    }
    if (a.gp) {
#pragma unroll
        for (int L = 0; L < 4; ++L) a.p.v[L] = T(2) * C.v[L] - a.m.v[L];
    }
}

// Q5.27 upwind value on an axis whose neighbours are both grid values (the
// side with the larger difference is the side with the larger value).
__device__ __forceinline__ int32_t q_upwind_value(int32_t m, int32_t p, int mode)
{
    if (mode == HJ_AXIS_CONTROL) return p > m ? p : m;
    return mode == HJ_AXIS_PLUS ? p : m;
}

// Q5.27 upwind neighbour of an axis with possibly one extrapolated side (gm:
// index - 1, gp: index + 1): the grid value u to weigh and whether it stands
// for the ghost 2 V_c - u (ghost set; the caller then weighs u by -W and V_c
// by +2W).  The side is the one q_upwind takes from the differences.
__device__ __forceinline__ int32_t q_upwind_ghost(int32_t m, int32_t p, bool gm, bool gp, int32_t vc, int mode,
                                                  bool &ghost)
{
    if (mode == HJ_AXIS_CONTROL) {
        // the larger neighbour; a ghost 2 V_c - V_o is the larger one when V_c >= V_o
        if (gp) {
            ghost = vc >= m;
            return m;
        }
        if (gm) {
            ghost = p < vc;
            return p;
        }
        ghost = false;
        return p > m ? p : m;
    }
    if (mode == HJ_AXIS_PLUS) {
        ghost = gp;
        return gp ? m : p;
    }
    ghost = gm;
    return gm ? p : m;
}

// Shared-memory bytes of a CTA's coefficient tables: per (v, theta) arrays
// with the rows' pitch p4 (a quad's four entries are one 16- or 32-byte
// load) and per-speed arrays.
size_t resident_table_bytes(const hj_grid *g)
{
    const size_t n3 = (size_t)g->n[2], p4 = (size_t)g->p4;
    size_t b;
    if (g->prec == HJ_FP32) b = 8 * n3 * p4 + 4 * n3;
    else if (g->prec == HJ_FP64) b = 24 * n3 * p4 + 8 * n3;
    else b = 4 * (2 * n3 * p4 + HJ_QW_TAIL + n3);
    return (b + 15) / 16 * 16;
}

// Four consecutive table entries from shared memory (16-byte aligned).
__device__ __forceinline__ Quad<float> sm_quad(const float *p)
{
    const float4 a = *(const float4 *)p;
    return {{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ Quad<int32_t> sm_quad(const int32_t *p)
{
    const int4 a = *(const int4 *)p;
    return {{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ Quad<double> sm_quad(const double *p)
{
    const double2 a = *(const double2 *)p, b = *((const double2 *)p + 1);
    return {{a.x, a.y, b.x, b.y}};
}

// FP64 tables for dt: w1, w2, w0 per (v, theta) (hj_scaled_entry), w4 per
// speed; padding lanes 0.  All threads of the block call it.
__device__ __forceinline__ void resident_table64(double *w1t, double *w2t, double *w0t, double *w4t,
                                                 const HjCoef<double> *coef, const double *k4, int n3, int n4,
                                                 int p4, double dt)
{
    for (int e = threadIdx.x; e < n3 * p4; e += blockDim.x) {
        const int k = e / p4, l = e - k * p4;
        HjScaledCoef o = {0.0, 0.0, 0.0, 0.0};
        if (l < n4) o = hj_scaled_entry(coef[k * n4 + l], k4[k], dt);
        w1t[e] = o.w1;
        w2t[e] = o.w2;
        w0t[e] = o.w0;
    }
    for (int k = threadIdx.x; k < n3; k += blockDim.x) w4t[k] = hj_scaled_entry(coef[k * n4], k4[k], dt).w4;
}

// CTAs per SM the register budget is set for: 3 for the 4-byte types (FP32
// and Q5.27 at 80 registers; Q5.27 with a few spills, still faster than 2),
// 2 for FP64
template <typename T>
constexpr int res_min_blocks()
{
    return std::is_same<T, double>::value ? 2 : 3;
}

template <typename T, bool TRACK>
__global__ void __launch_bounds__(RES_THREADS, res_min_blocks<T>()) hj_step_resident_kernel(
    const T *__restrict__ v0, T *buf, const void *__restrict__ coefp, const void *__restrict__ k4tab,
    HjDevState *st, const HjGeom g, long long nint, const QuadDivisors dv, HjResidentSync *sync, long long ksteps,
    unsigned long long limit_ns)
{
    constexpr bool Q = std::is_same<T, int32_t>::value;
    constexpr bool F32 = std::is_same<T, float>::value;
    extern __shared__ __align__(16) unsigned char res_smem[];
    __shared__ HjDevState s;
    __shared__ unsigned long long scratch[96];
    __shared__ double s_alpha[2];
    __shared__ int s_ok;

    const int N1 = g.n1, N2 = g.n2, N3 = g.n3, N4 = g.n4, P4 = g.p4, tot = N3 * P4;
    const int per = g.periodic;
    // the CTA's coefficient tables: FP32 c1, c2 per (v, theta) and k4 per v;
    // FP64 the dt-scaled w1, w2, w0 per (v, theta) and w4 per v; Q5.27 the
    // fixed-point weights (qw layout)
    float *c1t = (float *)res_smem, *c2t = c1t + tot, *k4s = c2t + tot;
    double *w1t = (double *)res_smem, *w2t = w1t + tot, *w0t = w2t + tot, *w4t = w0t + tot;
    int32_t *qtab = (int32_t *)res_smem;

    if (threadIdx.x == 0) s = *st;
    // alpha^max over the coefficient table (= over the grid's cells)
    unsigned long long a1 = 0ull, a2 = 0ull, dz = 0ull;
    if constexpr (F32) {
        const HjCoef<float> *coef = (const HjCoef<float> *)coefp;
        for (int e = threadIdx.x; e < tot; e += blockDim.x) {
            const int k = e / P4, l = e - k * P4;
            float c1 = 0.f, c2 = 0.f;
            if (l < N4) {
                const HjCoef<float> c = coef[k * N4 + l];
                c1 = c.c1;
                c2 = c.c2;
                const unsigned long long b1 = hj_abits(c.a1), b2 = hj_abits(c.a2);
                a1 = a1 > b1 ? a1 : b1;
                a2 = a2 > b2 ? a2 : b2;
            }
            c1t[e] = c1;
            c2t[e] = c2;
        }
        for (int k = threadIdx.x; k < N3; k += blockDim.x) k4s[k] = ((const float2 *)k4tab)[k].x;
    } else {
        const HjCoef<double> *coef = (const HjCoef<double> *)coefp;
        for (int e = threadIdx.x; e < N3 * N4; e += blockDim.x) {
            const unsigned long long b1 = hj_abits(coef[e].a1), b2 = hj_abits(coef[e].a2);
            a1 = a1 > b1 ? a1 : b1;
            a2 = a2 > b2 ? a2 : b2;
        }
    }
    hj_block_max3(a1, a2, dz, scratch);
    if (threadIdx.x == 0) {
        s_alpha[0] = __longlong_as_double((long long)a1);
        s_alpha[1] = __longlong_as_double((long long)a2);
    }
    __syncthreads();
    double table_dt = 0.0;  // dt the FP64 / Q5.27 table holds (0: not built)
    if constexpr (!F32) {
        if (!s.done) {
            if constexpr (Q)
                hj_rescale_qweights(qtab, (const HjCoef<double> *)coefp, N3, N4, P4, g.k3, (const double *)k4tab,
                                    s.dt);
            else
                resident_table64(w1t, w2t, w0t, w4t, (const HjCoef<double> *)coefp, (const double *)k4tab, N3, N4,
                                 P4, s.dt);
            table_dt = s.dt;
            __syncthreads();
        }
    }

    const long long s2 = (long long)N3 * P4, s1 = (long long)N2 * s2;
    const unsigned int Q4 = (unsigned int)(P4 / 4);
    const unsigned long long nquad = (unsigned long long)N1 * N2 * N3 * Q4;
    const unsigned long long q0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const unsigned long long qstride = (unsigned long long)gridDim.x * blockDim.x;
    const bool per4 = (per >> 3) & 1;
    unsigned int barriers = 0;
    bool aborted = false;
    for (long long it = 0; it < ksteps && !s.done; ++it) {
        const T *vin;
        T *vout;
        hj_io_buffers<T>(v0, buf, nint, s.n, vin, vout);
        const T dt = (T)s.dt;
        const double k3dt = g.k3 * s.dt;
        StepMax m;
        for (unsigned long long q = q0; q < nquad; q += qstride) {
            const uint32_t q32 = (uint32_t)q, row = fast_div(q32, dv.q4);
            const int l0 = 4 * (int)(q32 - row * Q4);
            const uint32_t r2 = fast_div(row, dv.n3);
            const uint32_t i32 = fast_div(r2, dv.n2);
            const int k = (int)(row - r2 * N3), i = (int)i32, j = (int)(r2 - i32 * N2);
            const T *rp = vin + (long long)row * P4;
            const T *pc = rp + l0;
            const Quad<T> C = ld_quad(pc);
            QuadAxis<T> ax = quad_axis(pc, i, N1, s1, per & 1);
            QuadAxis<T> ay = quad_axis(pc, j, N2, s2, (per >> 1) & 1);
            QuadAxis<T> av = quad_axis(pc, k, N3, P4, (per >> 2) & 1);
            // theta neighbours outside the quad: before lane 0 and after lane 3
            // (wrapped on a periodic axis; unused at an extrapolated end)
            const T em = l0 > 0 ? __ldcg(rp + l0 - 1) : (per4 ? __ldcg(rp + N4 - 1) : T(0));
            const T ep = l0 + 4 < N4 ? __ldcg(rp + l0 + 4) : (per4 ? __ldcg(rp) : T(0));
            const Quad<T> Z = ld_quad_ro(v0 + (pc - vin));
            const int nv = N4 - l0 < 4 ? N4 - l0 : 4;  // lanes of the quad inside the row
            // the value before lane 0 and after lane nv - 1 (for FP32 / FP64 the
            // extrapolated ghosts at the row's ends are formed here, once)
            T lo_m = em, hi_p = ep;
            if constexpr (!Q) {
                apply_ghosts(ax, C);
                apply_ghosts(ay, C);
                apply_ghosts(av, C);
                if (l0 == 0 && !per4) lo_m = T(2) * C.v[0] - C.v[1];
                if (l0 + nv == N4 && !per4) {  // lane nv - 1 holds l = N4 - 1
                    const T cl = nv == 4 ? C.v[3] : (nv == 3 ? C.v[2] : (nv == 2 ? C.v[1] : C.v[0]));
                    const T cm = nv == 4 ? C.v[2] : (nv == 3 ? C.v[1] : (nv == 2 ? C.v[0] : em));
                    hi_p = T(2) * cl - cm;
                }
            }
            // the quad's coefficients (one vector load per table)
            const int e0 = k * P4 + l0;
            Quad<float> cq1, cq2;
            Quad<double> wq1, wq2, wq0;
            Quad<int32_t> qq1, qq2;
            if constexpr (F32) {
                cq1 = sm_quad(c1t + e0);
                cq2 = sm_quad(c2t + e0);
            } else if constexpr (Q) {
                qq1 = sm_quad(qtab + e0);
                qq2 = sm_quad(qtab + tot + e0);
            } else {
                wq1 = sm_quad(w1t + e0);
                wq2 = sm_quad(w2t + e0);
                wq0 = sm_quad(w0t + e0);
            }
            // Q5.27: no extrapolated ghost among the quad's neighbours
            const bool qinterior = !(ax.gm || ax.gp || ay.gm || ay.gp || av.gm || av.gp) &&
                                   (per4 || (l0 > 0 && l0 + nv < N4));
            Quad<T> out = C;
#pragma unroll
            for (int L = 0; L < 4; ++L) {
                if (L >= nv) continue;
                const int l = l0 + L;
                const T vc = C.v[L];
                const T mraw = L > 0 ? C.v[L > 0 ? L - 1 : 0] : lo_m;
                const T praw = L < nv - 1 ? C.v[L < 3 ? L + 1 : 3] : hi_p;
                T vn;
                if constexpr (Q) {
                    const int32_t w3 = qtab[2 * tot], w4 = qtab[2 * tot + HJ_QW_TAIL + k];
                    if (qinterior) {  // every neighbour is a grid value: the int32 form (exact, same sum)
                        const int32_t w1 = qq1.v[L], w2 = qq2.v[L], a1 = abs(w1), a2 = abs(w2);
                        const int32_t u1 = w1 >= 0 ? ax.p.v[L] : ax.m.v[L];
                        const int32_t u2 = w2 >= 0 ? ay.p.v[L] : ay.m.v[L];
                        const int32_t u3 = q_upwind_value(av.m.v[L], av.p.v[L], g.mode3);
                        const int32_t u4 = q_upwind_value(mraw, praw, g.mode4);
                        const int32_t nsum = -(a1 + a2 + w3 + w4);
                        vn = nsum >= -(1 << 30)
                                 ? hj_q527_update_interior32(vc, Z.v[L], u1, u2, u3, u4, a1, a2, w3, w4, nsum)
                                 : hj_q527_update_interior(vc, Z.v[L], u1, u2, u3, u4, a1, a2, w3, w4, nsum);
                    } else {
                        // an extrapolated ghost on some axis: the ghost 2 V_c - V_o of an upwind
                        // side enters as -W on V_o and +2W on V_c (the operands stay int32; the
                        // sum, exact, is the one of hj_q527_update)
                        const bool gm4 = l == 0 && !per4, gp4 = l == N4 - 1 && !per4;
                        const int32_t w1 = qq1.v[L], w2 = qq2.v[L], a1 = abs(w1), a2 = abs(w2);
                        const bool xpos = w1 >= 0, ypos = w2 >= 0;
                        const bool hx = xpos ? ax.gp : ax.gm, hy = ypos ? ay.gp : ay.gm;
                        const int32_t ux = (xpos != hx) ? ax.p.v[L] : ax.m.v[L];
                        const int32_t uy = (ypos != hy) ? ay.p.v[L] : ay.m.v[L];
                        bool hv, ht;
                        const int32_t uv = q_upwind_ghost(av.m.v[L], av.p.v[L], av.gm, av.gp, vc, g.mode3, hv);
                        const int32_t ut = q_upwind_ghost(mraw, praw, gm4, gp4, vc, g.mode4, ht);
                        const int32_t c0 = -(a1 + a2 + w3 + w4) + (hx ? 2 * a1 : 0) + (hy ? 2 * a2 : 0) +
                                           (hv ? 2 * w3 : 0) + (ht ? 2 * w4 : 0);
                        vn = hj_q527_update_interior(vc, Z.v[L], ux, uy, uv, ut, hx ? -a1 : a1, hy ? -a2 : a2,
                                                     hv ? -w3 : w3, ht ? -w4 : w4, c0);
                    }
                } else {
                    const Neigh<T> nx = {ax.m.v[L], ax.p.v[L]};
                    const Neigh<T> ny = {ay.m.v[L], ay.p.v[L]};
                    const Neigh<T> nvv = {av.m.v[L], av.p.v[L]};
                    const Neigh<T> nt = {mraw, praw};
                    if constexpr (F32) {
                        vn = hj_min(Z.v[L], cell_value(vc, nx, ny, nvv, nt, cq1.v[L], cq2.v[L], (float)g.k3,
                                                       k4s[k], dt, g.mode3, g.mode4));
                    } else {
                        const HjScaledCoef sc = {wq1.v[L], wq2.v[L], wq0.v[L], w4t[k]};
                        vn = hj_min(Z.v[L], cell_value(vc, nx, ny, nvv, nt, sc, k3dt, g.mode3, g.mode4));
                    }
                }
                out.v[L] = vn;
                if constexpr (TRACK) track_change(m, vn, vc);
            }
            st_quad(vout + (pc - vin), out, nv);
        }
        unsigned long long *slot = &sync->slot[(int)(it % 3)];
        if constexpr (TRACK) {  // the step's largest change of V, grid-wide
            unsigned long long u1 = 0ull, u2 = 0ull, d;
            step_max_bits<T>(m, u1, u2, d);
            hj_block_max3(u1, u2, d, scratch);
            if (threadIdx.x == 0 && d) atomicMax(slot, d);
        }
        ++barriers;
        if (!hj_grid_sync(&sync->count, gridDim.x * barriers, limit_ns, &s_ok)) {
            aborted = true;
            break;
        }
        if (threadIdx.x == 0) {
            double eps = 0.0;
            if constexpr (TRACK) {
                eps = __longlong_as_double((long long)__ldcg(slot));
                // the slot of step it - 1 is read by every CTA by now: clear it for step it + 2
                if (blockIdx.x == 0) sync->slot[(int)((it + 2) % 3)] = 0ull;
            }
            hj_finalise_values(&s, g, s_alpha[0], s_alpha[1], eps);
        }
        __syncthreads();
        if constexpr (!F32) {
            if (!s.done && s.dt != table_dt) {  // after the first step and before the cut last one
                if constexpr (Q)
                    hj_rescale_qweights(qtab, (const HjCoef<double> *)coefp, N3, N4, P4, g.k3,
                                        (const double *)k4tab, s.dt);
                else
                    resident_table64(w1t, w2t, w0t, w4t, (const HjCoef<double> *)coefp, (const double *)k4tab, N3,
                                     N4, P4, s.dt);
                table_dt = s.dt;
                __syncthreads();
            }
        }
    }
    if (threadIdx.x != 0) return;
    if (aborted) {
        atomicCAS(&st->status, (int)HJ_OK, (int)HJ_ERR_TIMEOUT);
        return;
    }
    if (blockIdx.x == 0) {  // every CTA holds the same state; the global tables were not touched
        st->t = s.t;
        st->dt = s.dt;
        st->dt_prev = s.dt_prev;
        st->n = s.n;
        st->last = s.last;
        st->done = s.done;
        for (int d = 0; d < 4; ++d) st->alpha_prev[d] = s.alpha_prev[d];
        st->converged = s.converged;
        st->delta_last = s.delta_last;
        if (s.status != HJ_OK) atomicCAS(&st->status, (int)HJ_OK, s.status);
    }
}

template <typename T, bool TRACK>
cudaError_t launch_resident(hj_grid *g, long long k)
{
    const void *fn = (const void *)hj_step_resident_kernel<T, TRACK>;
    const size_t smem = resident_table_bytes(g);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, RES_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1 || sms < 1) return cudaErrorCooperativeLaunchTooLarge;
    if (per_sm > RES_MAX_PER_SM) per_sm = RES_MAX_PER_SM;
    const long long nquad = g->nint / 4;
    const long long want = (nquad + RES_THREADS - 1) / RES_THREADS;
    const long long cap = (long long)sms * per_sm;
    const int blocks = (int)(want < cap ? (want > 0 ? want : 1) : cap);
    QuadDivisors dv;
    dv.q4 = make_fastdiv((uint32_t)(g->p4 / 4));
    dv.n3 = make_fastdiv((uint32_t)g->n[2]);
    dv.n2 = make_fastdiv((uint32_t)g->n[1]);
    const T *v0 = (const T *)g->v0;
    T *buf = (T *)g->buf;
    const void *coef = g->coef;
    const void *k4 = g->k4tab;
    HjDevState *st = g->dstate;
    HjGeom geom = g->geom;
    long long nint = g->nint;
    HjResidentSync *sync = g->rsync;
    long long ksteps = k;
    unsigned long long limit = RES_WAIT_NS;
    void *args[] = {&v0, &buf, &coef, &k4, &st, &geom, &nint, &dv, &sync, &ksteps, &limit};
    return cudaLaunchCooperativeKernel(fn, blocks, RES_THREADS, args, smem, g->stream);
}

}  // namespace

bool hj_resident_supported(const hj_grid *g)
{
    int coop = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, g->device) != cudaSuccess) return false;
    return coop != 0 && g->nint < (1LL << 32) && resident_table_bytes(g) <= RES_MAX_TABLE;
}

cudaError_t hj_launch_step_resident(hj_grid *g, long long k)
{
    if (!g->rsync) {
        cudaError_t e = cudaMalloc(&g->rsync, sizeof(HjResidentSync));
        if (e != cudaSuccess) {
            g->rsync = nullptr;
            return e;
        }
        g->device_bytes += sizeof(HjResidentSync);
    }
    cudaError_t e = cudaMemsetAsync(g->rsync, 0, sizeof(HjResidentSync), g->stream);
    if (e != cudaSuccess) return e;
    if (g->prec == HJ_Q527) return g->track ? launch_resident<int32_t, true>(g, k) : launch_resident<int32_t, false>(g, k);
    if (g->prec == HJ_FP64) return g->track ? launch_resident<double, true>(g, k) : launch_resident<double, false>(g, k);
    return g->track ? launch_resident<float, true>(g, k) : launch_resident<float, false>(g, k);
}

// Launch of a step kernel as a programmatic dependent of the previous launch
// on the stream (the kernel waits for that grid before it reads its state).
template <typename... KArgs, typename... Args>
static cudaError_t launch_dependent(void (*fn)(KArgs...), int blocks, int threads, cudaStream_t stream, Args... args)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, (KArgs)args...);
}

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
    cudaError_t le = cudaSuccess;
#define HJ_LAUNCH_Q(F, K)                                                                                      \
    le = launch_dependent(hj_step_q527_kernel<F, K>, blocks, threads, g->stream, (const int32_t *)g->v0,      \
                          (int32_t *)g->buf, (const HjCoef<double> *)g->coef, g->qw, (const double *)g->k4tab, \
                          g->dstate, g->geom, g->nint, dv)
#define HJ_LAUNCH(T, F, K)                                                                                     \
    le = launch_dependent(hj_step_generic_kernel<T, F, K>, blocks, threads, g->stream, (const T *)g->v0,      \
                          (T *)g->buf, (const HjCoef<T> *)g->coef, g->scaled, (const void *)g->k4tab, g->dstate, \
                          g->geom, g->nint, dv)
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
    return le != cudaSuccess ? le : cudaGetLastError();
}
