/*
 * FP64 CPU oracle for the 4D Hamilton-Jacobi reachability time step
 * (arxiv 2012.04011, "Real-Time Formal Verification of Autonomous Systems
 * With An FPGA").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
 * restatement of the numerical scheme that the CUDA path is checked against.
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may load it.  It shares no code, header, table or constant with the CUDA
 * library, and it never calls that library.
 *
 * What it computes, in the paper's order and notation:
 *   - Eq. (central_diff): one-sided differences D-_d, D+_d and their mean
 *     D_d on every axis d = 1..4, with extrapolated points at the two ends of
 *     each non-periodic axis (Sec. II-B) and a periodic wrap on theta.
 *   - Algorithm 1 sweep 1 with Algorithm 2's local dissipation:
 *     u_opt = argmax_u grad(V).f(z,u) (bang-bang), xdot = f(z,u_opt),
 *     H = grad(V).xdot, alpha_d = |xdot_d|,
 *     L = H + sum_d alpha_d (D+_d - D-_d)/2, alpha_d^max = max over the grid.
 *   - Algorithm 1: dt = CFL / sum_d alpha_d^max / dx_d, the last step cut so
 *     that t lands on the horizon T.
 *   - Algorithm 1/2: V_{t+1} = min(V_0, V_t + dt * L)  (the BRT min after
 *     every Euler step).
 *
 * Readings where the paper is silent or garbled (each one a single place in
 * this file):
 *   - extrapolated points: linear, V_{-1} = 2 V_0 - V_1 and
 *     V_N = 2 V_{N-1} - V_{N-2}                               (ghost_value)
 *   - dissipation sign: ADDED.  The printed "H - sum alpha (D+ - D-)/2" with
 *     "V + H dt" is anti-diffusive; writing the backward PDE D_s V + H = 0 in
 *     tau = -s gives dV/dtau = H and Lax-Friedrichs adds + alpha (D+ - D-)/2.
 *                                                             (cell_rate)
 *   - bang-bang tie: p_d >= 0 selects the upper control bound. (cell_rate)
 *   - dt: CFL / S with S = sum alpha^max/dx; S == 0 means one step to T.
 *                                                             (hjo_cfl_dt)
 *   - grid: x_i = lo + i (hi - lo)/(N - 1) on non-periodic axes (both ends on
 *     the grid), theta_l = lo + l (hi - lo)/N on the periodic axis.
 *                                                             (hjo_spacing)
 *   - car dynamics of the experiments (Sec. IV-A, Eq. car_dynamics) with the
 *     heading rate used as a bounded control w: x' = v cos th, y' = v sin th,
 *     v' = a, th' = w, |a| <= a_max, |w| <= w_max, no disturbance; and the
 *     paper's own steering form th' = v tan(delta) / L, |delta| <= delta_max
 *     (Eq. car_dynamics as printed: a in [-1.5, 1.5], delta in
 *     [-pi/18, pi/18], L = 0.3 m).
 *
 * Compiled with -O2 -ffp-contract=off (no fused multiply-add), scalar code,
 * optional OpenMP over the slowest axis only: the only cross-cell reduction
 * is a max, which is order independent, so every thread count gives the same
 * bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define HJO_DYN_CAR4D 0 /* params {a_max, w_max} */
#define HJO_DYN_CONST 1 /* params {c1, c2, c3, c4}: xdot = c, no control */
#define HJO_DYN_CAR4D_STEER 2 /* params {a_max, delta_max, L}: th' = v tan(delta) / L */

typedef struct {
    int32_t n[4];       /* grid points per axis, axis 4 (theta) fastest */
    double lo[4];       /* lower bound per axis */
    double hi[4];       /* upper bound per axis */
    uint32_t periodic;  /* bit d set: axis d is periodic */
    int32_t dyn;        /* HJO_DYN_* */
    double p[4];        /* dynamics parameters */
} hjo_problem;

/* ---- grid ------------------------------------------------------------ */

static int is_periodic(const hjo_problem *P, int d) { return (P->periodic >> d) & 1u; }

/* Grid spacing dx_d.  Non-periodic axes include both end points; a periodic
 * axis of N points covers [lo, hi) once. */
double hjo_spacing(const hjo_problem *P, int d)
{
    if (is_periodic(P, d))
        return (P->hi[d] - P->lo[d]) / (double)P->n[d];
    return (P->hi[d] - P->lo[d]) / (double)(P->n[d] - 1);
}

/* State x_{d,i} of grid index i on axis d. */
double hjo_coord(const hjo_problem *P, int d, int i)
{
    return P->lo[d] + (double)i * hjo_spacing(P, d);
}

int64_t hjo_cell_count(const hjo_problem *P)
{
    return (int64_t)P->n[0] * P->n[1] * P->n[2] * P->n[3];
}

/* ---- one cell ---------------------------------------------------------- */

typedef struct {
    int64_t stride[4];
    double h[4];
    double *cos_th; /* cos(theta_l), l = 0..N4-1 */
    double *sin_th; /* sin(theta_l) */
    double *v;      /* v_k, k = 0..N3-1 */
} hjo_tables;

static int tables_init(const hjo_problem *P, hjo_tables *T)
{
    T->stride[3] = 1;
    T->stride[2] = P->n[3];
    T->stride[1] = (int64_t)P->n[2] * P->n[3];
    T->stride[0] = (int64_t)P->n[1] * P->n[2] * P->n[3];
    for (int d = 0; d < 4; ++d)
        T->h[d] = hjo_spacing(P, d);
    /* State look-up tables (Sec. III-A keeps the state vectors and cos/sin
     * of theta in on-chip tables; here they are just arrays). */
    T->cos_th = (double *)malloc(sizeof(double) * (size_t)P->n[3]);
    T->sin_th = (double *)malloc(sizeof(double) * (size_t)P->n[3]);
    T->v = (double *)malloc(sizeof(double) * (size_t)P->n[2]);
    if (!T->cos_th || !T->sin_th || !T->v)
        return -1;
    for (int l = 0; l < P->n[3]; ++l) {
        double th = hjo_coord(P, 3, l);
        T->cos_th[l] = cos(th);
        T->sin_th[l] = sin(th);
    }
    for (int k = 0; k < P->n[2]; ++k)
        T->v[k] = hjo_coord(P, 2, k);
    return 0;
}

static void tables_free(hjo_tables *T)
{
    free(T->cos_th);
    free(T->sin_th);
    free(T->v);
}

/* Value at grid index idx[d] + dir (dir = -1 or +1) on axis d, seen from
 * the cell at flat offset c.  Inside the grid it is a plain read; past the
 * end of a periodic axis it wraps; past the end of a non-periodic axis it is
 * the point extrapolated linearly through the two nearest grid points
 * (Sec. II-B: "computed with extrapolated points"). */
static double ghost_value(const hjo_problem *P, const hjo_tables *T, const double *V,
                          int64_t c, const int idx[4], int d, int dir)
{
    int i = idx[d] + dir;
    int N = P->n[d];
    if (i >= 0 && i < N)
        return V[c + dir * T->stride[d]];
    if (is_periodic(P, d)) {
        int w = (i + N) % N;
        return V[c + (int64_t)(w - idx[d]) * T->stride[d]];
    }
    /* i == -1:  V_{-1} = 2 V_0 - V_1;   i == N:  V_N = 2 V_{N-1} - V_{N-2} */
    return 2.0 * V[c] - V[c - dir * T->stride[d]];
}

/* Algorithm 2, lines 3-7 for one cell: returns L = H + dissipation and the
 * |xdot_d| used as the local dissipation coefficients alpha_d. */
static double cell_rate(const hjo_problem *P, const hjo_tables *T, const double *V,
                        int64_t c, const int idx[4], double alpha[4])
{
    double Dm[4], Dp[4], p[4], xdot[4];
    double Vc = V[c];
    for (int d = 0; d < 4; ++d) {
        double Vm = ghost_value(P, T, V, c, idx, d, -1);
        double Vp = ghost_value(P, T, V, c, idx, d, +1);
        Dm[d] = (Vc - Vm) / T->h[d];  /* D-_d V(x_{d,i}) */
        Dp[d] = (Vp - Vc) / T->h[d];  /* D+_d V(x_{d,i}) */
        p[d] = (Dp[d] + Dm[d]) / 2.0; /* D_d V(x_{d,i}), the gradient used in H */
    }
    if (P->dyn == HJO_DYN_CAR4D) {
        double a_max = P->p[0], w_max = P->p[1];
        double v = T->v[idx[2]];
        /* u_opt = argmax_u p . f(z, u): f is affine in (a, w), so each
         * control sits at the bound with the sign of its costate. */
        double a_opt = (p[2] >= 0.0) ? a_max : -a_max;
        double w_opt = (p[3] >= 0.0) ? w_max : -w_max;
        xdot[0] = v * T->cos_th[idx[3]];
        xdot[1] = v * T->sin_th[idx[3]];
        xdot[2] = a_opt;
        xdot[3] = w_opt;
    } else if (P->dyn == HJO_DYN_CAR4D_STEER) {
        double a_max = P->p[0], d_max = P->p[1], L = P->p[2];
        double v = T->v[idx[2]];
        /* p_4 v tan(delta) / L is increasing in delta when p_4 v >= 0 (tan
         * is increasing on (-pi/2, pi/2)): delta_opt is the bound with the
         * sign of p_4 v. */
        double a_opt = (p[2] >= 0.0) ? a_max : -a_max;
        double d_opt = (p[3] * v >= 0.0) ? d_max : -d_max;
        xdot[0] = v * T->cos_th[idx[3]];
        xdot[1] = v * T->sin_th[idx[3]];
        xdot[2] = a_opt;
        xdot[3] = v * tan(d_opt) / L;
    } else {
        for (int d = 0; d < 4; ++d)
            xdot[d] = P->p[d];
    }
    double H = 0.0;
    for (int d = 0; d < 4; ++d)
        H = H + p[d] * xdot[d];
    double diss = 0.0;
    for (int d = 0; d < 4; ++d) {
        alpha[d] = fabs(xdot[d]);
        diss = diss + alpha[d] * (Dp[d] - Dm[d]) / 2.0;
    }
    return H + diss;
}

static void unflatten(const hjo_problem *P, int64_t c, int idx[4])
{
    idx[3] = (int)(c % P->n[3]);
    c /= P->n[3];
    idx[2] = (int)(c % P->n[2]);
    c /= P->n[2];
    idx[1] = (int)(c % P->n[1]);
    idx[0] = (int)(c / P->n[1]);
}

/* ---- sweeps ------------------------------------------------------------ */

/* Algorithm 1 sweeps 1-2 (with Algorithm 2's alpha_d = |xdot_d|): L for every
 * cell and alpha_d^max over the grid.  Loop order i, j, k, l with l
 * innermost. */
static void sweep_rate(const hjo_problem *P, const hjo_tables *T, const double *V,
                       double *L, double alpha_max[4], int nthreads)
{
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int N1 = P->n[0], N2 = P->n[1], N3 = P->n[2], N4 = P->n[3];
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1) \
    reduction(max : a0, a1, a2, a3)
#endif
    for (int i = 0; i < N1; ++i)
        for (int j = 0; j < N2; ++j)
            for (int k = 0; k < N3; ++k)
                for (int l = 0; l < N4; ++l) {
                    int idx[4] = {i, j, k, l};
                    int64_t c = ((((int64_t)i * N2 + j) * N3 + k) * N4) + l;
                    double al[4];
                    L[c] = cell_rate(P, T, V, c, idx, al);
                    a0 = fmax(a0, al[0]);
                    a1 = fmax(a1, al[1]);
                    a2 = fmax(a2, al[2]);
                    a3 = fmax(a3, al[3]);
                }
    alpha_max[0] = a0;
    alpha_max[1] = a1;
    alpha_max[2] = a2;
    alpha_max[3] = a3;
}

/* Stable step of Algorithm 1: dt = CFL * (sum_d alpha_d^max / dx_d)^-1.
 * Returns 0 when the sum is zero (nothing moves; the caller then steps
 * straight to the horizon). */
double hjo_cfl_dt(const hjo_problem *P, const double alpha_max[4], double cfl)
{
    double S = 0.0;
    for (int d = 0; d < 4; ++d)
        S = S + alpha_max[d] / hjo_spacing(P, d);
    if (S == 0.0)
        return 0.0;
    return cfl / S;
}

/* Euler step and BRT min of Algorithms 1-2: V_{t+1} = min(V_0, V_t + dt L). */
static void sweep_update(int64_t ncell, const double *V, const double *V0, const double *L,
                         double dt, double *Vn, int nthreads)
{
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t c = 0; c < ncell; ++c) {
        double v = V[c] + dt * L[c];
        Vn[c] = fmin(V0[c], v);
    }
}

/* ---- entry points ------------------------------------------------------ */

/* L = H + dissipation for every cell and alpha_d^max (both out-params). */
int hjo_rate(const hjo_problem *P, const double *V, double *L, double alpha_max[4], int nthreads)
{
    hjo_tables T;
    if (tables_init(P, &T)) {
        tables_free(&T);
        return -1;
    }
    sweep_rate(P, &T, V, L, alpha_max, nthreads);
    tables_free(&T);
    return 0;
}

/* One step of size dt from V (V0 is the BRT-min operand) for the m cells
 * listed in flat row-major indices idx; results in out[0..m). */
int hjo_step_cells(const hjo_problem *P, const double *V, const double *V0, double dt,
                   const int64_t *cells, int64_t m, double *out)
{
    hjo_tables T;
    if (tables_init(P, &T)) {
        tables_free(&T);
        return -1;
    }
    for (int64_t q = 0; q < m; ++q) {
        int idx[4];
        double al[4];
        int64_t c = cells[q];
        unflatten(P, c, idx);
        double L = cell_rate(P, &T, V, c, idx, al);
        double v = V[c] + dt * L;
        out[q] = fmin(V0[c], v);
    }
    tables_free(&T);
    return 0;
}

/* Advance V (in place) from time *t toward the horizon T_end, at most
 * max_steps steps.  Each step: sweep for L and alpha^max, dt from the CFL
 * rule, dt cut to T_end - t on the last step (t is then set to T_end exactly),
 * Euler update and BRT min against V0.  dts[s] receives each step's dt
 * (may be NULL).  Returns the number of steps taken, or -1 on allocation
 * failure. */
int64_t hjo_advance(const hjo_problem *P, const double *V0, double *V, double *t,
                    double T_end, double cfl, int64_t max_steps, double *dts, int nthreads)
{
    int64_t ncell = hjo_cell_count(P);
    hjo_tables T;
    double *L = (double *)malloc(sizeof(double) * (size_t)ncell);
    double *Vn = (double *)malloc(sizeof(double) * (size_t)ncell);
    if (!L || !Vn || tables_init(P, &T)) {
        free(L);
        free(Vn);
        tables_free(&T);
        return -1;
    }
    int64_t s = 0;
    while (*t < T_end && s < max_steps) {
        double alpha_max[4];
        sweep_rate(P, &T, V, L, alpha_max, nthreads);
        double dt = hjo_cfl_dt(P, alpha_max, cfl);
        int last = (dt == 0.0) || (*t + dt >= T_end);
        if (last)
            dt = T_end - *t;
        sweep_update(ncell, V, V0, L, dt, Vn, nthreads);
        memcpy(V, Vn, sizeof(double) * (size_t)ncell);
        if (dts)
            dts[s] = dt;
        *t = last ? T_end : *t + dt;
        ++s;
    }
    free(L);
    free(Vn);
    tables_free(&T);
    return s;
}

/* Algorithm 2's convergence test (the printed test is inverted; reading:
 * keep stepping while the step changed V): from (V, *t), take steps as
 * hjo_advance does and stop after the first step whose largest change
 * max over the grid of |V_{n+1} - V_n| is below threshold, or at T_end, or
 * after max_steps steps.  *eps_last receives that largest change of the last
 * step (0 if none was taken) and *converged whether the test stopped the
 * loop.  Returns the steps taken, or -1 on allocation failure. */
int64_t hjo_advance_converged(const hjo_problem *P, const double *V0, double *V, double *t, double T_end,
                              double cfl, double threshold, int64_t max_steps, double *dts, int nthreads,
                              double *eps_last, int *converged)
{
    int64_t ncell = hjo_cell_count(P);
    double *Vprev = (double *)malloc(sizeof(double) * (size_t)ncell);
    if (!Vprev)
        return -1;
    int64_t s = 0;
    *eps_last = 0.0;
    *converged = 0;
    while (*t < T_end && s < max_steps) {
        memcpy(Vprev, V, sizeof(double) * (size_t)ncell);
        double dt = 0.0;
        if (hjo_advance(P, V0, V, t, T_end, cfl, 1, &dt, nthreads) != 1) {
            free(Vprev);
            return -1;
        }
        if (dts)
            dts[s] = dt;
        ++s;
        double eps = 0.0; /* epsilon = |V_{t+1} - V_t| in the max norm */
        for (int64_t c = 0; c < ncell; ++c)
            eps = fmax(eps, fabs(V[c] - Vprev[c]));
        *eps_last = eps;
        if (eps < threshold) {
            *converged = 1;
            break;
        }
    }
    free(Vprev);
    return s;
}

/* Whole BRT solve from t = 0: V_out = V(T).  Returns the step count. */
int64_t hjo_solve(const hjo_problem *P, const double *V0, double T_end, double cfl,
                  double *V_out, int64_t max_steps, double *dts, int nthreads)
{
    int64_t ncell = hjo_cell_count(P);
    double t = 0.0;
    memcpy(V_out, V0, sizeof(double) * (size_t)ncell);
    return hjo_advance(P, V0, V_out, &t, T_end, cfl, max_steps, dts, nthreads);
}

int hjo_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- Q5.27 fixed-point variant ------------------------------------------
 *
 * Sec. III-C and Sec. IV-B: the FPGA holds V in 32-bit two's-complement
 * fixed point with 5 integer bits (sign included) and 27 fractional bits,
 * value = q * 2^-27, range [-16, 16), resolution 2^-27.  The paper fixes the
 * data format only; the arithmetic inside the processing element is not
 * given.  Readings (each a single place below):
 *   - conversion from FP64: nearest, ties to even, saturated to the int32
 *     range; NaN and Inf are rejected                         (hjo_to_q527)
 *   - time step: the FP64 dt sequence of the FP64 scheme (the paper computes
 *     dt once on the host, Sec. II-B); t stays FP64
 *   - coefficients: each axis enters Algorithm 2 through dt |xdot_d| / dx_d
 *     (D+-_d carry 1/dx_d, the Euler step carries dt), held as an unsigned
 *     fixed-point weight with 30 fractional bits,
 *     W_d = nearest-even(2^30 * (dt * (|xdot_d| / dx_d))),
 *     and the sign of xdot_d                                  (q_weight)
 *   - arithmetic: differences, H and the dissipation are exact integers in
 *     units of 2^-27 * 2^-30 (nothing is rounded inside the cell); the Euler
 *     increment dt (H + diss) is rounded once to 2^-27, half up
 *     (floor(x + 1/2))                                        (q_cell)
 *   - ghosts: the linear extrapolation of the FP64 scheme, exact in integers
 *   - the BRT min against the converted V0, then saturation to the int32
 *     range.
 */

typedef __int128 hjo_i128;

/* floor(a / b) for b > 0 */
static hjo_i128 floor_div(hjo_i128 a, hjo_i128 b)
{
    hjo_i128 q = a / b;
    if (a % b != 0 && a < 0)
        q -= 1;
    return q;
}

/* Q5.27 code of x: nearest (ties to even), saturated.  Returns -1 for NaN
 * or Inf, else 0. */
int hjo_to_q527(const double *x, int64_t m, int32_t *q)
{
    for (int64_t i = 0; i < m; ++i) {
        if (!isfinite(x[i]))
            return -1;
        double s = nearbyint(ldexp(x[i], 27));
        if (s >= 2147483647.0)
            q[i] = INT32_MAX;
        else if (s <= -2147483648.0)
            q[i] = INT32_MIN;
        else
            q[i] = (int32_t)s;
    }
    return 0;
}

void hjo_from_q527(const int32_t *q, int64_t m, double *x)
{
    for (int64_t i = 0; i < m; ++i)
        x[i] = ldexp((double)q[i], -27);
}

/* Fixed-point weight of one axis: dt |xdot_d| / dx_d with 30 fractional bits. */
static int64_t q_weight(double dt, double xdot_abs, double h)
{
    return (int64_t)nearbyint(ldexp(dt * (xdot_abs / h), 30));
}

static int64_t q_ghost_value(const hjo_problem *P, const hjo_tables *T, const int32_t *Q,
                             int64_t c, const int idx[4], int d, int dir)
{
    int i = idx[d] + dir;
    int N = P->n[d];
    if (i >= 0 && i < N)
        return Q[c + dir * T->stride[d]];
    if (is_periodic(P, d)) {
        int w = (i + N) % N;
        return Q[c + (int64_t)(w - idx[d]) * T->stride[d]];
    }
    return 2 * (int64_t)Q[c] - (int64_t)Q[c - dir * T->stride[d]];
}

/* xdot_d of one cell before the control is chosen (the car's v, theta
 * components; the constant field) and |xdot_d| for the CFL sum. */
static void q_xdot_abs(const hjo_problem *P, const hjo_tables *T, const int idx[4], double a[4])
{
    if (P->dyn == HJO_DYN_CAR4D || P->dyn == HJO_DYN_CAR4D_STEER) {
        double v = T->v[idx[2]];
        a[0] = fabs(v * T->cos_th[idx[3]]);
        a[1] = fabs(v * T->sin_th[idx[3]]);
        a[2] = P->p[0];
        a[3] = P->dyn == HJO_DYN_CAR4D ? P->p[1] : fabs(v) * tan(P->p[1]) / P->p[2];
    } else {
        for (int d = 0; d < 4; ++d)
            a[d] = fabs(P->p[d]);
    }
}

/* Algorithm 2, lines 3-9 for one cell in fixed point: returns V_{t+1}. */
static int32_t q_cell(const hjo_problem *P, const hjo_tables *T, const int32_t *Q, const int32_t *Q0,
                      int64_t c, const int idx[4], double dt)
{
    int64_t Vc = Q[c];
    hjo_i128 twice = 0; /* 2 (H + diss) dt, units 2^-57 */
    double xa[4];
    q_xdot_abs(P, T, idx, xa);
    for (int d = 0; d < 4; ++d) {
        int64_t dm = Vc - q_ghost_value(P, T, Q, c, idx, d, -1); /* dx_d D-_d */
        int64_t dp = q_ghost_value(P, T, Q, c, idx, d, +1) - Vc; /* dx_d D+_d */
        int64_t W = q_weight(dt, xa[d], T->h[d]);                /* dt |xdot_d| / dx_d */
        int sgn;                                                  /* sign of xdot_d */
        if (P->dyn == HJO_DYN_CAR4D || P->dyn == HJO_DYN_CAR4D_STEER) {
            if (d == 0)
                sgn = T->v[idx[2]] * T->cos_th[idx[3]] >= 0.0 ? 1 : -1;
            else if (d == 1)
                sgn = T->v[idx[2]] * T->sin_th[idx[3]] >= 0.0 ? 1 : -1;
            else /* bang-bang control: the bound with the sign of p_d (tie: upper) */
                sgn = (dp + dm) >= 0 ? 1 : -1;
        } else {
            sgn = P->p[d] >= 0.0 ? 1 : -1;
        }
        /* H term p_d xdot_d = sgn W (D+ + D-)/2, dissipation W (D+ - D-)/2 */
        twice += (hjo_i128)sgn * W * (dp + dm);
        twice += (hjo_i128)W * (dp - dm);
    }
    /* twice is even: each axis contributes 2 W dp or -2 W dm */
    hjo_i128 inc = floor_div(twice / 2 + ((hjo_i128)1 << 29), (hjo_i128)1 << 30);
    hjo_i128 vn = (hjo_i128)Vc + inc;
    if (vn > Q0[c])
        vn = Q0[c];
    if (vn < INT32_MIN)
        vn = INT32_MIN;
    return (int32_t)vn;
}

/* Advance the Q5.27 grid Q (in place) from *t toward T_end, at most
 * max_steps steps; dts as in hjo_advance.  Returns the steps taken, or -1 on
 * allocation failure. */
int64_t hjo_advance_q527(const hjo_problem *P, const int32_t *Q0, int32_t *Q, double *t, double T_end,
                         double cfl, int64_t max_steps, double *dts, int nthreads)
{
    int64_t ncell = hjo_cell_count(P);
    hjo_tables T;
    int32_t *Qn = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncell);
    if (!Qn || tables_init(P, &T)) {
        free(Qn);
        tables_free(&T);
        return -1;
    }
    int N1 = P->n[0], N2 = P->n[1], N3 = P->n[2], N4 = P->n[3];
    (void)nthreads;
    int64_t s = 0;
    while (*t < T_end && s < max_steps) {
        /* alpha_d^max over the grid (Algorithm 1); |xdot_d| of the car does
         * not depend on V */
        double am[4] = {0.0, 0.0, 0.0, 0.0};
        for (int k = 0; k < N3; ++k)
            for (int l = 0; l < N4; ++l) {
                int idx[4] = {0, 0, k, l};
                double xa[4];
                q_xdot_abs(P, &T, idx, xa);
                for (int d = 0; d < 4; ++d)
                    am[d] = fmax(am[d], xa[d]);
            }
        double dt = hjo_cfl_dt(P, am, cfl);
        int last = (dt == 0.0) || (*t + dt >= T_end);
        if (last)
            dt = T_end - *t;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
        for (int i = 0; i < N1; ++i)
            for (int j = 0; j < N2; ++j)
                for (int k = 0; k < N3; ++k)
                    for (int l = 0; l < N4; ++l) {
                        int idx[4] = {i, j, k, l};
                        int64_t c = ((((int64_t)i * N2 + j) * N3 + k) * N4) + l;
                        Qn[c] = q_cell(P, &T, Q, Q0, c, idx, dt);
                    }
        memcpy(Q, Qn, sizeof(int32_t) * (size_t)ncell);
        if (dts)
            dts[s] = dt;
        *t = last ? T_end : *t + dt;
        ++s;
    }
    free(Qn);
    tables_free(&T);
    return s;
}

/* One fixed-point step of size dt at the listed cells (sampled parity). */
int hjo_step_cells_q527(const hjo_problem *P, const int32_t *Q, const int32_t *Q0, double dt,
                        const int64_t *cells, int64_t m, int32_t *out)
{
    hjo_tables T;
    if (tables_init(P, &T)) {
        tables_free(&T);
        return -1;
    }
    for (int64_t q = 0; q < m; ++q) {
        int idx[4];
        unflatten(P, cells[q], idx);
        out[q] = q_cell(P, &T, Q, Q0, cells[q], idx, dt);
    }
    tables_free(&T);
    return 0;
}

/* The convergence test of hjo_advance_converged on the Q5.27 grid: the
 * largest change is max |Q_{n+1} - Q_n| in codes, as the exact value
 * codes * 2^-27. */
int64_t hjo_advance_converged_q527(const hjo_problem *P, const int32_t *Q0, int32_t *Q, double *t, double T_end,
                                   double cfl, double threshold, int64_t max_steps, double *dts, int nthreads,
                                   double *eps_last, int *converged)
{
    int64_t ncell = hjo_cell_count(P);
    int32_t *Qprev = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncell);
    if (!Qprev)
        return -1;
    int64_t s = 0;
    *eps_last = 0.0;
    *converged = 0;
    while (*t < T_end && s < max_steps) {
        memcpy(Qprev, Q, sizeof(int32_t) * (size_t)ncell);
        double dt = 0.0;
        if (hjo_advance_q527(P, Q0, Q, t, T_end, cfl, 1, &dt, nthreads) != 1) {
            free(Qprev);
            return -1;
        }
        if (dts)
            dts[s] = dt;
        ++s;
        int64_t m = 0;
        for (int64_t c = 0; c < ncell; ++c) {
            int64_t d = (int64_t)Q[c] - (int64_t)Qprev[c];
            if (d < 0)
                d = -d;
            if (d > m)
                m = d;
        }
        *eps_last = ldexp((double)m, -27);
        if (*eps_last < threshold) {
            *converged = 1;
            break;
        }
    }
    free(Qprev);
    return s;
}

/* ---- query: V, grad V and u_opt at arbitrary states -------------------
 *
 * Sec. IV-A: near the BRT boundary (Eq. closetoboundary, V < 0.15) the car
 * applies u_opt = argmax_u grad V(z)^T f(z, u) (Eq. uopt_max) at its
 * current state z.  Readings (the paper does not say how V and grad V are
 * evaluated between grid points):
 *   - V(z): multilinear interpolation of the grid values over the cell that
 *     contains z (cell index floor((z_d - lo_d) / dx_d), the last cell for
 *     z_d at the upper end); theta wraps; states beyond a non-periodic axis
 *     are clamped onto it.
 *   - grad V(z): the gradient of that interpolant, i.e. on axis d the
 *     interpolation over the other three axes of (V(i_d + 1) - V(i_d)) / dx_d.
 *   - u_opt: the bang-bang argmax of Eq. uopt_max; ties (p_d = 0) take the
 *     upper bound, as in the step. */
static void query_cell(const hjo_problem *P, int d, double z, int *i0, double *f)
{
    int N = P->n[d];
    double h = hjo_spacing(P, d);
    double lo = P->lo[d];
    if (is_periodic(P, d)) {
        double span = h * (double)N;
        double u = fmod(z - lo, span);
        if (u < 0.0)
            u += span;
        double r = u / h;
        int i = (int)floor(r);
        if (i >= N)
            i = N - 1;
        *i0 = i;
        *f = r - (double)i;
        return;
    }
    double r = (z - lo) / h;
    if (r <= 0.0) {
        *i0 = 0;
        *f = 0.0;
        return;
    }
    if (r >= (double)(N - 1)) {
        *i0 = N - 2;
        *f = 1.0;
        return;
    }
    int i = (int)floor(r);
    if (i > N - 2)
        i = N - 2;
    *i0 = i;
    *f = r - (double)i;
}

int hjo_query(const hjo_problem *P, const double *V, const double *states, int64_t m, double *value,
              double *grad, double *control)
{
    int64_t stride[4];
    stride[3] = 1;
    stride[2] = P->n[3];
    stride[1] = (int64_t)P->n[2] * P->n[3];
    stride[0] = (int64_t)P->n[1] * P->n[2] * P->n[3];
    for (int64_t q = 0; q < m; ++q) {
        int i0[4], i1[4];
        double f[4];
        for (int d = 0; d < 4; ++d) {
            query_cell(P, d, states[4 * q + d], &i0[d], &f[d]);
            i1[d] = i0[d] + 1;
            if (i1[d] >= P->n[d])
                i1[d] = is_periodic(P, d) ? 0 : P->n[d] - 1;
        }
        /* the 16 corners: bit d of c picks i1 on axis d */
        double val = 0.0, g[4] = {0.0, 0.0, 0.0, 0.0};
        for (int c = 0; c < 16; ++c) {
            int64_t off = 0;
            double w = 1.0;
            for (int d = 0; d < 4; ++d) {
                int hi = (c >> d) & 1;
                off += (int64_t)(hi ? i1[d] : i0[d]) * stride[d];
                w *= hi ? f[d] : 1.0 - f[d];
            }
            val += w * V[off];
            for (int d = 0; d < 4; ++d) {
                /* d/dz_d of the weight: the other factors times +-1/dx_d */
                double wd = ((c >> d) & 1) ? 1.0 : -1.0;
                for (int e = 0; e < 4; ++e)
                    if (e != d)
                        wd *= ((c >> e) & 1) ? f[e] : 1.0 - f[e];
                g[d] += wd * V[off] / hjo_spacing(P, d);
            }
        }
        value[q] = val;
        if (grad)
            for (int d = 0; d < 4; ++d)
                grad[4 * q + d] = g[d];
        if (control) {
            double v = states[4 * q + 2];
            if (P->dyn == HJO_DYN_CAR4D) {
                control[2 * q] = g[2] >= 0.0 ? P->p[0] : -P->p[0];
                control[2 * q + 1] = g[3] >= 0.0 ? P->p[1] : -P->p[1];
            } else if (P->dyn == HJO_DYN_CAR4D_STEER) {
                control[2 * q] = g[2] >= 0.0 ? P->p[0] : -P->p[0];
                control[2 * q + 1] = g[3] * v >= 0.0 ? P->p[1] : -P->p[1];
            } else {
                control[2 * q] = 0.0;
                control[2 * q + 1] = 0.0;
            }
        }
    }
    return 0;
}
