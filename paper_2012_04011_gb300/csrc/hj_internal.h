// Internal declarations of libhj shared by its translation units.
// Nothing here is part of the C ABI (include/hj.h).
#pragma once

#include <cuda.h>  // CUtensorMap (type only; the driver is reached through cudaGetDriverEntryPointByVersion)
#include <cuda_runtime.h>
#include <stdint.h>

#include "hj.h"

// Per-axis treatment of the upwind side on axes 3 and 4 (v and theta).
enum HjAxisMode : int32_t {
    HJ_AXIS_CONTROL = 0,  // bang-bang control: u_opt follows the sign of the costate, so the
                          // upwind value is max(V+, V-)  (Alg. 2, u_opt = argmax)
    HJ_AXIS_PLUS = 1,     // fixed velocity >= 0: upwind value is V+
    HJ_AXIS_MINUS = 2     // fixed velocity < 0: upwind value is V-
};

// Device-resident time-loop state of one grid.  Written by the prologue
// kernel and by the last CTA of every step kernel ("finaliser"), read by the
// next kernel on the same stream.
struct HjDevState {
    double t;                          // simulated time at the start of the next step
    double dt;                         // size of the next step
    double dt_prev;                    // size of the step just taken
    double T;                          // horizon of the current call
    double cfl;                        // Courant number of the current call
    long long n;                       // steps since V0 was set
    int last;                          // the next step is cut to land on T
    int done;                          // t has reached T: step kernels exit at once
    unsigned long long alpha_bits[2];  // running max of |xdot_1|, |xdot_2| of this step (FP64 bit patterns)
    double alpha_prev[4];              // alpha_d^max reduced by the last step (or the prologue)
    unsigned int blocks_done;          // CTAs of the current step that have finished
    int status;                        // hj_status raised on the device (HJ_OK if none)
    int nonfinite;                     // ingest saw a NaN or Inf
    int alpha_stale;                   // dynamics changed: the next prologue re-reduces alpha^max
    double dt_scaled;                  // dt the FP64 dt-scaled coefficient table holds (0: none yet)
    int track;                         // convergence mode: the steps reduce max |V_{n+1} - V_n|
    int converged;                     // the last step changed V by less than the threshold
    double threshold;                  // convergence threshold of the current call
    unsigned long long delta_bits;     // running max |V_{n+1} - V_n| of this step (FP64 bit pattern)
    double delta_last;                 // max |V_{n+1} - V_n| of the step just taken (convergence mode)
};

// FP64 coefficients with dt folded in (per (v, theta)): w1 = dt xdot_1/dx_1,
// w2 = dt xdot_2/dx_2 (signed: the sign picks the upwind side), w0 = 1 - dt
// (|xdot_1|/dx_1 + |xdot_2|/dx_2 + k3 + k4(v)), w4 = dt k4(v).  V_new = w0 V_c +
// |w1| V_up1 + |w2| V_up2 + dt k3 V_up3 + w4 V_up4.
struct HjScaledCoef {
    double w1, w2, w0, w4;  // w4 = dt |xdot_4| / dx_4 (depends on v for the steering car)
};

// Device-side bookkeeping of the resident step kernel: the grid barrier's
// arrival counter and three rotating slots of the per-step largest change
// of V (convergence mode; FP64 bit patterns).  Zeroed before every resident
// launch.
struct HjResidentSync {
    unsigned int count;
    unsigned int unused;
    unsigned long long slot[3];
};

// Grid geometry handed to kernels by value.
struct HjGeom {
    int32_t n1, n2, n3, n4;  // points per axis
    int32_t p4;              // internal row pitch along theta (n4 rounded up to a multiple of 4)
    int32_t periodic;        // bit d: axis d periodic
    int32_t mode3, mode4;    // HjAxisMode of axes 3 and 4
    double h[4];             // grid spacing dx_d (FP64, as the API defines it)
    double k3, k4;           // |xdot_3|/dx_3 and |xdot_4|/dx_4 (constant over the grid)
    double alpha3, alpha4;   // |xdot_3|, |xdot_4| (constant over the grid)
};

// Per-(v, theta) coefficients: c1 = xdot_1/dx_1, c2 = xdot_2/dx_2 (signed),
// ks = |c1| + |c2| + k3 + k4 in the working precision; a1 = |xdot_1|,
// a2 = |xdot_2| in FP64 for every precision, so that alpha^max, and with it
// the dt sequence of Algorithm 1, is the FP64 one whatever V is stored in.
template <typename T>
struct HjCoef {
    T c1, c2, ks;
    double a1, a2;
};

struct hj_grid {
    int32_t n[4];
    int32_t p4;
    double lo[4], hi[4], h[4];
    uint32_t periodic;
    hj_precision prec;
    size_t esize;          // bytes per value on the device
    long long ncell;       // n1*n2*n3*n4
    long long nint;        // n1*n2*n3*p4 (internal values per array)
    cudaStream_t stream;
    bool own_stream;
    cudaEvent_t ev_in;  // own stream: orders device inputs after the legacy default stream
    int device;

    void *v0;              // V0 (internal layout)
    void *buf;             // two ping-pong buffers, back to back (2*nint values)
    void *coef;            // HjCoef<T>[n3*n4]
    HjScaledCoef *scaled;  // FP64 grids: dt-scaled coefficients [n3*n4]
    int32_t *qw;           // Q5.27 grids: fixed-point axis weights (hj_rescale_qweights)
    void *k4tab;           // theta coefficient per speed: |xdot_4|/dx_4 (double[n3]; FP32 grids: float2[n3] of
                           // (k4, -(k3 + k4)))
    void *v0xy;            // V0 as an N1 x N2 field (element type of the grid), when V0 depends on x, y only
    bool v0_bcast;         // V0 was set from the (x, y) field: the tiled kernel reads v0xy
    bool track;            // a convergence-mode call is running: launch the kernels that reduce the change
    float *tab_tiled;      // tiled-kernel tables: v_k [n3], cos/dx1 [p4], sin/dx2 [p4], quad signs [p4]
    double2 *amax_q;       // per (v_k, theta quad q) [n3][p4 / 4]: the largest FP64 |xdot_1|, |xdot_2| over the
                           // quad's headings (the tiled kernel's alpha^max partials, one load per work item)
    HjDevState *dstate;
    HjDevState *hstate;    // pinned host mirror

    bool has_dyn, has_value;
    hj_dynamics dyn;
    double params[4];
    HjGeom geom;

    hj_kernel kernel_req;  // requested by hj_set_kernel
    bool tiled_ok;         // the tiled kernel supports this grid
    CUtensorMap tmap[4];   // V0, buffer A, buffer B with the halo box; V0 with the tile box (tiled kernel)
    int32_t tile_req[4];   // requested (ty, tv, xc, stages); 0 = choose automatically
    int32_t tile_ty, tile_tv, tile_xc, tile_stages;
    int32_t tiled_ctas, tiled_per_sm;
    bool tiled_usign;      // every theta quad has one sign of cos and of sin

    cudaEvent_t ev[4];
    // CUDA graphs of k back-to-back step launches (small grids, where the
    // launches cost more than the steps); kernel parameters are captured by
    // value, so a graph is valid while `launch_version` is unchanged
    struct StepGraph {
        long long k;
        int kernel, track;
        unsigned version;
        cudaGraphExec_t exec;
    } graphs[4];
    unsigned launch_version;  // bumped whenever a step kernel's parameters may change
    unsigned graph_tick;
    HjResidentSync *rsync;    // resident kernel bookkeeping (allocated on first use)
    size_t device_bytes;
};

// Launchers (each returns the CUDA error of its launch).
cudaError_t hj_launch_step_generic(hj_grid *g);
cudaError_t hj_launch_step_tiled(hj_grid *g);
// Up to k steps in one cooperative launch of the resident kernel (it stops
// early when the time loop is done); allocates g->rsync on first use.
cudaError_t hj_launch_step_resident(hj_grid *g, long long k);
// Whether the device can run the resident kernel (cooperative launch).
bool hj_resident_supported(const hj_grid *g);
// Set up the tiled kernel for g (tensor maps, tile shape); false if unsupported.
bool hj_tiled_setup(hj_grid *g, char *why, size_t why_len);
// Consumer threads a tile of ty x tv rows needs (one per row and theta quad),
// and whether that shape can run at all.
int hj_tiled_threads(const hj_grid *g, int ty, int tv);
// Consumer threads of the tiled kernel's launch-bound class i (0..3), per precision.
int hj_tiled_variant(bool fixed, int i);

// cos and sin of grid headings for the FP32 tables: values below 1e-12 are
// rounding artefacts of theta_l = lo + l dx at +-pi/2, 0, +-pi (the next
// smallest |cos| or |sin| on a grid of at most 4096 headings is ~1.5e-3), and
// are set to exactly 0 so that every FP32 kernel uses the same upwind side.
static inline double hj_flush_trig(double x) { return (x < 1e-12 && x > -1e-12) ? 0.0 : x; }

// Query kernel (hj_query.cu): value, gradient and u_opt of V (the grid's
// current value array, internal layout) at m states; grad and control may be
// NULL.  Device pointers; runs on the grid's stream.
cudaError_t hj_launch_query(const hj_grid *g, const void *V, const double *states, long long m, double *value,
                            double *grad, double *control);

// Sets the message hj_last_error() returns on this host thread.
void hj_internal_set_error(const char *msg);

// Ingest (dense FP64/FP32 -> padded FP32 rows), readback (padded FP32 rows
// [row0, row0 + nrows) -> dense FP64/FP32) and the solve prologue, for the
// batch API.
cudaError_t hj_launch_ingest_f32(const void *src, hj_precision src_type, float *dst, int n4, int p4, long long nrows,
                                 int *nonfinite, cudaStream_t stream);
cudaError_t hj_launch_ingest_xy_f32(const double *src_dev, float *dst, int n3, int n4, int p4, long long nxy,
                                    int *nonfinite, cudaStream_t stream);
cudaError_t hj_launch_readback_f32(const float *src, void *dst, hj_precision dst_type, int n4, int p4, long long row0,
                                   long long nrows, cudaStream_t stream);
cudaError_t hj_launch_prologue_f32(HjDevState *st, const HjGeom &g, const HjCoef<float> *coef, int ncoef, double T,
                                   double cfl, cudaStream_t stream);

// Rescale the FP64 coefficient table for dt (all threads of one block call
// it; the table covers n3 * n4 entries; k4 holds the theta coefficient of
// each speed).
// One entry of that table: coefficients c of a (v, theta), theta
// coefficient k4 of the speed.
__device__ __forceinline__ HjScaledCoef hj_scaled_entry(const HjCoef<double> &c, double k4, double dt)
{
    HjScaledCoef o;
    o.w1 = dt * c.c1;
    o.w2 = dt * c.c2;
    o.w0 = 1.0 - dt * c.ks;
    o.w4 = dt * k4;
    return o;
}

__device__ __forceinline__ void hj_rescale_table(HjScaledCoef *sc, const HjCoef<double> *coef, const double *k4,
                                                 int n3, int n4, double dt)
{
    for (int i = threadIdx.x; i < n3 * n4; i += blockDim.x) sc[i] = hj_scaled_entry(coef[i], k4[i / n4], dt);
}

// ---- Q5.27 fixed point (Sec. III-C, Sec. IV-B): int32 codes q, value q 2^-27

constexpr double HJ_Q527_SCALE = 134217728.0;  // 2^27
constexpr double HJ_QW_SCALE = 1073741824.0;   // 2^30: fractional bits of the axis weights

// Code of x: nearest, ties to even, saturated to the int32 range.
__device__ __forceinline__ int32_t hj_q527_from_f64(double x)
{
    const long long q = __double2ll_rn(__dmul_rn(x, HJ_Q527_SCALE));  // the product is exact
    return (int32_t)(q > 2147483647LL ? 2147483647LL : (q < -2147483648LL ? -2147483648LL : q));
}

// Exact value of a code.
__device__ __forceinline__ double hj_q527_to_f64(int32_t q) { return (double)q * (1.0 / HJ_Q527_SCALE); }

// Axis weight dt k (k = |xdot_d| / dx_d) with 30 fractional bits: nearest,
// ties to even, of the FP64 product (dt k <= Courant number <= 1).
__device__ __forceinline__ int32_t hj_qweight(double dt, double k)
{
    return (int32_t)__double2ll_rn(__dmul_rn(__dmul_rn(dt, k), HJ_QW_SCALE));
}

// Fixed-point weights for dt (all threads of one block call it):
//   qw[k p4 + l]            x weight of (v_k, theta_l), signed with xdot_1
//   qw[n3 p4 + k p4 + l]    y weight, signed with xdot_2
//   qw[2 n3 p4]             v weight (constant over the grid)
//   qw[2 n3 p4 + 4 + k]     theta weight of speed v_k
// Pad lanes (l >= n4) get 0.
constexpr int HJ_QW_TAIL = 4;  // entries between the y weights and the per-speed theta weights
__device__ __forceinline__ void hj_rescale_qweights(int32_t *qw, const HjCoef<double> *coef, int n3, int n4, int p4,
                                                    double k3, const double *k4, double dt)
{
    const int tot = n3 * p4;
    for (int i = threadIdx.x; i < tot; i += blockDim.x) {
        const int k = i / p4, l = i - (i / p4) * p4;
        int32_t w1 = 0, w2 = 0;
        if (l < n4) {
            const HjCoef<double> c = coef[k * n4 + l];
            w1 = hj_qweight(dt, fabs(c.c1));
            w2 = hj_qweight(dt, fabs(c.c2));
            if (c.c1 < 0.0) w1 = -w1;
            if (c.c2 < 0.0) w2 = -w2;
        }
        qw[i] = w1;
        qw[tot + i] = w2;
    }
    for (int k = threadIdx.x; k < n3; k += blockDim.x) qw[2 * tot + HJ_QW_TAIL + k] = hj_qweight(dt, k4[k]);
    if (threadIdx.x == 0) {
        qw[2 * tot] = hj_qweight(dt, k3);
        qw[2 * tot + 1] = 0;
    }
}

// Interior form of the same update (no extrapolated ghost on any axis):
// sum_d W_d (V_up,d - V_c) = sum_d W_d V_up,d - S V_c with S = sum_d W_d, all
// operands int32, so five 32x32->64 multiply-adds give the exact sum.
// nsum = -S; the rounding offset 2^29 starts the accumulator.
__device__ __forceinline__ int32_t hj_q527_update_interior(int32_t vc, int32_t v0, int32_t u1, int32_t u2, int32_t u3,
                                                           int32_t u4, int32_t w1, int32_t w2, int32_t w3, int32_t w4,
                                                           int32_t nsum)
{
    // three short chains instead of one long one (the sum is exact in any order)
    const long long a = (long long)nsum * vc + (long long)w1 * u1;
    const long long b = (long long)w2 * u2 + (long long)w3 * u3;
    const long long c = (long long)w4 * u4 + (1LL << 29);
    const long long acc = a + b + c;
    long long vn = (long long)vc + (acc >> 30);
    vn = vn < (long long)v0 ? vn : (long long)v0;
    return (int32_t)(vn < -2147483648LL ? -2147483648LL : vn);
}

// The same interior update when the weights sum to at most 2^30 (nsum >=
// -2^30; a Courant number below 1 guarantees it).  Then the increment
// floor((sum W_d (u_d - V_c) + 2^29) / 2^30) lies between the smallest and
// the largest of u_d - V_c and 0, so V_c plus it lies between the smallest and
// the largest of V_c and the u_d: it fits int32, needs no saturation, and
// the low 32 bits of the shifted sum, added to V_c modulo 2^32, are exact.
__device__ __forceinline__ int32_t hj_q527_update_interior32(int32_t vc, int32_t v0, int32_t u1, int32_t u2,
                                                             int32_t u3, int32_t u4, int32_t w1, int32_t w2,
                                                             int32_t w3, int32_t w4, int32_t nsum)
{
    long long acc = (long long)nsum * vc + (1LL << 29);
    acc += (long long)w1 * u1;
    acc += (long long)w2 * u2;
    acc += (long long)w3 * u3;
    acc += (long long)w4 * u4;
    const uint32_t inc = __funnelshift_r((uint32_t)acc, (uint32_t)((unsigned long long)acc >> 32), 30);
    const int32_t vn = (int32_t)((uint32_t)vc + inc);
    return vn < v0 ? vn : v0;
}

// One fixed-point cell update from the upwind differences d_d = V_up,d - V_c
// (exact, int64) and the weight magnitudes: V_c + floor((sum W_d d_d + 2^29)
// / 2^30), then the BRT min with V0 and saturation below.
__device__ __forceinline__ int32_t hj_q527_update(int32_t vc, int32_t v0, long long d1, long long d2, long long d3,
                                                  long long d4, int32_t w1, int32_t w2, int32_t w3, int32_t w4)
{
    long long acc = (long long)w1 * d1;
    acc += (long long)w2 * d2;
    acc += (long long)w3 * d3;
    acc += (long long)w4 * d4;
    long long vn = (long long)vc + ((acc + (1LL << 29)) >> 30);  // arithmetic shift: floor
    vn = vn < (long long)v0 ? vn : (long long)v0;
    return (int32_t)(vn < -2147483648LL ? -2147483648LL : vn);
}

// Batch internals for the server: pull all slot states once, then query the
// host copy (done flag and step count of a slot).
hj_status hj_batch_refresh(hj_batch *b);
bool hj_batch_cached_done(const hj_batch *b, int32_t slot, int64_t *steps);

// Pointer of the value buffer that holds V after n steps.
inline void *hj_value_ptr(const hj_grid *g, long long n)
{
    if (n == 0) return g->v0;
    char *base = (char *)g->buf;
    return base + ((n - 1) & 1) * (size_t)g->nint * g->esize;
}
