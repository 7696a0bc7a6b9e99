/*
 * libhj — GB300 (sm_103a) time stepping of the Hamilton-Jacobi reachability
 * PDE on a dense 4D grid, computing the Backward Reachable Tube (BRT) of the
 * 4D car of arxiv 2012.04011 ("Real-Time Formal Verification of Autonomous
 * Systems With An FPGA").
 *
 * Plain C ABI: status codes returned by value, plain pointers and sizes, no
 * C++ or framework types.  No exception and no exit() crosses this boundary.
 *
 * Problem (Sec. II-A): dynamics z' = f(z, u) (Eq. main_ode, no disturbance),
 * target set T = {z : V0(z) <= 0} given by an implicit surface V0
 * (Sec. II-A; Eq. init_V for round obstacles), and the BRT as the sub-zero
 * level set of the value function V of Eq. eq3, the viscosity solution of the
 * HJ variational inequality (Eq. HJ_variational_inequality).
 *
 * Scheme (Sec. II-B): one-sided differences D-, D+ and their mean on every
 * axis (Eq. central_diff) with extrapolated points at the ends of
 * non-periodic axes; u_opt = argmax_u grad(V).f (bang-bang); Lax-Friedrichs
 * Hamiltonian with the local dissipation alpha_d = |xdot_d| (Algorithm 2);
 * CFL step dt = CFL / sum_d alpha_d^max / dx_d from max reductions over the
 * grid (Algorithm 1); forward Euler; V <- min(V0, V) after every step
 * (Algorithms 1-2).  Time runs from t = 0 to the horizon T; the last step is
 * cut so that t lands on T.
 *
 * Grid layout everywhere in this API: row-major [N1][N2][N3][N4] over the
 * axes (x, y, v, theta), theta (axis 4) fastest, matching the loop order
 * i, j, k, l of Algorithms 1-2.  Non-periodic axes include both end points:
 * x_i = lo + i (hi - lo)/(N - 1).  A periodic axis of N points covers
 * [lo, hi): x_i = lo + i (hi - lo)/N.
 *
 * Call order: hj_create_grid -> hj_set_dynamics -> hj_set_initial_value[_device]
 * -> hj_solve_brt / hj_advance_brt (repeatable: each call continues from the
 * current (V, t)) -> hj_read_value[_device] -> hj_destroy_grid.
 *
 * Threading: a grid is not thread safe; different grids may be used from
 * different host threads.  All device work of a grid runs on the grid's
 * stream.  The calls below block until their device work is complete unless
 * stated otherwise.
 *
 * Caller-owned device arrays (the *_device calls, of grids and batches): on a
 * caller's stream they are ordered by that stream.  A grid or batch on its own
 * stream first waits, without blocking the host, for the work already queued
 * on the legacy default stream (where PyTorch's default stream and callers
 * that name no stream run); work on any other stream that writes or reads
 * such an array must be complete before the call.
 */
#ifndef HJ_H
#define HJ_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HJ_API __attribute__((visibility("default")))
#else
#define HJ_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hj_grid hj_grid; /* opaque; created and freed by the library */

typedef enum {
    HJ_OK = 0,
    HJ_ERR_INVALID_ARG = 1, /* a bad size, bound, pointer, count or a non-finite value */
    HJ_ERR_STATE = 2,       /* call out of order (e.g. solving before V0 is set) */
    HJ_ERR_OOM = 3,         /* device or host allocation failed */
    HJ_ERR_CUDA = 4,        /* a CUDA runtime or driver call failed (message: hj_last_error) */
    HJ_ERR_UNSTABLE = 5,    /* the CFL step came out non-finite or non-positive */
    HJ_ERR_TIMEOUT = 6,     /* a device-side wait ran out of time; the grid must be destroyed */
    HJ_ERR_UNSUPPORTED = 7  /* valid request this build does not implement */
} hj_status;

/* Arithmetic of the value function on the device (and the element type of
 * device arrays passed with a dtype).
 *   HJ_FP64, HJ_FP32: IEEE double / float.
 *   HJ_Q527: the FPGA's fixed-point format (Sec. III-C, Sec. IV-B): int32
 *     codes q with value q * 2^-27 (5 integer bits including the sign, 27
 *     fractional bits; range [-16, 16), resolution 2^-27).  Conversion from
 *     floating point: nearest, ties to even, saturated to the int32 range;
 *     conversion back is exact.  One step per cell: the upwind differences,
 *     H and the dissipation of Algorithm 2 are exact integers; each axis is
 *     weighted by dt |xdot_d| / dx_d held with 30 fractional bits (nearest,
 *     ties to even, from the FP64 dt); the Euler increment is rounded once
 *     to 2^-27, half up; then the BRT min with V0 and saturation.  dt and t
 *     are FP64 as for the other precisions. */
typedef enum { HJ_FP64 = 0, HJ_FP32 = 1, HJ_Q527 = 2 } hj_precision;

typedef enum {
    /* Sec. IV-A car with the heading rate as a bounded control:
     * x' = v cos(th), y' = v sin(th), v' = a, th' = w; |a| <= p[0] (a_max),
     * |w| <= p[1] (w_max).  Axes must be (x, y, v, theta). */
    HJ_DYN_CAR4D = 0,
    /* Constant velocity xdot = (p[0], p[1], p[2], p[3]), no control
     * (closed-form test cases). */
    HJ_DYN_CONST = 1,
    /* The car of Eq. car_dynamics as printed in Sec. IV-A, steered by the
     * wheel angle: x' = v cos(th), y' = v sin(th), v' = a,
     * th' = v tan(delta) / L; |a| <= p[0] (a_max), |delta| <= p[1]
     * (delta_max, 0 <= delta_max < pi/2), p[2] = L > 0 (the paper: 1.5,
     * pi/18, 0.3 m).  The heading rate bound is |v| tan(delta_max) / L, so
     * the theta dissipation varies with the speed. */
    HJ_DYN_CAR4D_STEER = 2
} hj_dynamics;

/* Step-kernel selection.  HJ_KERNEL_AUTO picks, by measured speed:
 * HJ_KERNEL_RESIDENT for FP32 grids of up to 4 M cells and Q5.27 grids of up
 * to 8 M cells, else HJ_KERNEL_TILED where it supports the grid, else
 * HJ_KERNEL_GENERIC (always for FP64 grids). */
typedef enum {
    HJ_KERNEL_AUTO = 0,
    HJ_KERNEL_GENERIC = 1, /* one thread per cell, loads through L1/L2 */
    HJ_KERNEL_TILED = 2,   /* FP32, Q5.27 car grids (theta periodic, x, y, v not; theta rows of at
                            * most 256 points; every size the API accepts): TMA-staged 4D tiles
                            * streamed along x */
    HJ_KERNEL_RESIDENT = 3 /* the per-cell update of HJ_KERNEL_GENERIC (identical results, any
                            * precision and grid of fewer than 2^32 values whose coefficient
                            * tables fit in shared memory), the whole time loop in one
                            * cooperative launch with a grid barrier between steps; a barrier
                            * wait that runs out (2 s) ends the call with HJ_ERR_TIMEOUT */
} hj_kernel;

typedef struct {
    int64_t steps;         /* steps taken by this call */
    int64_t total_steps;   /* steps since the last hj_set_initial_value */
    double t_final;        /* simulated time reached */
    double dt_first;       /* dt of the first step of this call (0 if none) */
    double dt_last;        /* dt of the last step of this call (0 if none) */
    double alpha_max[4];   /* alpha_d^max reduced by the last step (|xdot_d| maxima) */
    double device_ms;      /* device time of the whole call (CUDA events) */
    double loop_ms;        /* device time of the time loop only (step kernels) */
    int32_t kernel;        /* hj_kernel actually used */
    int32_t launches;      /* kernels launched by this call */
    double last_change;    /* hj_solve_converged: max |V_{n+1} - V_n| of the last step (0 otherwise) */
    int32_t converged;     /* hj_solve_converged: the convergence test ended the loop */
} hj_solve_stats;

/* One tile shape of the tiled kernel and its measured step time. */
typedef struct {
    int32_t shape[4];      /* rows along y, rows along v, x planes per work item, smem ring stages */
    int32_t threads;       /* threads per CTA */
    int32_t ctas;          /* CTAs per launch */
    double ms_per_step;    /* mean device time of one step kernel (CUDA events) */
    double ms_retimed;     /* the second, longer trial's time (0: not re-timed) */
} hj_tile_result;

typedef struct {
    int32_t n[4];
    int32_t pitch4;        /* internal row pitch along theta (N4 rounded up) */
    int32_t precision;     /* hj_precision */
    int32_t kernel;        /* hj_kernel that hj_solve_brt will use */
    double lo[4], hi[4], dx[4];
    uint32_t periodic_mask;
    int32_t has_value;     /* V0 has been set */
    int64_t total_steps;
    double t;
    size_t device_bytes;   /* device memory held by the grid */
    int32_t tile[4];       /* tiled kernel shape in use (zeros if the tiled kernel is unavailable) */
    int32_t tile_ctas;     /* CTAs per tiled step launch */
    int32_t v0_broadcast;  /* 1: V0 was set from its (x, y) field and the tiled kernel reads that field */
} hj_grid_info;

/* Create a grid of n[0]*n[1]*n[2]*n[3] cells on the current CUDA device.
 *   n:             points per axis; N_d >= 3 on every axis; N4 <= 4096.
 *   lo, hi:        axis bounds, finite, hi > lo.
 *   periodic_mask: bit d set makes axis d periodic (bit 3 = theta).
 *   prec:          arithmetic of the value function on the device; the
 *                  simulated time and dt are always FP64.
 *   cuda_stream:   a cudaStream_t to run on (e.g. a PyTorch stream), or NULL
 *                  for a stream owned by the grid.  The caller keeps a passed
 *                  stream alive until hj_destroy_grid.
 *   out:           receives the grid; written only on HJ_OK.
 * Allocates three device arrays (V0 and two ping-pong buffers) of
 * n1*n2*n3*pitch4 values each. */
HJ_API hj_status hj_create_grid(const int32_t n[4], const double lo[4], const double hi[4],
                         uint32_t periodic_mask, hj_precision prec, void *cuda_stream,
                         hj_grid **out);

/* Set the dynamics (Eq. main_ode; car: Eq. car_dynamics of Sec. IV-A with
 * th' = w, or with the steering angle).  params: HJ_DYN_CAR4D {a_max >= 0,
 * w_max >= 0}; HJ_DYN_CONST {c1, c2, c3, c4}; HJ_DYN_CAR4D_STEER {a_max >= 0,
 * 0 <= delta_max < pi/2, L > 0}.  nparams must match (2, 4 or 3), values
 * finite.
 * Uploads the (v, theta) state tables once (Sec. III-A keeps the state
 * vectors and cos/sin of theta in small on-chip look-up tables). */
HJ_API hj_status hj_set_dynamics(hj_grid *g, hj_dynamics kind, const double *params, int32_t nparams);

/* Initial value V0 (Sec. II-A, target set {V0 <= 0}) from a HOST array of
 * count = N1*N2*N3*N4 doubles in the layout above.  The library copies it
 * (the caller keeps ownership) and resets t = 0, V = V0.  Non-finite values
 * give HJ_ERR_INVALID_ARG (checked on the device).  Pinned host memory makes
 * the copy faster; pageable memory works. */
HJ_API hj_status hj_set_initial_value(hj_grid *g, const double *v0, size_t count);

/* As hj_set_initial_value for a V0 that depends on position only (as Eq.
 * init_V does): v0_xy is a host array of count = N1*N2 doubles, row-major
 * [N1][N2], replicated over v and theta on the device.  The grid also keeps
 * the field itself, and the tiled step kernel then reads V0 from it
 * (8 instead of 12 bytes of HBM traffic per FP32 / Q5.27 cell-update; same
 * results bit for bit).  Any other hj_set_initial_value* call switches back
 * to the full 4D V0. */
HJ_API hj_status hj_set_initial_value_xy(hj_grid *g, const double *v0_xy, size_t count);

/* As hj_set_initial_value_xy from a DEVICE array of count = N1*N2 values of
 * dtype (HJ_FP64, HJ_FP32 or HJ_Q527 codes) on the grid's device; read on
 * the grid's stream; the caller keeps ownership. */
HJ_API hj_status hj_set_initial_value_xy_device(hj_grid *g, const void *v0_xy_device, hj_precision dtype,
                                                size_t count);

/* As hj_set_initial_value, from a DEVICE array (dtype HJ_FP64 = double,
 * HJ_FP32 = float, HJ_Q527 = int32 codes) of count values on the grid's
 * device, dense layout above, converted to the grid's precision.  The array
 * is read on the grid's stream; the caller keeps ownership. */
HJ_API hj_status hj_set_initial_value_device(hj_grid *g, const void *v0_device, hj_precision dtype,
                                      size_t count);

/* Integrate from the current time to the horizon T (T >= 0, finite) with
 * Courant number cfl (0 < cfl <= 1).  T <= current t is a no-op returning
 * HJ_OK.  stats may be NULL.  HJ_ERR_STATE without dynamics or V0. */
HJ_API hj_status hj_solve_brt(hj_grid *g, double T, double cfl, hj_solve_stats *stats);

/* As hj_solve_brt but takes at most max_steps (>= 0) steps toward T; a later
 * call continues.  Lets a caller bound the work of one call. */
HJ_API hj_status hj_advance_brt(hj_grid *g, double T, double cfl, int64_t max_steps,
                         hj_solve_stats *stats);

/* Algorithm 2's convergence test (the printed test is inverted; read as:
 * keep stepping while a step changes V): integrate from the current (V, t)
 * and stop after the first step whose largest change over the grid,
 * max |V_{n+1} - V_n| (in the grid's precision, exact for Q5.27), is below
 * threshold (> 0, finite), or when t reaches T_max, or after max_steps
 * steps.  stats->converged says whether the test ended the loop and
 * stats->last_change gives that step's largest change.  Same steps, dt and
 * results as hj_advance_brt otherwise. */
HJ_API hj_status hj_solve_converged(hj_grid *g, double threshold, double T_max, double cfl, int64_t max_steps,
                                    hj_solve_stats *stats);

/* Copy the current V into a HOST buffer of count = N1*N2*N3*N4 doubles
 * (caller-owned), layout above (exact for every precision). */
HJ_API hj_status hj_read_value(const hj_grid *g, double *out, size_t count);

/* Copy the current V into a DEVICE buffer of count values of dtype
 * (HJ_FP64, HJ_FP32 or HJ_Q527), layout above, converted from the grid's
 * precision as for the ingest; caller-owned.  Runs on the grid's stream;
 * returns once the copy is queued and completed. */
HJ_API hj_status hj_read_value_device(const hj_grid *g, void *out_device, hj_precision dtype,
                               size_t count);

/* V, grad V and the optimal control at m arbitrary states, from the grid's
 * current V: the controller of Sec. IV-A, which applies
 * u_opt = argmax_u grad V^T f (Eq. uopt_max) when V < 0.15 at the car's
 * state (Eq. closetoboundary).  The paper does not say how V is evaluated
 * between grid points; here:
 *   - value[i]: multilinear interpolation of the grid values over the cell
 *     that contains states[i] (cell floor((z_d - lo_d)/dx_d); theta wraps;
 *     a coordinate beyond a non-periodic axis is clamped onto it);
 *   - grad[4i..4i+3] (may be NULL): the gradient of that interpolant;
 *   - control[2i..2i+1] (may be NULL): u_opt with ties to the upper bound:
 *     HJ_DYN_CAR4D (a, w), HJ_DYN_CAR4D_STEER (a, delta: the sign of
 *     dV/dth * v), HJ_DYN_CONST (0, 0).
 * states: m x 4 doubles (x, y, v, theta), row-major.  FP64 arithmetic; the
 * grid values are read in the grid's precision.  hj_query takes HOST arrays
 * (staged through the grid's free ping-pong buffer, nothing allocated);
 * hj_query_device takes DEVICE arrays on the grid's device.  HJ_ERR_STATE
 * without V0 (or without dynamics when control is requested). */
HJ_API hj_status hj_query(const hj_grid *g, const double *states, int64_t m, double *value, double *grad,
                          double *control);
HJ_API hj_status hj_query_device(const hj_grid *g, const double *states, int64_t m, double *value, double *grad,
                                 double *control);

/* Choose the step kernel.  HJ_KERNEL_TILED on a grid that it does not
 * support returns HJ_ERR_UNSUPPORTED and leaves the choice unchanged. */
HJ_API hj_status hj_set_kernel(hj_grid *g, hj_kernel kernel);

/* Tile shape of the tiled kernel: shape = {rows along y, rows along v, x
 * planes per work item, shared-memory stages}; a 0 entry is chosen
 * automatically.  HJ_ERR_UNSUPPORTED if the grid has no tiled kernel or the
 * shape does not fit (the previous shape then stays). */
HJ_API hj_status hj_set_tile_shape(hj_grid *g, const int32_t shape[4]);

/* Autotune the tiled kernel: time steps_per_trial (>= 1) step launches for
 * each candidate tile shape, re-time the three fastest with three times the
 * steps (their ms_retimed; this second pass needs results), and keep the
 * fastest of those.  Must be called right
 * after hj_set_initial_value[_device] (no step taken yet): trial steps read
 * V0 and write only the ping-pong buffers, and the time-loop state is put
 * back afterwards, so the next solve is unchanged.  results (may be NULL)
 * receives up to max_results candidates in the order tried, *nresults (may
 * be NULL) their count.  HJ_ERR_UNSUPPORTED without a tiled kernel,
 * HJ_ERR_STATE after a step. */
HJ_API hj_status hj_autotune(hj_grid *g, int32_t steps_per_trial, hj_tile_result *results, int32_t max_results,
                             int32_t *nresults);

/* One time step on caller-owned DEVICE arrays, allocating nothing.  The paper
 * has no counterpart: this entry point exists for callers that cannot
 * allocate device memory, such as code whose device memory all belongs to a
 * host framework's own pool, code on a memory budget fixed at start-up, or
 * code that must not call cudaMalloc (which can synchronise the device) at
 * the moment it steps.
 *
 * Computes v_out = min(v0, v_in + dt * rate(v_in)) for every cell: the same
 * step as hj_advance_brt, with the dt the caller gives (>= 0, finite).
 * Arrays are dense [N1][N2][N3][N4] of double (HJ_FP64) or float (HJ_FP32)
 * on the current device, owned by the caller; `bytes` is the size of each of
 * the three arrays and must equal N1*N2*N3*N4 * sizeof(element), and v_out
 * must overlap neither v_in nor v0 (HJ_ERR_INVALID_ARG otherwise: the library
 * cannot see the arrays' real sizes, so a short array would be overrun).
 * Grid, periodic mask and dynamics are as for hj_create_grid and
 * hj_set_dynamics (HJ_DYN_CAR4D and HJ_DYN_CONST; other kinds give
 * HJ_ERR_INVALID_ARG).
 * alpha_max_out (host, may be NULL) receives alpha_d^max over the grid, from
 * which a caller forms the next CFL step (dt = CFL / sum_d alpha_d^max/dx_d).
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine.  Its working
 * data (the per-(v, theta) coefficient table and the alpha^max accumulators)
 * live in a fixed device array of 640 KiB that every GPU which loads the
 * library holds until the process exits; N3 * N4 may therefore be at most
 * 16384 (HJ_ERR_INVALID_ARG beyond).  The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  All calls share the array and it keeps the
 * last call's contents (each call clears what must start at zero), so calls
 * whose work overlaps on the GPU race with one another: serialise them on
 * one stream.  Runs on cuda_stream (NULL: the legacy default stream); every
 * call reads alpha^max back and synchronises cuda_stream before it returns,
 * so it blocks until the step is complete.  A CUDA error left pending by the
 * caller's earlier work is cleared at entry and not reported as this call's. */
HJ_API hj_status hj_step_noalloc(const int32_t n[4], const double lo[4], const double hi[4], uint32_t periodic_mask,
                                 hj_precision prec, hj_dynamics kind, const double *params, int32_t nparams,
                                 const void *v_in, const void *v0, void *v_out, size_t bytes, double dt,
                                 void *cuda_stream, double alpha_max_out[4]);

/* ---- Batches: many independent car grids stepped together ---------------
 *
 * A batch holds up to max_slots grids ("slots"), each with its own size,
 * bounds, control bounds, V0, horizon and time loop (Sec. II-B scheme as
 * above, FP32, theta periodic, the other axes not).  A batch step advances
 * every slot that has not reached its horizon by its own CFL step;
 * hj_batch_advance runs up to 1024 batch steps per launch of one persistent
 * kernel, in which each slot starts its next step as soon as its own step is
 * done.  Slots may be added and removed between calls (admission is
 * by device memory: a slot needs hj_batch_slot_bytes(n) of the batch's
 * budget). */
typedef struct hj_batch hj_batch;

typedef struct {
    int64_t steps;      /* batch steps taken by this call */
    int64_t launches;   /* kernel launches (each runs up to 1024 batch steps) */
    int32_t active;     /* slots with steps left after this call */
    int32_t finished;   /* slots at their horizon */
    double device_ms;   /* device time of the call (CUDA events) */
    int32_t nconsumer;  /* consumer threads per CTA of the batch kernel */
    int32_t ctas;       /* CTAs per batch step */
    int32_t items;      /* work items per batch step in the last item layout (the running slots) */
} hj_batch_stats;

typedef struct {
    int32_t n[4];
    int64_t steps;      /* steps since the slot's initial value */
    double t, T;        /* simulated time reached, horizon */
    double dt_last;     /* size of the slot's last step */
    int32_t done;       /* reached T (or no horizon set yet) */
    int32_t has_value;
    int32_t tile[3];    /* rows along y and v, x planes per work item */
    size_t device_bytes;
} hj_batch_slot_info;

/* Create an empty batch on the current device.  memory_budget: bytes the
 * slots may hold (0: 90% of the free device memory).  cuda_stream: as for
 * hj_create_grid. */
HJ_API hj_status hj_batch_create(int32_t max_slots, size_t memory_budget, void *cuda_stream, hj_batch **out);

/* Device bytes a slot of n[0]*n[1]*n[2]*n[3] cells needs (V0, two buffers,
 * tables). */
HJ_API size_t hj_batch_slot_bytes(const int32_t n[4]);

/* Add a car grid (x, y, v, theta; bounds as hj_create_grid, theta periodic)
 * with params = {a_max, w_max}.  *slot receives its index.  HJ_ERR_OOM if no
 * slot is free or the budget would be exceeded. */
HJ_API hj_status hj_batch_add(hj_batch *b, const int32_t n[4], const double lo[4], const double hi[4],
                              const double params[2], int32_t *slot);

/* Free a slot (its device memory returns to the budget). */
HJ_API hj_status hj_batch_remove(hj_batch *b, int32_t slot);

/* V0 of a slot from a host FP64 array or a device FP32/FP64 array (layout as
 * hj_set_initial_value); resets the slot's time to 0.  The slot takes no step
 * until hj_batch_set_horizon. */
HJ_API hj_status hj_batch_set_initial_value(hj_batch *b, int32_t slot, const double *v0, size_t count);
HJ_API hj_status hj_batch_set_initial_value_device(hj_batch *b, int32_t slot, const void *v0, hj_precision dtype,
                                                   size_t count);

/* The same for several slots in one call: slots[k] takes the device array
 * v0[k] of counts[k] values (dtype HJ_FP32 or HJ_FP64; layout as
 * hj_set_initial_value).  Every argument is checked before anything is
 * queued; the conversions are queued back to back and one stream
 * synchronisation covers every slot's NaN / Inf check, so a batch's V0 set
 * costs one wait instead of one per slot.  A slot whose V0 holds NaN or Inf
 * is left without a value and the call returns HJ_ERR_INVALID_ARG naming the
 * first such slot; the others are set. */
HJ_API hj_status hj_batch_set_initial_values_device(hj_batch *b, int32_t nslots, const int32_t *slots,
                                                    const void *const *v0, hj_precision dtype, const size_t *counts);

/* As hj_set_initial_value_xy, for a slot. */
HJ_API hj_status hj_batch_set_initial_value_xy(hj_batch *b, int32_t slot, const double *v0_xy, size_t count);

/* Horizon T and Courant number of a slot (computes its first dt on the
 * device; queued on the batch's stream, ordered before the next batch step,
 * without waiting for it). */
HJ_API hj_status hj_batch_set_horizon(hj_batch *b, int32_t slot, double T, double cfl);

/* The same for several slots in one call (slots[k] takes T[k], cfl[k]);
 * every argument is checked before anything is queued. */
HJ_API hj_status hj_batch_set_horizons(hj_batch *b, int32_t nslots, const int32_t *slots, const double *T,
                                       const double *cfl);

/* Take up to max_steps batch steps (each unfinished slot advances one step
 * per batch step) and return when every slot has reached its horizon or the
 * step budget is used.  stats may be NULL. */
HJ_API hj_status hj_batch_advance(hj_batch *b, int64_t max_steps, hj_batch_stats *stats);

/* State of a slot. */
HJ_API hj_status hj_batch_get_slot_info(const hj_batch *b, int32_t slot, hj_batch_slot_info *info);

/* Current V of a slot into a host FP64 buffer or a device FP32/FP64 buffer
 * (layout as hj_read_value). */
HJ_API hj_status hj_batch_read_value(hj_batch *b, int32_t slot, double *out, size_t count);
HJ_API hj_status hj_batch_read_value_device(hj_batch *b, int32_t slot, void *out_device, hj_precision dtype,
                                            size_t count);

/* Kernel shape: consumer threads per CTA (0: automatic, else a multiple of 32
 * in [128, 736]; shapes of at most 288 run two CTAs per SM, each with half
 * of the SM's shared memory) and x chunks per slot column (1: whole columns; 0:
 * automatic, whole columns unless the running slots have fewer (y, v)
 * columns than the kernel has resident CTAs, then as many chunks as fill
 * them, each at least 4 x planes long). */
HJ_API hj_status hj_batch_set_shape(hj_batch *b, int32_t nconsumer, int32_t chunks);

/* Time steps_per_trial batch steps for each candidate kernel shape and keep
 * the fastest.  Every slot must hold an initial value and have taken no step
 * (trial steps read V0 and write only the ping-pong buffers; slot states are
 * put back afterwards).  Outputs may be NULL. */
HJ_API hj_status hj_batch_autotune(hj_batch *b, int32_t steps_per_trial, int32_t *best_nconsumer, int32_t *best_chunks,
                                   double *best_ms_per_step);

/* Free the batch and all its slots (NULL is a no-op). */
HJ_API void hj_batch_destroy(hj_batch *b);

/* ---- Re-solve server: continuous batching of BRT requests ----------------
 *
 * The paper's real-time use (Sec. I; Sec. IV-C: re-computing the BRT at
 * 5 Hz as the environment changes): requests arrive at any time, are
 * admitted into a batch when a slot and enough device memory are free, and
 * are stepped together with the requests already in flight; results stay on
 * the device until fetched.  Times are seconds on the server's clock. */
typedef struct hj_server hj_server;

typedef struct {
    int32_t state;      /* 0 queued, 1 running, 2 done, 3 failed (fetch returns the reason) */
    int32_t slot;       /* batch slot while running or done */
    int64_t steps;      /* time steps taken (when done) */
    double t_submit, t_admit, t_done;
} hj_request_info;

/* max_slots and memory_budget as hj_batch_create; steps_per_tick: batch
 * steps per hj_server_tick (>= 1): smaller admits new requests sooner. */
HJ_API hj_status hj_server_create(int32_t max_slots, size_t memory_budget, int32_t steps_per_tick, void *cuda_stream,
                                  hj_server **out);

/* Queue a request: a car grid (as hj_batch_add), V0 as a host FP64 array
 * (copied), horizon T and Courant number.  *request_id identifies it. */
HJ_API hj_status hj_server_submit(hj_server *s, const int32_t n[4], const double lo[4], const double hi[4],
                                  const double params[2], const double *v0, double T, double cfl,
                                  int64_t *request_id);

/* As hj_server_submit with V0 given by its N1*N2 (x, y) field (see
 * hj_set_initial_value_xy). */
HJ_API hj_status hj_server_submit_xy(hj_server *s, const int32_t n[4], const double lo[4], const double hi[4],
                                     const double params[2], const double *v0_xy, double T, double cfl,
                                     int64_t *request_id);

/* Admit queued requests (arrival order) while slots and memory last, take
 * steps_per_tick batch steps, and mark requests at their horizon done.
 * Outputs (may be NULL): requests completed by this tick, still running,
 * still queued. */
HJ_API hj_status hj_server_tick(hj_server *s, int32_t *completed, int32_t *running, int32_t *queued);

/* State and timestamps of a request. */
HJ_API hj_status hj_server_request_info(const hj_server *s, int64_t request_id, hj_request_info *info);

/* Copy a done request's V into a host FP64 buffer (or a device FP32/FP64
 * buffer) and release its slot; the request is forgotten afterwards. */
HJ_API hj_status hj_server_fetch(hj_server *s, int64_t request_id, double *out, size_t count);
HJ_API hj_status hj_server_fetch_device(hj_server *s, int64_t request_id, void *out_device, hj_precision dtype,
                                        size_t count);

/* Seconds since the server was created (the clock of the timestamps). */
HJ_API double hj_server_clock(const hj_server *s);

/* Ticks and batch steps taken so far (outputs may be NULL). */
HJ_API hj_status hj_server_stats(const hj_server *s, int64_t *ticks, int64_t *batch_steps);

/* Free the server, its batch and every request (NULL is a no-op). */
HJ_API void hj_server_destroy(hj_server *s);

/* Describe the grid (sizes, spacings, time, memory). */
HJ_API hj_status hj_get_info(const hj_grid *g, hj_grid_info *info);

/* Self-test of failure detection (the paper has no counterpart): runs a
 * kernel whose warps wait, with the same bounded mbarrier wait as the step
 * kernels, on a barrier phase that nothing completes.  The wait gives up
 * after limit_ns (1 ms .. 2 s) and the kernel records HJ_ERR_TIMEOUT, the
 * status a step kernel reports when a wait runs out.  No fault, trap or hang
 * is involved and the context stays usable.  Returns HJ_OK with *status =
 * HJ_ERR_TIMEOUT (or HJ_OK if the wait had completed) and *waited_ns (may be
 * NULL) = the time the kernel waited.  Allocates a few bytes; synchronises
 * the current device. */
HJ_API hj_status hj_wait_selftest(int64_t limit_ns, int32_t *status, int64_t *waited_ns);

/* The same self-test for the grid barrier of HJ_KERNEL_RESIDENT: a
 * cooperative launch of two CTAs waits, with the resident kernel's bounded
 * barrier, for a third CTA that does not exist.  Each wait gives up after
 * limit_ns (1 ms .. 2 s) and the kernel records HJ_ERR_TIMEOUT, the status
 * the resident kernel reports when a barrier runs out.  Same outputs and
 * side effects as hj_wait_selftest. */
HJ_API hj_status hj_barrier_selftest(int64_t limit_ns, int32_t *status, int64_t *waited_ns);

/* FP64 fused multiply-add throughput probe.  The paper has no counterpart:
 * it measures the FP64 rate that the FP64 step kernel and the query kernel
 * are held against (their roofline).  Launches one kernel on cuda_stream
 * (NULL: the legacy default stream) of blocks_per_sm (1..64) x SMs CTAs of
 * 256 threads, each thread running 8 independent chains of `iters`
 * (1..2^40) dependent FMAs.  *fma_out (may be NULL) = the FMAs issued (2
 * flops each).  Asynchronous: time it with events on cuda_stream.  Allocates
 * nothing; HJ_ERR_INVALID_ARG for out-of-range arguments, HJ_ERR_CUDA if the
 * launch fails. */
HJ_API hj_status hj_fp64_fma_probe(int64_t iters, int32_t blocks_per_sm, void *cuda_stream, int64_t *fma_out);

/* Free all device and host resources of the grid (NULL is a no-op). */
HJ_API void hj_destroy_grid(hj_grid *g);

/* Static string naming a status code. */
HJ_API const char *hj_status_string(hj_status s);

/* Message of the last error raised on the calling host thread ("" if none). */
HJ_API const char *hj_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
HJ_API int32_t hj_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HJ_H */
