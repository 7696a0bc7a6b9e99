// C-ABI implementation of libhj (declarations and documentation: hj.h).
//
// Host side of the HJ reachability solver for arxiv 2012.04011: grid and
// buffer management, the (v, theta) state tables (Sec. III-A), V0 ingest,
// the time loop driving the step kernels (Algorithms 1-2, Sec. II-B), and
// readback.  Simulated time and dt live on the device in FP64 and are
// advanced by the step kernels themselves (fused alpha^max reduction and
// finaliser, hj_device.cuh); the host only launches steps and reads the
// state back to know when the horizon is reached.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <type_traits>

#include "hj_device.cuh"

#define HJ_VERSION 10000

namespace {

thread_local char g_err[512] = "";

hj_status set_err(hj_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

#define HJ_CUDA(call)                                                                                 \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) {                                                                      \
            cudaGetLastError(); /* a failed call (not a sticky fault) must not fail later checks */   \
            return set_err(e_ == cudaErrorMemoryAllocation ? HJ_ERR_OOM : HJ_ERR_CUDA, "%s: %s (%s:%d)", \
                           #call, cudaGetErrorString(e_), __FILE__, __LINE__);                        \
        }                                                                                             \
    } while (0)

// ---------------------------------------------------------------- kernels

// Element conversions of the ingest and readback kernels: int32_t stands for
// Q5.27 codes (nearest-even and saturating from FP64, exact back to FP64).
template <typename T>
__device__ __forceinline__ double elem_to_f64(T v)
{
    if constexpr (std::is_same<T, int32_t>::value) return hj_q527_to_f64(v);
    else return (double)v;
}

template <typename T>
__device__ __forceinline__ T elem_from_f64(double x)
{
    if constexpr (std::is_same<T, int32_t>::value) return hj_q527_from_f64(x);
    else return (T)x;
}

// Dense row-major [N1][N2][N3][N4] (any of double/float) -> internal layout
// (rows padded to p4, pad lanes zero).  Flags non-finite input.
template <typename Tin, typename T>
__global__ void ingest_kernel(const Tin *__restrict__ src, T *__restrict__ dst, int n4, int p4, long long nrows,
                              int *nonfinite)
{
    long long total = nrows * p4;
    int bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        long long row = i / p4;
        int l = (int)(i - row * p4);
        T v = T(0);
        if (l < n4) {
            double x = elem_to_f64<Tin>(src[row * n4 + l]);
            if (!isfinite(x)) bad = 1;
            v = elem_from_f64<T>(x);
        }
        dst[i] = v;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(nonfinite, 1);
}

// V0 that depends only on (x, y): an N1*N2 field replicated over v and theta
// (Eq. init_V depends on the position only), written in the internal layout.
template <typename Tin, typename T>
__global__ void ingest_xy_kernel(const Tin *__restrict__ src, T *__restrict__ dst, int n3, int n4, int p4,
                                 long long nxy, int *nonfinite)
{
    const long long per = (long long)n3 * p4, total = nxy * per;
    int bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long xy = i / per;
        const int l = (int)(i - xy * per) % p4;
        T v = T(0);
        if (l < n4) {
            const double x = elem_to_f64<Tin>(src[xy]);
            if (!isfinite(x)) bad = 1;
            v = elem_from_f64<T>(x);
        }
        dst[i] = v;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(nonfinite, 1);
}

// Internal layout -> dense (rows [row0, row0 + nrows)), converting type.
template <typename T, typename Tout>
__global__ void readback_kernel(const T *__restrict__ src, Tout *__restrict__ dst, int n4, int p4, long long row0,
                                long long nrows)
{
    long long total = nrows * n4;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        long long row = i / n4;
        int l = (int)(i - row * n4);
        dst[i] = elem_from_f64<Tout>(elem_to_f64<T>(src[(row0 + row) * p4 + l]));
    }
}

// Start of a solve call: horizon, Courant number and the dt of the first
// step.  Right after V0 is set (n == 0), alpha^max is reduced over the
// (v, theta) table, which holds |xdot_1|, |xdot_2| of every cell (the car's
// velocity depends only on v and theta).
template <typename T>
__global__ void prologue_kernel(HjDevState *st, const HjGeom g, const HjCoef<T> *__restrict__ coef, int ncoef,
                                double T_end, double cfl, HjScaledCoef *scaled = nullptr, int32_t *qw = nullptr,
                                const double *k4 = nullptr, double threshold = 0.0)
{
    __shared__ unsigned long long scratch[64];
    hj_prologue_block(st, g, coef, ncoef, T_end, cfl, threshold, scratch);
    if (scaled || qw) {  // FP64 / Q5.27 grids: the dt-scaled tables must match the first dt
        __syncthreads();
        const volatile HjDevState *vs = st;
        const double dt = vs->dt;
        if (!vs->done && dt != vs->dt_scaled) {
            if (scaled) hj_rescale_table(scaled, (const HjCoef<double> *)coef, k4, g.n3, g.n4, dt);
            else hj_rescale_qweights(qw, (const HjCoef<double> *)coef, g.n3, g.n4, g.p4, g.k3, k4, dt);
            __syncthreads();
            if (threadIdx.x == 0) st->dt_scaled = dt;
        }
    }
}

int grid_blocks(long long work, int threads)
{
    long long b = (work + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    return b < 1 ? 1 : (int)b;
}

bool finite_all(const double *p, int n)
{
    for (int i = 0; i < n; ++i)
        if (!isfinite(p[i])) return false;
    return true;
}

hj_status check_grid(const hj_grid *g)
{
    if (!g) return set_err(HJ_ERR_INVALID_ARG, "grid is NULL");
    return HJ_OK;
}

hj_status activate(const hj_grid *g)
{
    int cur = -1;
    HJ_CUDA(cudaGetDevice(&cur));
    if (cur != g->device) HJ_CUDA(cudaSetDevice(g->device));
    return HJ_OK;
}

hj_status pull_state(hj_grid *g)
{
    HJ_CUDA(cudaMemcpyAsync(g->hstate, g->dstate, sizeof(HjDevState), cudaMemcpyDeviceToHost, g->stream));
    HJ_CUDA(cudaStreamSynchronize(g->stream));
    return HJ_OK;
}

hj_status upload_tables(hj_grid *g)
{
    const int N3 = g->n[2], N4 = g->n[3], P4 = g->p4;
    const bool car = g->dyn == HJ_DYN_CAR4D || g->dyn == HJ_DYN_CAR4D_STEER;
    // per-(v, theta) coefficients in FP64: xdot_1 = v cos(theta), xdot_2 = v sin(theta)
    size_t nco = (size_t)N3 * N4;
    double *f1 = (double *)malloc(sizeof(double) * nco), *f2 = (double *)malloc(sizeof(double) * nco);
    float *tab = (float *)calloc((size_t)N3 + 3 * (size_t)P4, sizeof(float));
    if (!f1 || !f2 || !tab) {
        free(f1);
        free(f2);
        free(tab);
        return set_err(HJ_ERR_OOM, "host allocation failed");
    }
    // FP64 tables keep libm's cos/sin; FP32 tables flush rounding artefacts
    const bool f32 = g->prec == HJ_FP32;
    for (int k = 0; k < N3; ++k) {
        double v = g->lo[2] + (double)k * g->h[2];
        tab[k] = (float)v;
        for (int l = 0; l < N4; ++l) {
            double th = g->lo[3] + (double)l * g->h[3];
            const double c = f32 ? hj_flush_trig(cos(th)) : cos(th), sn = f32 ? hj_flush_trig(sin(th)) : sin(th);
            f1[(size_t)k * N4 + l] = car ? v * c : g->params[0];
            f2[(size_t)k * N4 + l] = car ? v * sn : g->params[1];
        }
    }
    for (int l = 0; l < N4; ++l) {
        double th = g->lo[3] + (double)l * g->h[3];
        tab[N3 + l] = (float)(hj_flush_trig(cos(th)) / g->h[0]);
        tab[N3 + P4 + l] = (float)(hj_flush_trig(sin(th)) / g->h[1]);
    }
    // theta coefficient per speed, |xdot_4| / dx_4: the steering car's heading
    // rate bound is |v| tan(delta_max) / L; the other dynamics have one value
    double *k4v = (double *)malloc(sizeof(double) * (size_t)N3);
    float *k4f = (float *)malloc(2 * sizeof(float) * (size_t)N3);
    const double k3 = g->geom.k3;
    hj_status st = HJ_OK;
    if (!k4v || !k4f) st = set_err(HJ_ERR_OOM, "host allocation failed");
    for (int k = 0; st == HJ_OK && k < N3; ++k) {
        if (g->dyn == HJ_DYN_CAR4D_STEER) {
            const double v = g->lo[2] + (double)k * g->h[2];
            k4v[k] = (fabs(v) * tan(g->params[1])) / g->params[2] / g->h[3];
        } else {
            k4v[k] = g->geom.k4;
        }
        k4f[2 * k] = (float)k4v[k];
        k4f[2 * k + 1] = (float)(-(k3 + k4v[k]));
    }
    if (st == HJ_OK) {
        cudaError_t e = cudaMemcpy(g->k4tab, g->prec == HJ_FP32 ? (const void *)k4f : (const void *)k4v,
                                   g->prec == HJ_FP32 ? 2 * sizeof(float) * N3 : sizeof(double) * N3,
                                   cudaMemcpyHostToDevice);
        if (e != cudaSuccess) st = set_err(HJ_ERR_CUDA, "table upload: %s", cudaGetErrorString(e));
    }
    if (g->prec != HJ_FP32) {
        HjCoef<double> *c = (HjCoef<double> *)malloc(sizeof(HjCoef<double>) * nco);
        if (!c) st = set_err(HJ_ERR_OOM, "host allocation failed");
        for (size_t i = 0; c && i < nco; ++i) {
            c[i].c1 = f1[i] / g->h[0];
            c[i].c2 = f2[i] / g->h[1];
            c[i].ks = fabs(c[i].c1) + fabs(c[i].c2) + k3 + k4v[i / N4];
            c[i].a1 = fabs(f1[i]);
            c[i].a2 = fabs(f2[i]);
        }
        if (c) {
            cudaError_t e = cudaMemcpy(g->coef, c, sizeof(HjCoef<double>) * nco, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) st = set_err(HJ_ERR_CUDA, "table upload: %s", cudaGetErrorString(e));
        }
        free(c);
    } else {
        HjCoef<float> *c = (HjCoef<float> *)malloc(sizeof(HjCoef<float>) * nco);
        if (!c) st = set_err(HJ_ERR_OOM, "host allocation failed");
        for (size_t i = 0; c && i < nco; ++i) {
            double c1 = f1[i] / g->h[0], c2 = f2[i] / g->h[1];
            c[i].c1 = (float)c1;
            c[i].c2 = (float)c2;
            c[i].ks = (float)(fabs(c1) + fabs(c2) + k3 + k4v[i / N4]);
            c[i].a1 = fabs(f1[i]);
            c[i].a2 = fabs(f2[i]);
        }
        if (c) {
            cudaError_t e = cudaMemcpy(g->coef, c, sizeof(HjCoef<float>) * nco, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) st = set_err(HJ_ERR_CUDA, "table upload: %s", cudaGetErrorString(e));
        }
        free(c);
    }
    if (st == HJ_OK) {
        cudaError_t e = cudaMemcpy(g->tab_tiled, tab, sizeof(float) * ((size_t)N3 + 3 * (size_t)P4),
                                   cudaMemcpyHostToDevice);
        if (e != cudaSuccess) st = set_err(HJ_ERR_CUDA, "table upload: %s", cudaGetErrorString(e));
    }
    // the largest |xdot_1|, |xdot_2| over each theta quad's real headings, per speed
    if (st == HJ_OK) {
        const int Q4 = P4 / 4;
        double2 *aq = (double2 *)malloc(sizeof(double2) * (size_t)N3 * Q4);
        if (!aq) st = set_err(HJ_ERR_OOM, "host allocation failed");
        for (int k = 0; aq && k < N3; ++k)
            for (int q = 0; q < Q4; ++q) {
                double m1 = 0.0, m2 = 0.0;
                for (int l = 4 * q; l < 4 * q + 4 && l < N4; ++l) {
                    const double a1 = fabs(f1[(size_t)k * N4 + l]), a2 = fabs(f2[(size_t)k * N4 + l]);
                    if (a1 > m1) m1 = a1;
                    if (a2 > m2) m2 = a2;
                }
                aq[(size_t)k * Q4 + q] = make_double2(m1, m2);
            }
        if (aq) {
            cudaError_t e = cudaMemcpy(g->amax_q, aq, sizeof(double2) * (size_t)N3 * Q4, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) st = set_err(HJ_ERR_CUDA, "table upload: %s", cudaGetErrorString(e));
        }
        free(aq);
    }
    free(f1);
    free(f2);
    free(tab);
    free(k4v);
    free(k4f);
    return st;
}

hj_status reset_state(hj_grid *g)
{
    memset(g->hstate, 0, sizeof(HjDevState));
    g->hstate->status = HJ_OK;
    HJ_CUDA(cudaMemcpyAsync(g->dstate, g->hstate, sizeof(HjDevState), cudaMemcpyHostToDevice, g->stream));
    return HJ_OK;
}

// Whether HJ_KERNEL_AUTO takes the resident kernel: FP32 grids of up to 4 M
// cells and Q5.27 grids of up to 8 M cells (measured crossovers against the
// tiled kernel), where a step takes a few microseconds and the per-step
// launch and last-CTA finaliser of the other kernels cost about as much.
// Larger grids stream faster through the tiled kernel; FP64 steps are bound
// by the FP64 unit, where the resident form gains nothing.
bool resident_auto(const hj_grid *g)
{
    const long long cap = g->prec == HJ_FP32 ? (4LL << 20) : (g->prec == HJ_Q527 ? (8LL << 20) : 0);
    return g->ncell <= cap && hj_resident_supported(g);
}

hj_kernel effective_kernel(const hj_grid *g)
{
    if (g->kernel_req == HJ_KERNEL_GENERIC) return HJ_KERNEL_GENERIC;
    if (g->kernel_req == HJ_KERNEL_RESIDENT) return HJ_KERNEL_RESIDENT;
    if (g->kernel_req == HJ_KERNEL_AUTO && resident_auto(g)) return HJ_KERNEL_RESIDENT;
    return g->tiled_ok ? HJ_KERNEL_TILED : HJ_KERNEL_GENERIC;
}

hj_status launch_step(hj_grid *g, hj_kernel k)
{
    cudaError_t e = (k == HJ_KERNEL_TILED)     ? hj_launch_step_tiled(g)
                    : (k == HJ_KERNEL_RESIDENT) ? hj_launch_step_resident(g, 1)
                                                : hj_launch_step_generic(g);
    if (e != cudaSuccess) {
        cudaGetLastError();  // a failed call (not a sticky fault) must not fail later checks
        return set_err(e == cudaErrorMemoryAllocation ? HJ_ERR_OOM : HJ_ERR_CUDA, "step launch: %s",
                       cudaGetErrorString(e));
    }
    return HJ_OK;
}

// Grids below this many cells take a step in a few microseconds, less than
// launching it costs, so their time loop replays captured graphs.
constexpr long long GRAPH_MAX_CELLS = 1LL << 24;

// k step launches as one graph launch (captured on first use, kept in a
// 4-entry cache); false if a graph cannot be used here (the stream is being
// captured by the caller, or capture failed), and the caller launches the
// steps one by one.
bool launch_steps_graph(hj_grid *g, hj_kernel kern, long long k)
{
    if (g->ncell >= GRAPH_MAX_CELLS || k < 4 || k > 4096) return false;
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(g->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
    int hit = -1, victim = 0;
    for (int i = 0; i < 4; ++i) {
        const hj_grid::StepGraph &e = g->graphs[i];
        if (e.exec && e.k == k && e.kernel == (int)kern && e.track == (int)g->track && e.version == g->launch_version)
            hit = i;
        if (!g->graphs[i].exec) victim = i;
    }
    if (hit < 0) {
        if (g->graphs[victim].exec) victim = (int)(g->graph_tick++ % 4);
        hj_grid::StepGraph &e = g->graphs[victim];
        if (e.exec) {
            cudaGraphExecDestroy(e.exec);
            e.exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        bool ok = true;
        for (long long i = 0; i < k && ok; ++i)
            ok = ((kern == HJ_KERNEL_TILED) ? hj_launch_step_tiled(g) : hj_launch_step_generic(g)) == cudaSuccess;
        const cudaError_t ce = cudaStreamEndCapture(g->stream, &graph);
        if (!ok || ce != cudaSuccess || !graph) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return false;
        }
        const cudaError_t ie = cudaGraphInstantiate(&e.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            e.exec = nullptr;
            cudaGetLastError();
            return false;
        }
        e.k = k;
        e.kernel = (int)kern;
        e.track = (int)g->track;
        e.version = g->launch_version;
        hit = victim;
    }
    return cudaGraphLaunch(g->graphs[hit].exec, g->stream) == cudaSuccess;
}

// Calls f with a value of the grid element type: double, float or int32_t
// (Q5.27 codes).
template <typename F>
void with_elem(hj_precision p, F &&f)
{
    if (p == HJ_FP64) f(double(0));
    else if (p == HJ_FP32) f(float(0));
    else f(int32_t(0));
}

bool valid_prec(hj_precision p) { return p == HJ_FP64 || p == HJ_FP32 || p == HJ_Q527; }

// Start of a solve call (horizon, Courant number, first dt, and the FP64 /
// fixed-point tables scaled for it).
void launch_prologue(hj_grid *g, double T, double cfl, double threshold = 0.0)
{
    const int ncoef = g->n[2] * g->n[3];
    if (g->prec == HJ_FP32)
        prologue_kernel<float><<<1, 256, 0, g->stream>>>(g->dstate, g->geom, (const HjCoef<float> *)g->coef, ncoef, T,
                                                         cfl, nullptr, nullptr, nullptr, threshold);
    else
        prologue_kernel<double><<<1, 256, 0, g->stream>>>(g->dstate, g->geom, (const HjCoef<double> *)g->coef, ncoef,
                                                          T, cfl, g->scaled, g->qw, (const double *)g->k4tab,
                                                          threshold);
}

void free_grid(hj_grid *g)
{
    if (!g) return;
    if (g->v0) cudaFree(g->v0);
    if (g->buf) cudaFree(g->buf);
    if (g->coef) cudaFree(g->coef);
    if (g->tab_tiled) cudaFree(g->tab_tiled);
    if (g->amax_q) cudaFree(g->amax_q);
    if (g->scaled) cudaFree(g->scaled);
    if (g->qw) cudaFree(g->qw);
    if (g->v0xy) cudaFree(g->v0xy);
    if (g->k4tab) cudaFree(g->k4tab);
    if (g->rsync) cudaFree(g->rsync);
    if (g->dstate) cudaFree(g->dstate);
    if (g->hstate) cudaFreeHost(g->hstate);
    for (int i = 0; i < 4; ++i)
        if (g->ev[i]) cudaEventDestroy(g->ev[i]);
    if (g->ev_in) cudaEventDestroy(g->ev_in);
    for (int i = 0; i < 4; ++i)
        if (g->graphs[i].exec) cudaGraphExecDestroy(g->graphs[i].exec);
    if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
    delete g;
}

}  // namespace

void hj_internal_set_error(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

// Launchers of the ingest, readback and prologue kernels for other parts of
// the library (the batch API); all return the launch's CUDA error.
cudaError_t hj_launch_ingest_f32(const void *src, hj_precision src_type, float *dst, int n4, int p4, long long nrows,
                                 int *nonfinite, cudaStream_t stream)
{
    const int blocks = grid_blocks(nrows * p4, 256);
    if (src_type == HJ_FP64)
        ingest_kernel<double, float><<<blocks, 256, 0, stream>>>((const double *)src, dst, n4, p4, nrows, nonfinite);
    else
        ingest_kernel<float, float><<<blocks, 256, 0, stream>>>((const float *)src, dst, n4, p4, nrows, nonfinite);
    return cudaGetLastError();
}

cudaError_t hj_launch_ingest_xy_f32(const double *src_dev, float *dst, int n3, int n4, int p4, long long nxy,
                                    int *nonfinite, cudaStream_t stream)
{
    ingest_xy_kernel<double, float><<<grid_blocks(nxy * n3 * p4, 256), 256, 0, stream>>>(src_dev, dst, n3, n4, p4, nxy,
                                                                                 nonfinite);
    return cudaGetLastError();
}

cudaError_t hj_launch_readback_f32(const float *src, void *dst, hj_precision dst_type, int n4, int p4, long long row0,
                                   long long nrows, cudaStream_t stream)
{
    const int blocks = grid_blocks(nrows * n4, 256);
    if (dst_type == HJ_FP64)
        readback_kernel<float, double><<<blocks, 256, 0, stream>>>(src, (double *)dst, n4, p4, row0, nrows);
    else
        readback_kernel<float, float><<<blocks, 256, 0, stream>>>(src, (float *)dst, n4, p4, row0, nrows);
    return cudaGetLastError();
}

cudaError_t hj_launch_prologue_f32(HjDevState *st, const HjGeom &g, const HjCoef<float> *coef, int ncoef, double T,
                                   double cfl, cudaStream_t stream)
{
    prologue_kernel<float><<<1, 256, 0, stream>>>(st, g, coef, ncoef, T, cfl);
    return cudaGetLastError();
}

// ==================================================================== C ABI

extern "C" {

int32_t hj_version(void) { return HJ_VERSION; }

const char *hj_last_error(void) { return g_err; }

const char *hj_status_string(hj_status s)
{
    switch (s) {
    case HJ_OK: return "HJ_OK";
    case HJ_ERR_INVALID_ARG: return "HJ_ERR_INVALID_ARG";
    case HJ_ERR_STATE: return "HJ_ERR_STATE";
    case HJ_ERR_OOM: return "HJ_ERR_OOM";
    case HJ_ERR_CUDA: return "HJ_ERR_CUDA";
    case HJ_ERR_UNSTABLE: return "HJ_ERR_UNSTABLE";
    case HJ_ERR_TIMEOUT: return "HJ_ERR_TIMEOUT";
    case HJ_ERR_UNSUPPORTED: return "HJ_ERR_UNSUPPORTED";
    }
    return "HJ_ERR_UNKNOWN";
}

hj_status hj_create_grid(const int32_t n[4], const double lo[4], const double hi[4], uint32_t periodic_mask,
                         hj_precision prec, void *cuda_stream, hj_grid **out)
{
    g_err[0] = 0;
    if (!n || !lo || !hi || !out) return set_err(HJ_ERR_INVALID_ARG, "NULL argument");
    if (!valid_prec(prec)) return set_err(HJ_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    if (periodic_mask & ~0xFu) return set_err(HJ_ERR_INVALID_ARG, "periodic_mask has bits above 3");
    long long ncell = 1;
    for (int d = 0; d < 4; ++d) {
        if (n[d] < 3) return set_err(HJ_ERR_INVALID_ARG, "N%d = %d < 3", d + 1, n[d]);
        if (!isfinite(lo[d]) || !isfinite(hi[d]) || !(hi[d] > lo[d]))
            return set_err(HJ_ERR_INVALID_ARG, "axis %d bounds must be finite with hi > lo", d + 1);
        ncell *= n[d];
    }
    if (n[3] > 4096) return set_err(HJ_ERR_INVALID_ARG, "N4 = %d > 4096", n[3]);
    if (ncell > (1LL << 33)) return set_err(HJ_ERR_INVALID_ARG, "grid of %lld cells is too large", ncell);

    hj_grid *g = new (std::nothrow) hj_grid();
    if (!g) return set_err(HJ_ERR_OOM, "host allocation failed");
    memset(g, 0, sizeof(*g));
    for (int d = 0; d < 4; ++d) {
        g->n[d] = n[d];
        g->lo[d] = lo[d];
        g->hi[d] = hi[d];
        bool per = (periodic_mask >> d) & 1u;
        g->h[d] = (hi[d] - lo[d]) / (double)(per ? n[d] : n[d] - 1);
    }
    g->p4 = (n[3] + 3) / 4 * 4;
    g->periodic = periodic_mask;
    g->prec = prec;
    g->esize = prec == HJ_FP64 ? 8 : 4;  // FP32 and Q5.27: 4 bytes
    g->ncell = ncell;
    g->nint = (long long)n[0] * n[1] * n[2] * g->p4;
    g->kernel_req = HJ_KERNEL_AUTO;

    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess && cuda_stream) {
        g->stream = (cudaStream_t)cuda_stream;
    } else if (e == cudaSuccess) {
        e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
        g->own_stream = e == cudaSuccess;
    }
    size_t arr = (size_t)g->nint * g->esize;
    size_t ncoef = (size_t)n[2] * n[3];
    if (e == cudaSuccess) e = cudaMalloc(&g->v0, arr);
    if (e == cudaSuccess) e = cudaMalloc(&g->buf, 2 * arr);
    // FP64 coefficients for FP64 and Q5.27 grids (alpha^max and dt are FP64)
    const size_t coef_bytes = ncoef * (prec == HJ_FP32 ? sizeof(HjCoef<float>) : sizeof(HjCoef<double>));
    const size_t qw_bytes = prec == HJ_Q527 ? sizeof(int32_t) * (2 * (size_t)n[2] * g->p4 + HJ_QW_TAIL + n[2]) : 0;
    const size_t k4_bytes = (size_t)n[2] * (prec == HJ_FP32 ? 2 * sizeof(float) : sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&g->coef, coef_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&g->tab_tiled, sizeof(float) * ((size_t)n[2] + 3 * (size_t)g->p4));
    if (e == cudaSuccess) e = cudaMalloc(&g->amax_q, sizeof(double2) * (size_t)n[2] * (g->p4 / 4));
    if (e == cudaSuccess && prec == HJ_FP64) e = cudaMalloc(&g->scaled, ncoef * sizeof(HjScaledCoef));
    if (e == cudaSuccess && prec == HJ_Q527) e = cudaMalloc(&g->qw, qw_bytes);
    const size_t xy_bytes = (size_t)n[0] * n[1] * g->esize;
    if (e == cudaSuccess) e = cudaMalloc(&g->v0xy, xy_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&g->k4tab, k4_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&g->dstate, sizeof(HjDevState));
    if (e == cudaSuccess) e = cudaHostAlloc(&g->hstate, sizeof(HjDevState), cudaHostAllocDefault);
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&g->ev[i]);
    if (e == cudaSuccess && g->own_stream) e = cudaEventCreateWithFlags(&g->ev_in, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();  // the failed allocation must not fail later launch checks
        hj_status s = set_err(e == cudaErrorMemoryAllocation ? HJ_ERR_OOM : HJ_ERR_CUDA, "hj_create_grid: %s",
                              cudaGetErrorString(e));
        free_grid(g);
        return s;
    }
    g->device_bytes = 3 * arr + coef_bytes + qw_bytes + (prec == HJ_FP64 ? ncoef * sizeof(HjScaledCoef) : 0) +
                      xy_bytes + k4_bytes + sizeof(HjDevState);
    hj_status s = reset_state(g);
    if (s == HJ_OK) {
        cudaError_t e2 = cudaStreamSynchronize(g->stream);
        if (e2 != cudaSuccess) s = set_err(HJ_ERR_CUDA, "hj_create_grid: %s", cudaGetErrorString(e2));
    }
    if (s != HJ_OK) {
        free_grid(g);
        return s;
    }
    *out = g;
    return HJ_OK;
}

void hj_destroy_grid(hj_grid *g)
{
    if (!g) return;
    if (activate(g) == HJ_OK && g->stream) cudaStreamSynchronize(g->stream);
    free_grid(g);
}

hj_status hj_set_dynamics(hj_grid *g, hj_dynamics kind, const double *params, int32_t nparams)
{
    g_err[0] = 0;
    hj_status s = check_grid(g);
    if (s != HJ_OK) return s;
    if (!params) return set_err(HJ_ERR_INVALID_ARG, "params is NULL");
    if (kind == HJ_DYN_CAR4D) {
        if (nparams != 2) return set_err(HJ_ERR_INVALID_ARG, "car dynamics take 2 parameters (a_max, w_max)");
        if (!finite_all(params, 2) || params[0] < 0 || params[1] < 0)
            return set_err(HJ_ERR_INVALID_ARG, "a_max and w_max must be finite and >= 0");
    } else if (kind == HJ_DYN_CONST) {
        if (nparams != 4) return set_err(HJ_ERR_INVALID_ARG, "constant dynamics take 4 parameters");
        if (!finite_all(params, 4)) return set_err(HJ_ERR_INVALID_ARG, "parameters must be finite");
    } else if (kind == HJ_DYN_CAR4D_STEER) {
        if (nparams != 3)
            return set_err(HJ_ERR_INVALID_ARG, "steering dynamics take 3 parameters (a_max, delta_max, L)");
        if (!finite_all(params, 3) || params[0] < 0 || params[1] < 0 || !(params[1] < 1.5707963267948966) ||
            !(params[2] > 0))
            return set_err(HJ_ERR_INVALID_ARG, "need a_max >= 0, 0 <= delta_max < pi/2 and L > 0");
    } else {
        return set_err(HJ_ERR_INVALID_ARG, "unknown dynamics %d", (int)kind);
    }
    if ((s = activate(g)) != HJ_OK) return s;
    HJ_CUDA(cudaStreamSynchronize(g->stream));
    g->dyn = kind;
    for (int i = 0; i < 4; ++i) g->params[i] = i < nparams ? params[i] : 0.0;

    HjGeom &G = g->geom;
    memset(&G, 0, sizeof(G));
    G.n1 = g->n[0];
    G.n2 = g->n[1];
    G.n3 = g->n[2];
    G.n4 = g->n[3];
    G.p4 = g->p4;
    G.periodic = (int32_t)g->periodic;
    for (int d = 0; d < 4; ++d) G.h[d] = g->h[d];
    if (kind == HJ_DYN_CAR4D) {
        G.mode3 = HJ_AXIS_CONTROL;
        G.mode4 = HJ_AXIS_CONTROL;
        G.alpha3 = params[0];
        G.alpha4 = params[1];
    } else if (kind == HJ_DYN_CAR4D_STEER) {
        // alpha_4^max = max_k |v_k| tan(delta_max) / L (the end points of the v axis)
        G.mode3 = HJ_AXIS_CONTROL;
        G.mode4 = HJ_AXIS_CONTROL;
        G.alpha3 = params[0];
        double vmax = 0.0;
        for (int k = 0; k < g->n[2]; ++k) vmax = fmax(vmax, fabs(g->lo[2] + (double)k * g->h[2]));
        G.alpha4 = (vmax * tan(params[1])) / params[2];
    } else {
        G.mode3 = params[2] >= 0 ? HJ_AXIS_PLUS : HJ_AXIS_MINUS;
        G.mode4 = params[3] >= 0 ? HJ_AXIS_PLUS : HJ_AXIS_MINUS;
        G.alpha3 = fabs(params[2]);
        G.alpha4 = fabs(params[3]);
    }
    G.k3 = G.alpha3 / g->h[2];
    G.k4 = G.alpha4 / g->h[3];
    if ((s = upload_tables(g)) != HJ_OK) return s;
    // a solve in progress continues under the new dynamics: the next
    // prologue re-reduces alpha^max from the new table (Alg. 2 takes it from
    // the current Hamiltonian) and rebuilds the FP64 dt-scaled table
    HJ_CUDA(cudaMemsetAsync(&g->dstate->dt_scaled, 0, sizeof(double), g->stream));
    HJ_CUDA(cudaMemsetAsync(&g->dstate->alpha_stale, 1, sizeof(int), g->stream));
    g->has_dyn = true;
    char why[160];
    g->tiled_ok = hj_tiled_setup(g, why, sizeof(why));
    if (g->kernel_req == HJ_KERNEL_TILED && !g->tiled_ok) g->kernel_req = HJ_KERNEL_AUTO;
    // a previously set V0 stays; the next solve continues with the new dynamics
    return HJ_OK;
}

// The tiled kernel's stage layout depends on whether V0 is broadcast from the
// (x, y) field; redo its setup when that changes.
static void set_v0_mode(hj_grid *g, bool bcast)
{
    if (g->v0_bcast == bcast) return;
    g->v0_bcast = bcast;
    if (g->has_dyn) {
        char why[160];
        g->tiled_ok = hj_tiled_setup(g, why, sizeof(why));
        if (g->kernel_req == HJ_KERNEL_TILED && !g->tiled_ok) g->kernel_req = HJ_KERNEL_AUTO;
    }
}

static hj_status finish_ingest(hj_grid *g);

// V0 from its (x, y) field on the device (src: nxy values of dtype): the 4D
// V0 (replicated over v and theta) and the field itself for the
// broadcast-V0 step kernel, with the same conversion.
static hj_status ingest_xy(hj_grid *g, const void *src, hj_precision dtype, long long nxy)
{
    int *flag = &g->dstate->nonfinite;
    const int blocks = grid_blocks(g->nint, 256);
    with_elem(dtype, [&](auto ein) {
        with_elem(g->prec, [&](auto e) {
            using Tin = decltype(ein);
            using T = decltype(e);
            ingest_xy_kernel<Tin, T><<<blocks, 256, 0, g->stream>>>((const Tin *)src, (T *)g->v0, g->n[2], g->n[3],
                                                                    g->p4, nxy, flag);
            ingest_kernel<Tin, T><<<grid_blocks(nxy, 256), 256, 0, g->stream>>>((const Tin *)src, (T *)g->v0xy,
                                                                                (int)nxy, (int)nxy, 1, flag);
        });
    });
    set_v0_mode(g, true);
    return finish_ingest(g);
}

static hj_status finish_ingest(hj_grid *g)
{
    HJ_CUDA(cudaGetLastError());
    HJ_CUDA(cudaStreamSynchronize(g->stream));
    HJ_CUDA(cudaMemcpy(g->hstate, g->dstate, sizeof(HjDevState), cudaMemcpyDeviceToHost));
    if (g->hstate->nonfinite) {
        g->has_value = false;
        reset_state(g);
        cudaStreamSynchronize(g->stream);
        return set_err(HJ_ERR_INVALID_ARG, "V0 contains NaN or Inf");
    }
    g->has_value = true;
    return HJ_OK;
}

// Device address of a host buffer the grid's device can reach directly
// (pinned host memory, mapped into the device's address space), else NULL.
// The ingest and readback kernels then read or write it over the host link
// in one pass instead of staging it through device memory with a copy.
static void *device_view(const hj_grid *g, const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    return a.device == g->device ? a.devicePointer : nullptr;
}

// A grid on its own (non-blocking) stream reads caller-owned device arrays
// only after the work already queued on the legacy default stream, where a
// caller that names no stream (PyTorch's default stream included) wrote them.
// A grid on a caller's stream is ordered by that stream.
static hj_status follow_default_stream(hj_grid *g)
{
    if (!g->own_stream) return HJ_OK;
    HJ_CUDA(cudaEventRecord(g->ev_in, cudaStreamLegacy));
    HJ_CUDA(cudaStreamWaitEvent(g->stream, g->ev_in, 0));
    return HJ_OK;
}

hj_status hj_set_initial_value(hj_grid *g, const double *v0, size_t count)
{
    g_err[0] = 0;
    hj_status s = check_grid(g);
    if (s != HJ_OK) return s;
    if (!v0) return set_err(HJ_ERR_INVALID_ARG, "v0 is NULL");
    if (count != (size_t)g->ncell)
        return set_err(HJ_ERR_INVALID_ARG, "count %zu != N1*N2*N3*N4 = %lld", count, g->ncell);
    if ((s = activate(g)) != HJ_OK) return s;
    if ((s = reset_state(g)) != HJ_OK) return s;
    // pinned host memory: the ingest kernel reads it directly; otherwise stage
    // the dense FP64 array in the ping-pong region (2 * nint * esize >= ncell * 8 bytes)
    const double *staging = (const double *)device_view(g, v0);
    if (!staging) {
        staging = (const double *)g->buf;
        HJ_CUDA(cudaMemcpyAsync(g->buf, v0, sizeof(double) * (size_t)g->ncell, cudaMemcpyHostToDevice, g->stream));
    }
    long long nrows = (long long)g->n[0] * g->n[1] * g->n[2];
    int *flag = &g->dstate->nonfinite;
    int blocks = grid_blocks(g->nint, 256);
    with_elem(g->prec, [&](auto e) {
        using T = decltype(e);
        ingest_kernel<double, T><<<blocks, 256, 0, g->stream>>>(staging, (T *)g->v0, g->n[3], g->p4, nrows, flag);
    });
    set_v0_mode(g, false);
    return finish_ingest(g);
}

hj_status hj_set_initial_value_xy(hj_grid *g, const double *v0_xy, size_t count)
{
    g_err[0] = 0;
    hj_status s = check_grid(g);
    if (s != HJ_OK) return s;
    if (!v0_xy) return set_err(HJ_ERR_INVALID_ARG, "v0_xy is NULL");
    const long long nxy = (long long)g->n[0] * g->n[1];
    if (count != (size_t)nxy) return set_err(HJ_ERR_INVALID_ARG, "count %zu != N1*N2 = %lld", count, nxy);
    if ((s = activate(g)) != HJ_OK) return s;
    if ((s = reset_state(g)) != HJ_OK) return s;
    double *staging = (double *)g->buf;  // N1*N2 doubles fit in the ping-pong region
    HJ_CUDA(cudaMemcpyAsync(staging, v0_xy, sizeof(double) * (size_t)nxy, cudaMemcpyHostToDevice, g->stream));
    return ingest_xy(g, staging, HJ_FP64, nxy);
}

hj_status hj_set_initial_value_xy_device(hj_grid *g, const void *v0_xy_device, hj_precision dtype, size_t count)
{
    g_err[0] = 0;
    hj_status s = check_grid(g);
    if (s != HJ_OK) return s;
    if (!v0_xy_device) return set_err(HJ_ERR_INVALID_ARG, "v0_xy_device is NULL");
    if (!valid_prec(dtype)) return set_err(HJ_ERR_INVALID_ARG, "unknown dtype");
    const long long nxy = (long long)g->n[0] * g->n[1];
    if (count != (size_t)nxy) return set_err(HJ_ERR_INVALID_ARG, "count %zu != N1*N2 = %lld", count, nxy);
    if ((s = activate(g)) != HJ_OK) return s;
    if ((s = follow_default_stream(g)) != HJ_OK) return s;
    if ((s = reset_state(g)) != HJ_OK) return s;
    return ingest_xy(g, v0_xy_device, dtype, nxy);
}

hj_status hj_set_initial_value_device(hj_grid *g, const void *v0_device, hj_precision dtype, size_t count)
{
    g_err[0] = 0;
    hj_status s = check_grid(g);
    if (s != HJ_OK) return s;
    if (!v0_device) return set_err(HJ_ERR_INVALID_ARG, "v0_device is NULL");
    if (!valid_prec(dtype)) return set_err(HJ_ERR_INVALID_ARG, "unknown dtype");
    if (count != (size_t)g->ncell)
        return set_err(HJ_ERR_INVALID_ARG, "count %zu != N1*N2*N3*N4 = %lld", count, g->ncell);
    if ((s = activate(g)) != HJ_OK) return s;
    if ((s = follow_default_stream(g)) != HJ_OK) return s;
    if ((s = reset_state(g)) != HJ_OK) return s;
    long long nrows = (long long)g->n[0] * g->n[1] * g->n[2];
    int *flag = &g->dstate->nonfinite;
    int blocks = grid_blocks(g->nint, 256);
    with_elem(dtype, [&](auto ein) {
        with_elem(g->prec, [&](auto e) {
            using Tin = decltype(ein);
            using T = decltype(e);
            ingest_kernel<Tin, T><<<blocks, 256, 0, g->stream>>>((const Tin *)v0_device, (T *)g->v0, g->n[3], g->p4,
                                                                 nrows, flag);
        });
    });
    set_v0_mode(g, false);
    return finish_ingest(g);
}

// The time loop of hj_advance_brt and hj_solve_converged (threshold > 0:
// Algorithm 2's convergence test ends the loop as well).
static hj_status advance_loop(hj_grid *g, double T, double cfl, int64_t max_steps, double threshold,
                              hj_solve_stats *stats);

static hj_status advance_impl(hj_grid *g, double T, double cfl, int64_t max_steps, double threshold,
                              hj_solve_stats *stats)
{
    // the step kernels that also reduce the change run only in this call
    g->track = threshold > 0.0;
    const hj_status s = advance_loop(g, T, cfl, max_steps, threshold, stats);
    g->track = false;
    return s;
}

static hj_status advance_loop(hj_grid *g, double T, double cfl, int64_t max_steps, double threshold,
                              hj_solve_stats *stats)
{
    hj_status s = HJ_OK;
    if (!isfinite(T) || T < 0) return set_err(HJ_ERR_INVALID_ARG, "T must be finite and >= 0");
    if (!isfinite(cfl) || !(cfl > 0) || cfl > 1) return set_err(HJ_ERR_INVALID_ARG, "cfl must be in (0, 1]");
    if (max_steps < 0) return set_err(HJ_ERR_INVALID_ARG, "max_steps must be >= 0");
    if (!g->has_dyn) return set_err(HJ_ERR_STATE, "hj_set_dynamics has not been called");
    if (!g->has_value) return set_err(HJ_ERR_STATE, "no initial value (hj_set_initial_value)");
    if ((s = activate(g)) != HJ_OK) return s;

    const hj_kernel kern = effective_kernel(g);
    int launches = 0;
    HJ_CUDA(cudaEventRecord(g->ev[0], g->stream));
    launch_prologue(g, T, cfl, threshold);
    ++launches;
    HJ_CUDA(cudaGetLastError());
    if ((s = pull_state(g)) != HJ_OK) return s;
    const long long n_start = g->hstate->n;
    const double dt_first = g->hstate->done ? 0.0 : g->hstate->dt;
    long long taken = 0;
    bool loop_started = false;
    while (!g->hstate->done && g->hstate->status == HJ_OK && taken < max_steps) {
        // predicted steps to the horizon (dt is constant until the cut last step)
        const HjDevState &h = *g->hstate;
        long long k = 1;
        if (!h.last && h.dt > 0) {
            double r = ceil((h.T - h.t) / h.dt);
            k = r > 1 ? (r < 1e15 ? (long long)r : (long long)1e15) : 1;
        }
        if (k > max_steps - taken) k = max_steps - taken;
        // the resident kernel ends the loop itself (horizon, convergence)
        if (kern == HJ_KERNEL_RESIDENT) k = max_steps - taken;
        if (threshold > 0.0 && k > 32 && kern != HJ_KERNEL_RESIDENT) k = 32;  // graphs: look every 32 steps
        if (k > (1 << 16)) k = 1 << 16;  // read the device state (and any error) at least this often
        if (!loop_started) {
            HJ_CUDA(cudaEventRecord(g->ev[1], g->stream));
            loop_started = true;
        }
        if (kern == HJ_KERNEL_RESIDENT) {
            HJ_CUDA(hj_launch_step_resident(g, k));
            ++launches;
        } else if (launch_steps_graph(g, kern, k)) {
            launches += (int)k;
        } else {
            for (long long i = 0; i < k; ++i) {
                if ((s = launch_step(g, kern)) != HJ_OK) return s;
                ++launches;
            }
        }
        HJ_CUDA(cudaEventRecord(g->ev[2], g->stream));
        if ((s = pull_state(g)) != HJ_OK) return s;
        taken = g->hstate->n - n_start;
    }
    HJ_CUDA(cudaEventRecord(g->ev[3], g->stream));
    HJ_CUDA(cudaEventSynchronize(g->ev[3]));
    const HjDevState &h = *g->hstate;
    if (h.status != HJ_OK)
        return set_err((hj_status)h.status, "device reported %s", hj_status_string((hj_status)h.status));
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->steps = h.n - n_start;
        stats->total_steps = h.n;
        stats->t_final = h.t;
        stats->dt_first = stats->steps > 0 ? dt_first : 0.0;
        stats->dt_last = stats->steps > 0 ? h.dt_prev : 0.0;
        for (int d = 0; d < 4; ++d) stats->alpha_max[d] = h.alpha_prev[d];
        float ms = 0.f;
        cudaEventElapsedTime(&ms, g->ev[0], g->ev[3]);
        stats->device_ms = ms;
        if (loop_started) {
            cudaEventElapsedTime(&ms, g->ev[1], g->ev[2]);
            stats->loop_ms = ms;
        }
        stats->kernel = kern;
        stats->launches = launches;
        stats->last_change = h.delta_last;
        stats->converged = h.converged;
    }
    return HJ_OK;
}

hj_status hj_advance_brt(hj_grid *g, double T, double cfl, int64_t max_steps, hj_solve_stats *stats)
{
    g_err[0] = 0;
    hj_status s = check_grid(g);
    if (s != HJ_OK) return s;
    return advance_impl(g, T, cfl, max_steps, 0.0, stats);
}

hj_status hj_solve_converged(hj_grid *g, double threshold, double T_max, double cfl, int64_t max_steps,
                             hj_solve_stats *stats)
{
    g_err[0] = 0;
    hj_status s = check_grid(g);
    if (s != HJ_OK) return s;
    if (!isfinite(threshold) || !(threshold > 0)) return set_err(HJ_ERR_INVALID_ARG, "threshold must be finite and > 0");
    return advance_impl(g, T_max, cfl, max_steps, threshold, stats);
}

hj_status hj_solve_brt(hj_grid *g, double T, double cfl, hj_solve_stats *stats)
{
    return hj_advance_brt(g, T, cfl, INT64_MAX, stats);
}

hj_status hj_read_value(const hj_grid *gc, double *out, size_t count)
{
    g_err[0] = 0;
    hj_grid *g = (hj_grid *)gc;
    hj_status s = check_grid(g);
    if (s != HJ_OK) return s;
    if (!out) return set_err(HJ_ERR_INVALID_ARG, "out is NULL");
    if (count != (size_t)g->ncell)
        return set_err(HJ_ERR_INVALID_ARG, "count %zu != N1*N2*N3*N4 = %lld", count, g->ncell);
    if (!g->has_value) return set_err(HJ_ERR_STATE, "no initial value (hj_set_initial_value)");
    if ((s = activate(g)) != HJ_OK) return s;
    if ((s = pull_state(g)) != HJ_OK) return s;
    const long long n = g->hstate->n;
    const void *src = hj_value_ptr(g, n);
    const long long nrows = (long long)g->n[0] * g->n[1] * g->n[2];
    // pinned host memory: the readback kernel writes it directly, in one pass
    if (double *dv = (double *)device_view(g, out)) {
        with_elem(g->prec, [&](auto e) {
            using T = decltype(e);
            readback_kernel<T, double><<<grid_blocks(nrows * g->n[3], 256), 256, 0, g->stream>>>(
                (const T *)src, dv, g->n[3], g->p4, 0, nrows);
        });
        HJ_CUDA(cudaGetLastError());
        HJ_CUDA(cudaStreamSynchronize(g->stream));
        return HJ_OK;
    }
    if (g->prec == HJ_FP64 && g->p4 == g->n[3]) {
        HJ_CUDA(cudaMemcpyAsync(out, src, sizeof(double) * (size_t)g->ncell, cudaMemcpyDeviceToHost, g->stream));
        HJ_CUDA(cudaStreamSynchronize(g->stream));
        return HJ_OK;
    }
    // convert in chunks of rows into a free buffer, then copy each chunk out
    void *free_buf;
    size_t free_bytes;
    if (n == 0) {
        free_buf = g->buf;
        free_bytes = 2 * (size_t)g->nint * g->esize;
    } else {
        free_buf = (char *)g->buf + (size_t)(n & 1) * g->nint * g->esize;  // the buffer the next step writes
        free_bytes = (size_t)g->nint * g->esize;
    }
    long long rows_per_chunk = (long long)(free_bytes / (sizeof(double) * (size_t)g->n[3]));
    if (rows_per_chunk < 1) return set_err(HJ_ERR_STATE, "no room to stage the readback");
    for (long long r0 = 0; r0 < nrows; r0 += rows_per_chunk) {
        long long nr = nrows - r0 < rows_per_chunk ? nrows - r0 : rows_per_chunk;
        int blocks = grid_blocks(nr * g->n[3], 256);
        with_elem(g->prec, [&](auto e) {
            using T = decltype(e);
            readback_kernel<T, double><<<blocks, 256, 0, g->stream>>>((const T *)src, (double *)free_buf, g->n[3],
                                                                      g->p4, r0, nr);
        });
        HJ_CUDA(cudaGetLastError());
        HJ_CUDA(cudaMemcpyAsync(out + r0 * g->n[3], free_buf, sizeof(double) * (size_t)(nr * g->n[3]),
                                cudaMemcpyDeviceToHost, g->stream));
    }
    HJ_CUDA(cudaStreamSynchronize(g->stream));
    return HJ_OK;
}

hj_status hj_query_device(const hj_grid *gc, const double *states, int64_t m, double *value, double *grad,
                          double *control)
{
    g_err[0] = 0;
    hj_grid *g = (hj_grid *)gc;
    hj_status s = check_grid(g);
    if (s != HJ_OK) return s;
    if (m < 0) return set_err(HJ_ERR_INVALID_ARG, "m must be >= 0");
    if (m > 0 && (!states || !value)) return set_err(HJ_ERR_INVALID_ARG, "states and value must not be NULL");
    if (!g->has_value) return set_err(HJ_ERR_STATE, "no initial value (hj_set_initial_value)");
    if (control && !g->has_dyn) return set_err(HJ_ERR_STATE, "the control needs the dynamics (hj_set_dynamics)");
    if ((s = activate(g)) != HJ_OK) return s;
    if ((s = follow_default_stream(g)) != HJ_OK) return s;
    if ((s = pull_state(g)) != HJ_OK) return s;
    HJ_CUDA(hj_launch_query(g, hj_value_ptr(g, g->hstate->n), states, m, value, grad, control));
    HJ_CUDA(cudaStreamSynchronize(g->stream));
    return HJ_OK;
}

hj_status hj_query(const hj_grid *gc, const double *states, int64_t m, double *value, double *grad, double *control)
{
    g_err[0] = 0;
    hj_grid *g = (hj_grid *)gc;
    hj_status s = check_grid(g);
    if (s != HJ_OK) return s;
    if (m < 0) return set_err(HJ_ERR_INVALID_ARG, "m must be >= 0");
    if (m > 0 && (!states || !value)) return set_err(HJ_ERR_INVALID_ARG, "states and value must not be NULL");
    if (!g->has_value) return set_err(HJ_ERR_STATE, "no initial value (hj_set_initial_value)");
    if (control && !g->has_dyn) return set_err(HJ_ERR_STATE, "the control needs the dynamics (hj_set_dynamics)");
    if ((s = activate(g)) != HJ_OK) return s;
    if ((s = pull_state(g)) != HJ_OK) return s;
    const long long n = g->hstate->n;
    // stage states and results in the buffer the next step writes (free now)
    char *free_buf;
    size_t free_bytes;
    if (n == 0) {
        free_buf = (char *)g->buf;
        free_bytes = 2 * (size_t)g->nint * g->esize;
    } else {
        free_buf = (char *)g->buf + (size_t)(n & 1) * g->nint * g->esize;
        free_bytes = (size_t)g->nint * g->esize;
    }
    const long long per = (long long)free_bytes / (11 * (long long)sizeof(double));
    if (per < 1) return set_err(HJ_ERR_STATE, "no room to stage the query");
    double *d_states = (double *)free_buf, *d_value = d_states + 4 * per, *d_grad = d_value + per,
           *d_ctl = d_grad + 4 * per;
    const void *V = hj_value_ptr(g, n);
    for (long long q0 = 0; q0 < m; q0 += per) {
        const long long k = m - q0 < per ? m - q0 : per;
        HJ_CUDA(cudaMemcpyAsync(d_states, states + 4 * q0, sizeof(double) * 4 * k, cudaMemcpyHostToDevice, g->stream));
        HJ_CUDA(hj_launch_query(g, V, d_states, k, d_value, grad ? d_grad : nullptr, control ? d_ctl : nullptr));
        HJ_CUDA(cudaMemcpyAsync(value + q0, d_value, sizeof(double) * k, cudaMemcpyDeviceToHost, g->stream));
        if (grad)
            HJ_CUDA(cudaMemcpyAsync(grad + 4 * q0, d_grad, sizeof(double) * 4 * k, cudaMemcpyDeviceToHost, g->stream));
        if (control)
            HJ_CUDA(cudaMemcpyAsync(control + 2 * q0, d_ctl, sizeof(double) * 2 * k, cudaMemcpyDeviceToHost,
                                    g->stream));
        HJ_CUDA(cudaStreamSynchronize(g->stream));  // the next chunk reuses the staging area
    }
    return HJ_OK;
}

hj_status hj_read_value_device(const hj_grid *gc, void *out_device, hj_precision dtype, size_t count)
{
    g_err[0] = 0;
    hj_grid *g = (hj_grid *)gc;
    hj_status s = check_grid(g);
    if (s != HJ_OK) return s;
    if (!out_device) return set_err(HJ_ERR_INVALID_ARG, "out_device is NULL");
    if (!valid_prec(dtype)) return set_err(HJ_ERR_INVALID_ARG, "unknown dtype");
    if (count != (size_t)g->ncell)
        return set_err(HJ_ERR_INVALID_ARG, "count %zu != N1*N2*N3*N4 = %lld", count, g->ncell);
    if (!g->has_value) return set_err(HJ_ERR_STATE, "no initial value (hj_set_initial_value)");
    if ((s = activate(g)) != HJ_OK) return s;
    if ((s = follow_default_stream(g)) != HJ_OK) return s;  // the output array too
    if ((s = pull_state(g)) != HJ_OK) return s;
    const void *src = hj_value_ptr(g, g->hstate->n);
    const long long nrows = (long long)g->n[0] * g->n[1] * g->n[2];
    int blocks = grid_blocks(g->ncell, 256);
    with_elem(g->prec, [&](auto e) {
        with_elem(dtype, [&](auto eout) {
            using T = decltype(e);
            using Tout = decltype(eout);
            readback_kernel<T, Tout><<<blocks, 256, 0, g->stream>>>((const T *)src, (Tout *)out_device, g->n[3], g->p4,
                                                                    0, nrows);
        });
    });
    HJ_CUDA(cudaGetLastError());
    HJ_CUDA(cudaStreamSynchronize(g->stream));
    return HJ_OK;
}

hj_status hj_set_kernel(hj_grid *g, hj_kernel kernel)
{
    g_err[0] = 0;
    hj_status s = check_grid(g);
    if (s != HJ_OK) return s;
    if (kernel != HJ_KERNEL_AUTO && kernel != HJ_KERNEL_GENERIC && kernel != HJ_KERNEL_TILED &&
        kernel != HJ_KERNEL_RESIDENT)
        return set_err(HJ_ERR_INVALID_ARG, "unknown kernel %d", (int)kernel);
    if (kernel == HJ_KERNEL_RESIDENT && !hj_resident_supported(g))
        return set_err(HJ_ERR_UNSUPPORTED, "the resident kernel needs cooperative launch and fewer than 2^32 cells");
    if (kernel == HJ_KERNEL_TILED && !g->tiled_ok)
        return set_err(HJ_ERR_UNSUPPORTED, "the tiled kernel does not support this grid (FP32 or Q5.27 car grids "
                                           "with periodic theta only; set the dynamics first)");
    g->kernel_req = kernel;
    return HJ_OK;
}

hj_status hj_set_tile_shape(hj_grid *g, const int32_t shape[4])
{
    g_err[0] = 0;
    hj_status s = check_grid(g);
    if (s != HJ_OK) return s;
    if (!shape) return set_err(HJ_ERR_INVALID_ARG, "shape is NULL");
    for (int i = 0; i < 4; ++i)
        if (shape[i] < 0 || shape[i] > 4096) return set_err(HJ_ERR_INVALID_ARG, "shape entries must be in [0, 4096]");
    if (!g->tiled_ok) return set_err(HJ_ERR_UNSUPPORTED, "this grid has no tiled kernel");
    if ((s = activate(g)) != HJ_OK) return s;
    HJ_CUDA(cudaStreamSynchronize(g->stream));
    int32_t old[4];
    memcpy(old, g->tile_req, sizeof(old));
    memcpy(g->tile_req, shape, sizeof(old));
    char why[160];
    if (!hj_tiled_setup(g, why, sizeof(why))) {
        memcpy(g->tile_req, old, sizeof(old));
        hj_tiled_setup(g, why, sizeof(why));
        return set_err(HJ_ERR_UNSUPPORTED, "tile shape rejected: %s", why);
    }
    return HJ_OK;
}

hj_status hj_autotune(hj_grid *g, int32_t steps_per_trial, hj_tile_result *results, int32_t max_results,
                      int32_t *nresults)
{
    g_err[0] = 0;
    hj_status s = check_grid(g);
    if (s != HJ_OK) return s;
    if (steps_per_trial < 1) return set_err(HJ_ERR_INVALID_ARG, "steps_per_trial must be >= 1");
    if (max_results < 0) return set_err(HJ_ERR_INVALID_ARG, "max_results must be >= 0");
    if (!g->tiled_ok) return set_err(HJ_ERR_UNSUPPORTED, "this grid has no tiled kernel");
    if (!g->has_value) return set_err(HJ_ERR_STATE, "no initial value (hj_set_initial_value)");
    if ((s = activate(g)) != HJ_OK) return s;
    if ((s = pull_state(g)) != HJ_OK) return s;
    if (g->hstate->n != 0) return set_err(HJ_ERR_STATE, "autotune must run before the first step");
    HjDevState saved = *g->hstate;
    int32_t keep[4];
    memcpy(keep, g->tile_req, sizeof(keep));

    // candidate (ty, tv): one consumer thread per (row, theta quad), at least
    // 8 warps; the 4 shapes with the fewest halo reads per row from each
    // launch-bound class of the tiled kernel (hj_tiled_variant)
    struct Cand {
        int ty, tv;
        double halo;
    } cands[17];
    int nc = 0;
    int class_hi[4];
    for (int i = 0; i < 4; ++i) class_hi[i] = hj_tiled_variant(g->prec == HJ_Q527, i);
    for (int cls = 0; cls < 4; ++cls) {
        Cand top[4];
        int nt = 0;
        for (int ty = 1; ty <= 16; ++ty)
            for (int tv = 1; tv <= 16; ++tv) {
                if (ty > g->n[1] || tv > g->n[2]) continue;
                const int th = hj_tiled_threads(g, ty, tv);
                if (th == 0) continue;
                const int cons = th - 32;
                if (cons < 256 || cons > class_hi[cls] || (cls > 0 && cons <= class_hi[cls - 1])) continue;
                const Cand c = {ty, tv, (double)(ty + 2) * (tv + 2) / (ty * tv)};
                if (nt < 4) {
                    top[nt++] = c;
                } else {
                    int worst = 0;
                    for (int i = 1; i < nt; ++i)
                        if (top[i].halo > top[worst].halo) worst = i;
                    if (c.halo < top[worst].halo) top[worst] = c;
                }
            }
        for (int i = 0; i < nt; ++i) cands[nc++] = top[i];
    }
    // and the default shape, which on a small grid trades halo reads for more
    // CTAs (the only candidate on a grid too small for the classes above)
    cands[nc++] = {0, 0, 0.0};

    auto run_steps = [&](int k) -> hj_status {
        *g->hstate = saved;
        HJ_CUDA(cudaMemcpyAsync(g->dstate, g->hstate, sizeof(HjDevState), cudaMemcpyHostToDevice, g->stream));
        launch_prologue(g, 1e300, 0.8);
        HJ_CUDA(cudaGetLastError());
        HJ_CUDA(cudaEventRecord(g->ev[1], g->stream));
        for (int i = 0; i < k; ++i) {
            hj_status r = launch_step(g, HJ_KERNEL_TILED);
            if (r != HJ_OK) return r;
        }
        HJ_CUDA(cudaEventRecord(g->ev[2], g->stream));
        HJ_CUDA(cudaEventSynchronize(g->ev[2]));
        return HJ_OK;
    };
    double best = 1e300;
    int32_t best_req[4] = {0, 0, 0, 0};
    int32_t count = 0;
    char why[160];
    for (int c = 0; c < nc; ++c) {
        int auto_xc = -1;
        for (int xc_mode = 0; xc_mode < 2; ++xc_mode) {
            g->tile_req[0] = cands[c].ty;
            g->tile_req[1] = cands[c].tv;
            g->tile_req[2] = xc_mode == 0 ? 0 : g->n[0];  // automatic chunks, or one chunk per column
            g->tile_req[3] = 0;
            if (!hj_tiled_setup(g, why, sizeof(why))) continue;
            if (xc_mode == 0) auto_xc = g->tile_xc;
            else if (g->tile_xc == auto_xc) continue;  // the automatic choice already was one chunk
            if ((s = run_steps(2)) != HJ_OK) break;  // warm-up
            if ((s = run_steps(steps_per_trial)) != HJ_OK) break;
            pull_state(g);
            if (g->hstate->status != HJ_OK) {
                s = set_err((hj_status)g->hstate->status, "device reported %s during autotune",
                            hj_status_string((hj_status)g->hstate->status));
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, g->ev[1], g->ev[2]);
            const double per = ms / steps_per_trial;
            if (results && count < max_results) {
                hj_tile_result &r = results[count];
                r.shape[0] = g->tile_ty;
                r.shape[1] = g->tile_tv;
                r.shape[2] = g->tile_xc;
                r.shape[3] = g->tile_stages;
                r.threads = hj_tiled_threads(g, g->tile_ty, g->tile_tv);
                r.ctas = g->tiled_ctas;
                r.ms_per_step = per;
                r.ms_retimed = 0.0;
            }
            ++count;
            if (per < best) {
                best = per;
                best_req[0] = g->tile_ty;
                best_req[1] = g->tile_tv;
                best_req[2] = g->tile_xc;
                best_req[3] = g->tile_stages;
            }
        }
        if (s != HJ_OK) break;
    }
    // second pass: re-time the three fastest shapes with three times the
    // steps and keep the best of those (single short trials are noisy)
    if (s == HJ_OK && results && count > 1) {
        int order[64];
        const int m = count < max_results ? (count < 64 ? count : 64) : (max_results < 64 ? max_results : 64);
        for (int i = 0; i < m; ++i) order[i] = i;
        for (int i = 0; i < m; ++i)
            for (int j = i + 1; j < m; ++j)
                if (results[order[j]].ms_per_step < results[order[i]].ms_per_step) {
                    const int t = order[i];
                    order[i] = order[j];
                    order[j] = t;
                }
        best = 1e300;
        for (int r = 0; r < 3 && r < m; ++r) {
            memcpy(g->tile_req, results[order[r]].shape, sizeof(g->tile_req));
            if (!hj_tiled_setup(g, why, sizeof(why))) continue;
            if ((s = run_steps(2)) != HJ_OK) break;
            if ((s = run_steps(3 * steps_per_trial)) != HJ_OK) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, g->ev[1], g->ev[2]);
            const double per = ms / (3 * steps_per_trial);
            results[order[r]].ms_retimed = per;
            if (per < best) {
                best = per;
                memcpy(best_req, results[order[r]].shape, sizeof(best_req));
            }
        }
    }
    // keep the winner (or the previous shape if nothing ran), restore the state
    if (best < 1e300)
        memcpy(g->tile_req, best_req, sizeof(best_req));
    else
        memcpy(g->tile_req, keep, sizeof(keep));
    if (!hj_tiled_setup(g, why, sizeof(why)) && s == HJ_OK)
        s = set_err(HJ_ERR_CUDA, "autotune: the chosen tile shape (%d, %d, %d, %d) was rejected: %s", g->tile_req[0],
                    g->tile_req[1], g->tile_req[2], g->tile_req[3], why);
    else if (s == HJ_OK && best < 1e300 &&
             (g->tile_ty != best_req[0] || g->tile_tv != best_req[1] || g->tile_xc != best_req[2] ||
              g->tile_stages != best_req[3]))
        s = set_err(HJ_ERR_CUDA, "autotune: tile shape (%d, %d, %d, %d) came out as (%d, %d, %d, %d)", best_req[0],
                    best_req[1], best_req[2], best_req[3], g->tile_ty, g->tile_tv, g->tile_xc, g->tile_stages);
    *g->hstate = saved;
    cudaMemcpyAsync(g->dstate, g->hstate, sizeof(HjDevState), cudaMemcpyHostToDevice, g->stream);
    cudaStreamSynchronize(g->stream);
    if (nresults) *nresults = count;
    return s;
}

hj_status hj_get_info(const hj_grid *g, hj_grid_info *info)
{
    g_err[0] = 0;
    hj_status s = check_grid(g);
    if (s != HJ_OK) return s;
    if (!info) return set_err(HJ_ERR_INVALID_ARG, "info is NULL");
    if ((s = activate(g)) != HJ_OK) return s;
    if ((s = pull_state((hj_grid *)g)) != HJ_OK) return s;
    memset(info, 0, sizeof(*info));
    for (int d = 0; d < 4; ++d) {
        info->n[d] = g->n[d];
        info->lo[d] = g->lo[d];
        info->hi[d] = g->hi[d];
        info->dx[d] = g->h[d];
    }
    info->pitch4 = g->p4;
    info->precision = g->prec;
    info->v0_broadcast = g->v0_bcast ? 1 : 0;
    info->kernel = effective_kernel(g);
    info->periodic_mask = g->periodic;
    info->has_value = g->has_value;
    info->total_steps = g->hstate->n;
    info->t = g->hstate->t;
    info->device_bytes = g->device_bytes;
    if (g->tiled_ok) {
        info->tile[0] = g->tile_ty;
        info->tile[1] = g->tile_tv;
        info->tile[2] = g->tile_xc;
        info->tile[3] = g->tile_stages;
        info->tile_ctas = g->tiled_ctas;
    }
    return HJ_OK;
}

}  // extern "C"
