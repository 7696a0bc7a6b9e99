// hj_step_noalloc: one time step on caller-owned device arrays, without
// allocating any memory.
//
// Some callers cannot allocate device memory: code that runs inside a
// framework whose device memory belongs to its own pool or allocator, code
// on a memory budget fixed at start-up, or code driven from a context where
// a cudaMalloc would synchronise the device at the wrong time.  This entry
// point takes the caller's arrays for V_n, V0 and V_{n+1} and keeps its own
// working data (the per-(v, theta) coefficient table and the alpha^max
// accumulators) in a file-scope device array of fixed size, which every GPU
// that loads the library holds until the process exits.
//
// The arithmetic per cell is the generic step kernel's (one step of
// Algorithm 2 in upwind form, hj_step_generic.cu), on the dense layout of the
// C ABI (no row padding).  The coefficient table is computed on the device
// from the grid and the dynamics (device cos/sin), so results agree with the
// grid API to rounding of the tables (FP64: far below 1e-12).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "hj_device.cuh"

namespace {

// Scratch: the state block, then the coefficient table (FP64 entries at most).
constexpr int NOALLOC_MAX_COEF = 16384;  // N3 * N4 at most
constexpr size_t NOALLOC_STATE_BYTES = 256;
constexpr size_t NOALLOC_BYTES = NOALLOC_STATE_BYTES + (size_t)NOALLOC_MAX_COEF * sizeof(HjCoef<double>);

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

static_assert(sizeof(HjDevState) <= NOALLOC_STATE_BYTES, "state block too small");

// Device address of the scratch array, per device, set up on the first call
// made with that device current.
std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[64] = {nullptr};

// Clears the accumulators and fills the coefficient table (c1, c2 signed
// xdot/dx on axes 1-2, ks = sum of |xdot_d|/dx_d, a1, a2 = |xdot_1|, |xdot_2|).
template <typename T>
__global__ void noalloc_init_kernel(HjDevState *st, HjCoef<T> *coef, const HjGeom g, double lo3, double lo4, int car,
                                    double c1, double c2)
{
    const int ncoef = g.n3 * g.n4;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->alpha_bits[0] = 0ull;
        st->alpha_bits[1] = 0ull;
        st->blocks_done = 0u;
        st->status = HJ_OK;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncoef; i += gridDim.x * blockDim.x) {
        const int k = i / g.n4, l = i - (i / g.n4) * g.n4;
        double f1 = c1, f2 = c2;
        if (car) {
            const double v = lo3 + (double)k * g.h[2], th = lo4 + (double)l * g.h[3];
            f1 = v * cos(th);
            f2 = v * sin(th);
        }
        const double q1 = f1 / g.h[0], q2 = f2 / g.h[1];
        HjCoef<T> c;
        c.c1 = (T)q1;
        c.c2 = (T)q2;
        c.ks = (T)(fabs(q1) + fabs(q2) + g.k3 + g.k4);
        c.a1 = fabs(f1);
        c.a2 = fabs(f2);
        coef[i] = c;
    }
}

__device__ __forceinline__ float noalloc_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double noalloc_fma(double a, double b, double c) { return fma(a, b, c); }

template <typename T>
__device__ __forceinline__ T noalloc_upwind(T p, T m, int mode)
{
    if (mode == HJ_AXIS_CONTROL) return hj_max(p, m);
    return mode == HJ_AXIS_PLUS ? p : m;
}

// One step from vin into vout (dense layout) and the block-reduced alpha^max
// partials, atomically merged into the scratch state.
template <typename T>
__global__ void __launch_bounds__(256) noalloc_step_kernel(const T *__restrict__ vin, const T *__restrict__ v0,
                                                           T *__restrict__ vout, const HjCoef<T> *__restrict__ coef,
                                                           HjDevState *st, const HjGeom g, double dtd)
{
    __shared__ unsigned long long scratch[64];
    const T dt = (T)dtd;
    const unsigned int N1 = g.n1, N2 = g.n2, N3 = g.n3, N4 = g.n4;
    const long long s3 = N4, s2 = (long long)N3 * N4, s1 = (long long)N2 * s2;
    const unsigned long long ncell = (unsigned long long)N1 * N2 * N3 * N4;
    const T k3 = (T)g.k3, k4 = (T)g.k4;
    unsigned long long am1 = 0ull, am2 = 0ull;
    for (unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; c < ncell;
         c += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long row = c / N4;
        const int l = (int)(c - row * N4);
        const unsigned long long r2 = row / N3;
        const int k = (int)(row - r2 * N3);
        const int i = (int)(r2 / N2);
        const int j = (int)(r2 - (unsigned long long)i * N2);
        const long long o = (long long)c;
        const T vc = vin[o];
        const int idx[4] = {i, j, k, l};
        const long long str[4] = {s1, s2, s3, 1};
        const int nn[4] = {(int)N1, (int)N2, (int)N3, (int)N4};
        T m[4], p[4];
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const bool per = (g.periodic >> d) & 1;
            if (idx[d] > 0) m[d] = vin[o - str[d]];
            else m[d] = per ? vin[o + (long long)(nn[d] - 1) * str[d]] : T(2) * vc - vin[o + str[d]];
            if (idx[d] < nn[d] - 1) p[d] = vin[o + str[d]];
            else p[d] = per ? vin[o - (long long)(nn[d] - 1) * str[d]] : T(2) * vc - vin[o - str[d]];
        }
        const HjCoef<T> cf = coef[k * N4 + l];
        const T u1 = cf.c1 >= T(0) ? p[0] : m[0];
        const T u2 = cf.c2 >= T(0) ? p[1] : m[1];
        const T u3 = noalloc_upwind<T>(p[2], m[2], g.mode3);
        const T u4 = noalloc_upwind<T>(p[3], m[3], g.mode4);
        const T K1 = cf.c1 >= T(0) ? cf.c1 : -cf.c1;
        const T K2 = cf.c2 >= T(0) ? cf.c2 : -cf.c2;
        T r = K1 * (u1 - vc);
        r = noalloc_fma(K2, u2 - vc, r);
        r = noalloc_fma(k3, u3 - vc, r);
        r = noalloc_fma(k4, u4 - vc, r);
        vout[o] = hj_min(v0[o], noalloc_fma(dt, r, vc));
        const unsigned long long b1 = hj_abits(cf.a1), b2 = hj_abits(cf.a2);
        am1 = am1 > b1 ? am1 : b1;
        am2 = am2 > b2 ? am2 : b2;
    }
    am1 = hj_warp_max_u64(am1);
    am2 = hj_warp_max_u64(am2);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        scratch[warp] = am1;
        scratch[32 + warp] = am2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            am1 = am1 > scratch[w] ? am1 : scratch[w];
            am2 = am2 > scratch[32 + w] ? am2 : scratch[32 + w];
        }
        atomicMax(&st->alpha_bits[0], am1);
        atomicMax(&st->alpha_bits[1], am2);
    }
}

}  // namespace

// Errors are reported through hj_last_error() like every other entry point.
static hj_status noalloc_fail(hj_status s, const char *msg)
{
    hj_internal_set_error(msg);
    return s;
}

static hj_status hj_noalloc_setup_ptr(void **out, int *dev_out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return noalloc_fail(HJ_ERR_CUDA, "hj_step_noalloc: no usable current CUDA device");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            char m[200];
            snprintf(m, sizeof(m), "hj_step_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return noalloc_fail(HJ_ERR_CUDA, m);
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    *dev_out = dev;
    return HJ_OK;
}

extern "C" {

hj_status hj_step_noalloc(const int32_t n[4], const double lo[4], const double hi[4], uint32_t periodic_mask,
                          hj_precision prec, hj_dynamics kind, const double *params, int32_t nparams,
                          const void *v_in, const void *v0, void *v_out, size_t bytes, double dt,
                          void *cuda_stream, double alpha_max_out[4])
{
    hj_internal_set_error("");
    (void)cudaGetLastError();  // an error pending from the caller's earlier work is not this call's
    if (!n || !lo || !hi || !params || !v_in || !v0 || !v_out)
        return noalloc_fail(HJ_ERR_INVALID_ARG, "hj_step_noalloc: NULL argument");
    if (prec != HJ_FP64 && prec != HJ_FP32) return noalloc_fail(HJ_ERR_INVALID_ARG, "hj_step_noalloc: unknown precision");
    if (periodic_mask & ~0xFu) return noalloc_fail(HJ_ERR_INVALID_ARG, "hj_step_noalloc: periodic_mask has bits above 3");
    long long ncell = 1;
    for (int d = 0; d < 4; ++d) {
        if (n[d] < 3) return noalloc_fail(HJ_ERR_INVALID_ARG, "hj_step_noalloc: every N_d must be >= 3");
        if (!isfinite(lo[d]) || !isfinite(hi[d]) || !(hi[d] > lo[d]))
            return noalloc_fail(HJ_ERR_INVALID_ARG, "hj_step_noalloc: bounds must be finite with hi > lo");
        ncell *= n[d];
    }
    if ((long long)n[2] * n[3] > NOALLOC_MAX_COEF)
        return noalloc_fail(HJ_ERR_INVALID_ARG,
                            "hj_step_noalloc: N3 * N4 exceeds 16384, the size of its fixed working array");
    if (ncell > (1LL << 33)) return noalloc_fail(HJ_ERR_INVALID_ARG, "hj_step_noalloc: grid too large");
    const size_t want_bytes = (size_t)ncell * (prec == HJ_FP64 ? sizeof(double) : sizeof(float));
    if (bytes != want_bytes)
        return noalloc_fail(HJ_ERR_INVALID_ARG,
                            "hj_step_noalloc: bytes must equal N1*N2*N3*N4 times the element size of prec");
    {
        // v_out is written while v_in and v0 are read: the ranges must be disjoint
        const uintptr_t o0 = (uintptr_t)v_out, o1 = o0 + bytes;
        const uintptr_t i0 = (uintptr_t)v_in, z0 = (uintptr_t)v0;
        if ((i0 < o1 && o0 < i0 + bytes) || (z0 < o1 && o0 < z0 + bytes))
            return noalloc_fail(HJ_ERR_INVALID_ARG, "hj_step_noalloc: v_out overlaps v_in or v0");
    }
    if (!isfinite(dt) || dt < 0) return noalloc_fail(HJ_ERR_INVALID_ARG, "hj_step_noalloc: dt must be finite and >= 0");
    if (kind == HJ_DYN_CAR4D) {
        if (nparams != 2 || !isfinite(params[0]) || !isfinite(params[1]) || params[0] < 0 || params[1] < 0)
            return noalloc_fail(HJ_ERR_INVALID_ARG, "hj_step_noalloc: car dynamics take a_max, w_max >= 0");
    } else if (kind == HJ_DYN_CONST) {
        if (nparams != 4) return noalloc_fail(HJ_ERR_INVALID_ARG, "hj_step_noalloc: constant dynamics take 4 values");
        for (int i = 0; i < 4; ++i)
            if (!isfinite(params[i])) return noalloc_fail(HJ_ERR_INVALID_ARG, "hj_step_noalloc: non-finite parameter");
    } else {
        return noalloc_fail(HJ_ERR_INVALID_ARG, "hj_step_noalloc: unknown dynamics");
    }

    void *base = nullptr;
    int dev = 0;
    hj_status s = hj_noalloc_setup_ptr(&base, &dev);
    if (s != HJ_OK) return s;
    HjDevState *st = (HjDevState *)base;
    void *coef = (unsigned char *)base + NOALLOC_STATE_BYTES;
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    HjGeom G;
    memset(&G, 0, sizeof(G));
    G.n1 = n[0];
    G.n2 = n[1];
    G.n3 = n[2];
    G.n4 = n[3];
    G.p4 = n[3];
    G.periodic = (int32_t)periodic_mask;
    for (int d = 0; d < 4; ++d) {
        const bool per = (periodic_mask >> d) & 1u;
        G.h[d] = (hi[d] - lo[d]) / (double)(per ? n[d] : n[d] - 1);
    }
    const bool car = kind == HJ_DYN_CAR4D;
    if (car) {
        G.mode3 = G.mode4 = HJ_AXIS_CONTROL;
        G.alpha3 = params[0];
        G.alpha4 = params[1];
    } else {
        G.mode3 = params[2] >= 0 ? HJ_AXIS_PLUS : HJ_AXIS_MINUS;
        G.mode4 = params[3] >= 0 ? HJ_AXIS_PLUS : HJ_AXIS_MINUS;
        G.alpha3 = fabs(params[2]);
        G.alpha4 = fabs(params[3]);
    }
    G.k3 = G.alpha3 / G.h[2];
    G.k4 = G.alpha4 / G.h[3];
    const double c1 = car ? 0.0 : params[0], c2 = car ? 0.0 : params[1];

    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long want = (ncell + 255) / 256, cap = (long long)(sms > 0 ? sms : 1) * 8;
    const int blocks = (int)(want < cap ? want : cap);
    if (prec == HJ_FP64) {
        noalloc_init_kernel<double><<<64, 256, 0, stream>>>(st, (HjCoef<double> *)coef, G, lo[2], lo[3], car, c1, c2);
        noalloc_step_kernel<double><<<blocks, 256, 0, stream>>>((const double *)v_in, (const double *)v0,
                                                               (double *)v_out, (const HjCoef<double> *)coef, st, G,
                                                               dt);
    } else {
        noalloc_init_kernel<float><<<64, 256, 0, stream>>>(st, (HjCoef<float> *)coef, G, lo[2], lo[3], car, c1, c2);
        noalloc_step_kernel<float><<<blocks, 256, 0, stream>>>((const float *)v_in, (const float *)v0, (float *)v_out,
                                                              (const HjCoef<float> *)coef, st, G, dt);
    }
    cudaError_t e = cudaGetLastError();
    unsigned long long bits[2] = {0ull, 0ull};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bits, st->alpha_bits, sizeof(bits), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        char m[200];
        snprintf(m, sizeof(m), "hj_step_noalloc: %s", cudaGetErrorString(e));
        return noalloc_fail(HJ_ERR_CUDA, m);
    }
    if (alpha_max_out) {
        double a0, a1;
        memcpy(&a0, &bits[0], sizeof(double));
        memcpy(&a1, &bits[1], sizeof(double));
        alpha_max_out[0] = a0;
        alpha_max_out[1] = a1;
        alpha_max_out[2] = G.alpha3;
        alpha_max_out[3] = G.alpha4;
    }
    return HJ_OK;
}

}  // extern "C"
