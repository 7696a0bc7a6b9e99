// Tiled FP32 HJ step kernel for sm_103a (the HBM-bound fast path).
//
// Same per-cell arithmetic as the generic kernel (one step of Algorithm 2 of
// arxiv 2012.04011 in upwind form, see hj_step_generic.cu), organised for
// bandwidth:
//   * A CTA owns a column of the grid: TY rows of y x TV rows of v x the full
//     theta row (so the periodic wrap stays inside the tile), and streams it
//     along x (the slowest axis), plane by plane.
//   * A producer warp loads each plane's tile plus its one-cell y/v halo as
//     one 4D TMA box (cp.async.bulk.tensor.4d) into a ring of shared-memory
//     stages guarded by mbarriers (full: bytes landed, empty: consumers done).
//     Out-of-range halo rows come back zero-filled and are replaced by
//     extrapolated ghosts.
//   * Consumer threads each own a theta quad (float4) of up to MAXR rows; the
//     x-1 / x / x+1 centres stay in registers, y/v/theta neighbours come from
//     the plane's stage.  V0 is streamed with float4 loads one plane ahead,
//     V_new is written with float4 stores.  Every V value is read from HBM
//     once per step; halos are served by shared memory and L2.
//   * All CTAs of a step sweep x concurrently (one column per CTA when there
//     are enough columns), so y/v halo rows of neighbouring columns are in
//     L2 when they are needed.
//   * alpha^max partials (|xdot_1|, |xdot_2| over the (v, theta) states of the
//     cells each thread updates) are reduced by warp shuffles and a block
//     reduction, and the last CTA computes the next CFL step (fused; no extra
//     pass over the grid).
// Every mbarrier wait is bounded by %globaltimer; on timeout the kernel
// records HJ_ERR_TIMEOUT in the device state, stops issuing work, waits
// (bounded) for its own copies in flight and returns.
#include <stdio.h>
#include <string.h>

#include "hj_device.cuh"

namespace {

constexpr int MAXR = 4;                 // rows per consumer thread
constexpr int MAX_STAGES = 8;
constexpr unsigned long long WAIT_NS = 4000000000ull;  // 4 s per wait: far beyond any healthy wait

struct TiledParams {
    int ty, tv;           // tile rows along y and v
    int xc;               // planes per work item
    int q4;               // float4 per theta row (p4 / 4)
    int rg;               // row groups: consumer thread t owns quad t % q4 of rows t / q4 + rg * m
    int nconsumer;        // consumer threads (multiple of 32)
    int stages;           // shared-memory ring depth
    int ncol_v, ncol;     // tiles along v; columns in total
    int nchunk, nitems;   // x chunks per column; work items = ncol * nchunk
    int stage_floats;     // p4 * (tv + 2) * (ty + 2)
    int stage_bytes;      // stage_floats * 4 rounded up to 128
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase with the given parity; false if the deadline passed.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned long long deadline)
{
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() > deadline) return false;
    }
    return true;
}
// Warp-uniform version for consumer warps: every lane observes the phase,
// and the timeout decision is the same for the whole warp.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t *bar, uint32_t parity, unsigned long long deadline)
{
    while (true) {
        bool done = mbar_try_wait(bar, parity);
        if (__all_sync(0xffffffffu, done)) return true;
        bool late = global_ns() > deadline;
        if (__any_sync(0xffffffffu, late)) return false;
    }
}
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1, int c2,
                                            int c3)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ float f4get(const float4 &v, int e)
{
    return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}
__device__ __forceinline__ void f4set(float4 &v, int e, float x)
{
    if (e == 0) v.x = x;
    else if (e == 1) v.y = x;
    else if (e == 2) v.z = x;
    else v.w = x;
}
__device__ __forceinline__ float4 f4ghost(const float4 &c, const float4 &o)
{
    return make_float4(2.f * c.x - o.x, 2.f * c.y - o.y, 2.f * c.z - o.z, 2.f * c.w - o.w);
}

struct ItemGeom {
    int y0, v0, x0, x1, pl0, pl1;
};

__device__ __forceinline__ ItemGeom item_geom(const TiledParams &P, const HjGeom &g, int item)
{
    ItemGeom it;
    int col = item % P.ncol, chunk = item / P.ncol;
    it.y0 = (col / P.ncol_v) * P.ty;
    it.v0 = (col % P.ncol_v) * P.tv;
    it.x0 = chunk * P.xc;
    it.x1 = min(it.x0 + P.xc, g.n1);
    it.pl0 = max(it.x0 - 1, 0);
    it.pl1 = min(it.x1, g.n1 - 1);
    return it;
}

__global__ void __launch_bounds__(256) hj_step_tiled_kernel(const __grid_constant__ CUtensorMap map_v0,
                                                             const __grid_constant__ CUtensorMap map_a,
                                                             const __grid_constant__ CUtensorMap map_b,
                                                             const float *__restrict__ v0, float *__restrict__ buf,
                                                             const HjCoef<float> *__restrict__ coef,
                                                             const float *__restrict__ tab, HjDevState *st,
                                                             const HjGeom g, const TiledParams P, long long nint)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    if (st->done) return;  // uniform across the grid

    // ---- shared memory carve-up
    float *stages = (float *)smem_raw;
    uint64_t *full = (uint64_t *)(smem_raw + (size_t)P.stages * P.stage_bytes);
    uint64_t *empty = full + MAX_STAGES;
    unsigned long long *scratch = (unsigned long long *)(empty + MAX_STAGES);
    float *vtab = (float *)(scratch + 64);
    volatile int *abort_flag = (volatile int *)(vtab + g.n3);

    const long long n = st->n;
    const float dt = (float)st->dt;
    const float *vin_unused;
    float *vout;
    hj_io_buffers<float>(v0, buf, nint, n, vin_unused, vout);
    const CUtensorMap *map_in = (n == 0) ? &map_v0 : (((n - 1) & 1) ? &map_b : &map_a);

    const int tid = threadIdx.x;
    const int nconsumer_warps = P.nconsumer >> 5;
    if (tid == 0) {
        for (int s = 0; s < P.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], nconsumer_warps);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    for (int k = tid; k < g.n3; k += blockDim.x) vtab[k] = tab[k];
    __syncthreads();

    const unsigned long long deadline = global_ns() + WAIT_NS;
    unsigned long long am1 = 0ull, am2 = 0ull;

    if (tid >= P.nconsumer) {
        // ------------------------------------------------------------ producer
        if (tid == P.nconsumer) {
            uint32_t seq = 0;
            int last_seq[MAX_STAGES];
            for (int s = 0; s < MAX_STAGES; ++s) last_seq[s] = -1;
            bool ok = true;
            for (int item = blockIdx.x; item < P.nitems && ok; item += gridDim.x) {
                ItemGeom it = item_geom(P, g, item);
                for (int p = it.pl0; p <= it.pl1; ++p, ++seq) {
                    int s = seq % P.stages;
                    uint32_t ph = (seq / P.stages) & 1u;
                    if (seq >= (uint32_t)P.stages && !mbar_wait(&empty[s], ph ^ 1u, deadline)) {
                        ok = false;
                        break;
                    }
                    if (*abort_flag) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[s], (uint32_t)(P.stage_floats * 4));
                    tma_load_4d(stages + (size_t)s * (P.stage_bytes / 4), map_in, &full[s], 0, it.v0 - 1,
                                it.y0 - 1, p);
                    last_seq[s] = (int)seq;
                }
            }
            if (!ok) {
                st->status = HJ_ERR_TIMEOUT;
                *abort_flag = 1;
            }
            // drain: every copy this CTA issued must land before the CTA exits
            const unsigned long long drain_deadline = global_ns() + WAIT_NS;
            for (int s = 0; s < P.stages; ++s)
                if (last_seq[s] >= 0 && !mbar_wait(&full[s], ((uint32_t)last_seq[s] / P.stages) & 1u, drain_deadline))
                    st->status = HJ_ERR_TIMEOUT;
        }
    } else {
        // ------------------------------------------------------------ consumers
        const int lane = tid & 31;
        const bool active = tid < P.q4 * P.rg;
        const int q = tid % P.q4;
        const int rgid = tid / P.q4;
        const int N1 = g.n1, N2 = g.n2, N3 = g.n3, N4 = g.n4, P4 = g.p4;
        const int rows = P.ty * P.tv;
        const int srow = P.tv + 2;  // smem rows per y row
        const float k3 = (float)g.k3, k4 = (float)g.k4;
        const long long s1 = (long long)N2 * N3 * P4, s2 = (long long)N3 * P4;

        // this thread's theta states: cos/dx1 and sin/dx2 of its quad
        float ch[4], sh[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            ch[e] = tab[N3 + 4 * q + e];
            sh[e] = tab[N3 + P4 + 4 * q + e];
        }
        const int lm = (4 * q - 1 + N4) % N4;    // theta index left of the quad
        const int lp = (4 * q + 4) % N4;         // right of the quad
        const int lreal = min(4, N4 - 4 * q);    // real lanes in the quad (< 4 only in a padded last quad)

        uint32_t seq = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < P.nitems && ok; item += gridDim.x) {
            const ItemGeom it = item_geom(P, g, item);
            const uint32_t seq0 = seq;
            seq += (uint32_t)(it.pl1 - it.pl0 + 1);

            // rows of this thread
            int rsm[MAXR];       // smem row index of the centre
            int ry[MAXR], rv[MAXR];
            bool rok[MAXR];
#pragma unroll
            for (int m = 0; m < MAXR; ++m) {
                int r = rgid + P.rg * m;
                int jy = r / P.tv, kv = r - jy * P.tv;
                ry[m] = it.y0 + jy;
                rv[m] = it.v0 + kv;
                rok[m] = active && r < rows && ry[m] < N2 && rv[m] < N3;
                // rows this thread does not own read a harmless in-tile row
                rsm[m] = rok[m] ? (jy + 1) * srow + (kv + 1) : srow + 1;
            }
            // alpha partials over this thread's (v, theta) states
#pragma unroll
            for (int m = 0; m < MAXR; ++m)
                if (rok[m])
                    for (int e = 0; e < lreal; ++e) {
                        const HjCoef<float> c = coef[rv[m] * N4 + 4 * q + e];
                        unsigned long long b1 = hj_abits((double)c.a1), b2 = hj_abits((double)c.a2);
                        am1 = am1 > b1 ? am1 : b1;
                        am2 = am2 > b2 ? am2 : b2;
                    }

            auto stage_of = [&](int p) -> float * {
                return stages + (size_t)((seq0 + (uint32_t)(p - it.pl0)) % P.stages) * (P.stage_bytes / 4);
            };
            auto wait_plane = [&](int p) -> bool {
                uint32_t sq = seq0 + (uint32_t)(p - it.pl0);
                return mbar_wait_warp(&full[sq % P.stages], (sq / P.stages) & 1u, deadline);
            };
            auto release_plane = [&](int p) {
                uint32_t sq = seq0 + (uint32_t)(p - it.pl0);
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[sq % P.stages]);
            };

            float4 prev[MAXR], cur[MAXR], nxt[MAXR], v0c[MAXR], v0n[MAXR];
            // item prologue: planes x0-1 (if any) and x0
            if (!wait_plane(it.pl0)) ok = false;
            if (ok && it.x0 > it.pl0 && !wait_plane(it.x0)) ok = false;
            if (!ok) break;
            {
                const float *sc = stage_of(it.x0);
                const float *sp = stage_of(it.pl0);
#pragma unroll
                for (int m = 0; m < MAXR; ++m) {
                    cur[m] = *(const float4 *)(sc + rsm[m] * P4 + 4 * q);
                    prev[m] = *(const float4 *)(sp + rsm[m] * P4 + 4 * q);  // == cur when x0 == 0 (ghost set below)
                    const long long o = ((long long)it.x0 * N2 + ry[m]) * s2 + (long long)rv[m] * P4 + 4 * q;
                    v0c[m] = rok[m] ? __ldcs((const float4 *)(v0 + o)) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            if (it.x0 > it.pl0) release_plane(it.pl0);

            for (int x = it.x0; x < it.x1; ++x) {
                if (__any_sync(0xffffffffu, *abort_flag != 0)) {
                    ok = false;
                    break;
                }
                const float *sx = stage_of(x);
                // centre of plane x+1, or the extrapolated ghost past the end
                if (x + 1 <= N1 - 1) {
                    if (!wait_plane(x + 1)) {
                        ok = false;
                        break;
                    }
                    const float *sn = stage_of(x + 1);
#pragma unroll
                    for (int m = 0; m < MAXR; ++m) nxt[m] = *(const float4 *)(sn + rsm[m] * P4 + 4 * q);
                } else {
#pragma unroll
                    for (int m = 0; m < MAXR; ++m) nxt[m] = f4ghost(cur[m], prev[m]);
                }
                if (x == 0) {
#pragma unroll
                    for (int m = 0; m < MAXR; ++m) prev[m] = f4ghost(cur[m], nxt[m]);
                }
                // V0 one plane ahead
                if (x + 1 < it.x1) {
#pragma unroll
                    for (int m = 0; m < MAXR; ++m) {
                        const long long o = ((long long)(x + 1) * N2 + ry[m]) * s2 + (long long)rv[m] * P4 + 4 * q;
                        v0n[m] = rok[m] ? __ldcs((const float4 *)(v0 + o)) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
#pragma unroll
                for (int m = 0; m < MAXR; ++m) {
                    if (!rok[m]) continue;
                    const float *row = sx + rsm[m] * P4;
                    const float4 c = cur[m];
                    float4 ym = *(const float4 *)(row - srow * P4 + 4 * q);
                    float4 yp = *(const float4 *)(row + srow * P4 + 4 * q);
                    float4 vm = *(const float4 *)(row - P4 + 4 * q);
                    float4 vp = *(const float4 *)(row + P4 + 4 * q);
                    if (ry[m] == 0) ym = f4ghost(c, yp);
                    if (ry[m] == N2 - 1) yp = f4ghost(c, ym);
                    if (rv[m] == 0) vm = f4ghost(c, vp);
                    if (rv[m] == N3 - 1) vp = f4ghost(c, vm);
                    const float tl = row[lm], tr = row[lp], t0 = row[0];
                    const float vk = vtab[rv[m]];
                    float4 out;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float vc = f4get(c, e);
                        const float tm = e == 0 ? tl : f4get(c, e - 1);
                        float tp = e == 3 ? tr : f4get(c, e + 1);
                        if (e == lreal - 1 && lreal < 4) tp = t0;  // wrap of a padded last quad
                        const float C1 = vk * ch[e], C2 = vk * sh[e];
                        const float u1 = C1 >= 0.f ? f4get(nxt[m], e) : f4get(prev[m], e);
                        const float u2 = C2 >= 0.f ? f4get(yp, e) : f4get(ym, e);
                        const float u3 = fmaxf(f4get(vp, e), f4get(vm, e));
                        const float u4 = fmaxf(tp, tm);
                        float r = fabsf(C1) * (u1 - vc);
                        r = fmaf(fabsf(C2), u2 - vc, r);
                        r = fmaf(k3, u3 - vc, r);
                        r = fmaf(k4, u4 - vc, r);
                        float vn = fminf(f4get(v0c[m], e), fmaf(dt, r, vc));
                        f4set(out, e, e < lreal ? vn : 0.f);
                    }
                    const long long o = ((long long)x * N2 + ry[m]) * s2 + (long long)rv[m] * P4 + 4 * q;
                    *(float4 *)(vout + o) = out;
                }
                release_plane(x);
#pragma unroll
                for (int m = 0; m < MAXR; ++m) {
                    prev[m] = cur[m];
                    cur[m] = nxt[m];
                    v0c[m] = v0n[m];
                }
            }
            if (!ok) break;
            if (it.x1 <= it.pl1) release_plane(it.x1);
        }
        if (!ok) {
            st->status = HJ_ERR_TIMEOUT;
            *abort_flag = 1;
        }
        (void)s1;
    }
    hj_step_epilogue(st, g, am1, am2, scratch);
}

size_t tiled_smem_bytes(const TiledParams &P, int n3)
{
    return (size_t)P.stages * P.stage_bytes + 2 * MAX_STAGES * sizeof(uint64_t) + 64 * sizeof(unsigned long long) +
           (size_t)n3 * sizeof(float) + 16;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

TiledParams make_params(const hj_grid *g, int ty, int tv, int stages, int slots)
{
    TiledParams P;
    memset(&P, 0, sizeof(P));
    P.ty = ty;
    P.tv = tv;
    P.stages = stages;
    P.q4 = g->p4 / 4;
    int rows = ty * tv;
    P.rg = (rows + MAXR - 1) / MAXR;
    P.nconsumer = ((P.q4 * P.rg + 31) / 32) * 32;
    P.ncol_v = (g->n[2] + tv - 1) / tv;
    P.ncol = ((g->n[1] + ty - 1) / ty) * P.ncol_v;
    P.stage_floats = g->p4 * (tv + 2) * (ty + 2);
    P.stage_bytes = ((P.stage_floats * 4 + 127) / 128) * 128;
    // enough work items to fill every CTA slot, but at least 4 planes per item
    int nchunk = 1;
    if (P.ncol * 4 < slots * 3) nchunk = (slots + P.ncol - 1) / P.ncol;
    int xc = (g->n[0] + nchunk - 1) / nchunk;
    if (xc < 4) xc = 4;
    P.xc = xc;
    P.nchunk = (g->n[0] + xc - 1) / xc;
    P.nitems = P.ncol * P.nchunk;
    return P;
}

}  // namespace

static TiledParams params_of(const hj_grid *g)
{
    TiledParams P = make_params(g, g->tile_ty, g->tile_tv, g->tile_stages, 0);
    P.xc = g->tile_xc;
    P.nchunk = (g->n[0] + P.xc - 1) / P.xc;
    P.nitems = P.ncol * P.nchunk;
    return P;
}

bool hj_tiled_setup(hj_grid *g, char *why, size_t why_len)
{
    auto fail = [&](const char *m) {
        snprintf(why, why_len, "%s", m);
        return false;
    };
    if (g->prec != HJ_FP32) return fail("tiled kernel is FP32 only");
    if (g->periodic != 0x8u) return fail("tiled kernel needs theta (axis 4) periodic and x, y, v not");
    if (!g->has_dyn || g->dyn != HJ_DYN_CAR4D) return fail("tiled kernel needs the car dynamics");
    if (g->p4 > 256) return fail("theta rows longer than 256 points");
    EncodeTiledFn enc = get_encode_fn();
    if (!enc) return fail("cuTensorMapEncodeTiled unavailable");

    int sms = 0, maxsmem = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    cudaDeviceGetAttribute(&maxsmem, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device);

    // tile shape: by default 8 x 4 rows of (y, v) (32 rows, MAXR per thread)
    // and a four-stage ring; at most 224 consumer threads (+ the producer warp)
    const int q4 = g->p4 / 4;
    const int max_rows = (224 / q4) * MAXR;
    if (max_rows < 1) return fail("theta rows too long for one CTA");
    int ty = g->tile_ty > 0 ? g->tile_ty : 8;
    int tv = g->tile_tv > 0 ? g->tile_tv : 4;
    if (tv > g->n[2]) tv = g->n[2];
    if (ty > g->n[1]) ty = g->n[1];
    while (ty * tv > max_rows && ty > 1) --ty;
    while (ty * tv > max_rows && tv > 1) --tv;
    int stages = g->tile_stages > 0 ? g->tile_stages : 4;
    if (stages < 3 || stages > MAX_STAGES) return fail("stage count out of range");
    TiledParams P = make_params(g, ty, tv, stages, 1);
    if (P.nconsumer + 32 > 256) return fail("tile needs more than 256 threads");
    size_t smem = tiled_smem_bytes(P, g->n[2]);
    if ((int)smem > maxsmem) return fail("tile does not fit in shared memory");
    if (cudaFuncSetAttribute(hj_step_tiled_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return fail("cannot raise the shared-memory limit");
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hj_step_tiled_kernel, P.nconsumer + 32, smem) !=
            cudaSuccess ||
        per_sm < 1)
        return fail("tile shape does not fit on an SM");
    int slots = sms * per_sm;
    P = make_params(g, ty, tv, stages, slots);
    if (g->tile_xc > 0) {
        P.xc = g->tile_xc;
        P.nchunk = (g->n[0] + P.xc - 1) / P.xc;
        P.nitems = P.ncol * P.nchunk;
    }

    // tensor maps over V0 and the two ping-pong buffers: dims (p4, n3, n2, n1)
    cuuint64_t dims[4] = {(cuuint64_t)g->p4, (cuuint64_t)g->n[2], (cuuint64_t)g->n[1], (cuuint64_t)g->n[0]};
    cuuint64_t strides[3] = {(cuuint64_t)g->p4 * 4, (cuuint64_t)g->p4 * g->n[2] * 4,
                             (cuuint64_t)g->p4 * g->n[2] * g->n[1] * 4};
    cuuint32_t box[4] = {(cuuint32_t)g->p4, (cuuint32_t)(tv + 2), (cuuint32_t)(ty + 2), 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    void *bases[3] = {g->v0, g->buf, (char *)g->buf + (size_t)g->nint * 4};
    for (int i = 0; i < 3; ++i) {
        CUresult r = enc(&g->tmap[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, bases[i], dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            snprintf(why, why_len, "cuTensorMapEncodeTiled failed (%d)", (int)r);
            return false;
        }
    }
    g->tile_ty = ty;
    g->tile_tv = tv;
    g->tile_xc = P.xc;
    g->tile_rg = P.rg;
    g->tile_stages = stages;
    g->tiled_ctas = P.nitems < slots ? P.nitems : slots;
    return true;
}

cudaError_t hj_launch_step_tiled(hj_grid *g)
{
    TiledParams P = params_of(g);
    size_t smem = tiled_smem_bytes(P, g->n[2]);
    hj_step_tiled_kernel<<<g->tiled_ctas, P.nconsumer + 32, smem, g->stream>>>(
        g->tmap[0], g->tmap[1], g->tmap[2], (const float *)g->v0, (float *)g->buf, (const HjCoef<float> *)g->coef,
        g->tab_tiled, g->dstate, g->geom, P, g->nint);
    return cudaGetLastError();
}
