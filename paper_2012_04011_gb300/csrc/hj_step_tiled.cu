// Host side of the tiled step kernel (hj_tiled_kernel.cuh): tile shape,
// tensor maps, shared-memory layout, kernel selection and launch.
#include "hj_tiled_kernel.cuh"

using namespace hj_tiled;

namespace {

KernelFn kernel_fn(bool fixed, bool padded, bool usign, bool bcast, bool track, int nconsumer, int rpt)
{
    // the fixed-point variant selects the upwind side per lane (no USIGN form)
    if (fixed) return select_q527(padded, bcast, track, nconsumer);
    return track ? select_f32_track(padded, usign, bcast, nconsumer, rpt)
                 : select_f32(padded, usign, bcast, nconsumer, rpt);
}

// v rows per consumer thread in the broadcast-V0 single-sided FP32 form
// (bound by data movement: several rows a thread let a CTA hold larger tiles,
// whose halo rows cost less L2 traffic per row, and share the per-plane
// ring and address work): four when tv is a multiple of 4 and that still
// leaves at least 8 consumer warps, else two when tv is even; one otherwise
// and in every other variant.  g->tiled_usign must be current
// (hj_tiled_setup sets it before it sizes a tile).
int tiled_rpt(const hj_grid *g, int ty, int tv)
{
    if (!(g->prec == HJ_FP32 && g->v0_bcast && g->tiled_usign && g->p4 == g->n[3])) return 1;
    if (tv % 4 == 0 && (g->p4 / 4) * ty * (tv / 4) >= 256) return 4;
    return tv % 2 == 0 ? 2 : 1;
}

int consumers_of(const hj_grid *g, int ty, int tv)
{
    return ((g->p4 / 4) * ty * (tv / tiled_rpt(g, ty, tv)) + 31) / 32 * 32;
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

TiledParams make_params(const hj_grid *g, int ty, int tv, int stages, int xc)
{
    TiledParams P;
    memset(&P, 0, sizeof(P));
    P.ty = ty;
    P.tv = tv;
    P.stages = stages;
    P.q4 = g->p4 / 4;
    P.rpt = tiled_rpt(g, ty, tv);
    P.nconsumer = consumers_of(g, ty, tv);
    P.ncol_v = (g->n[2] + tv - 1) / tv;
    P.ncol = ((g->n[1] + ty - 1) / ty) * P.ncol_v;
    P.halo_box = g->p4 * (tv + 2) * (ty + 2);
    P.halo_floats = (P.halo_box + 31) / 32 * 32;
    P.v0_floats = g->v0_bcast ? 0 : g->p4 * tv * ty;
    P.stage_bytes = ((P.halo_floats + P.v0_floats) * 4 + 127) / 128 * 128;
    P.xc = xc < 1 ? g->n[0] : (xc > g->n[0] ? g->n[0] : xc);
    P.nchunk = (g->n[0] + P.xc - 1) / P.xc;
    P.nitems = P.ncol * P.nchunk;
    P.k3 = (float)g->geom.k3;
    P.k4 = (float)g->geom.k4;
    P.mk34 = (float)(-(g->geom.k3 + g->geom.k4));
    return P;
}

// Planes per work item: all CTAs sweep x concurrently, so the time of a step
// is about (rounds of items) x (planes one item loads, halo planes included).
// Pick the chunk length that minimises it.
int best_chunk(const hj_grid *g, int ncol, int slots)
{
    const int n1 = g->n[0];
    int best_xc = n1;
    double best = 1e300;
    for (int nchunk = 1; nchunk <= n1 / 4 || nchunk == 1; ++nchunk) {
        const int xc = (n1 + nchunk - 1) / nchunk;
        const int nch = (n1 + xc - 1) / xc;
        const long long items = (long long)ncol * nch;
        const long long rounds = (items + slots - 1) / slots;
        const double cost = (double)rounds * (xc + (nch > 1 ? 2 : 0));
        if (cost < best - 1e-9) {
            best = cost;
            best_xc = xc;
        }
    }
    return best_xc;
}

size_t tiled_smem_bytes(const TiledParams &P)
{
    return (size_t)P.stages * P.stage_bytes + 2 * MAX_STAGES * sizeof(uint64_t) + 96 * sizeof(unsigned long long) +
           32;
}

// Whether every theta quad has one sign of cos and of sin (lanes whose value
// is exactly 0 after hj_flush_trig carry no weight and count as either);
// also writes the quads' dominant signs into tab_sign[4 * q].
bool sign_uniform(const hj_grid *g, float *tab_sign)
{
    const int N4 = g->n[3];
    double cmax = 0, smax = 0;
    for (int l = 0; l < N4; ++l) {
        const double th = g->lo[3] + (double)l * g->h[3];
        cmax = fmax(cmax, fabs(hj_flush_trig(cos(th))));
        smax = fmax(smax, fabs(hj_flush_trig(sin(th))));
    }
    bool ok = true;
    for (int q = 0; q < g->p4 / 4; ++q) {
        double bc = 0, bs = 0;
        int sc = 1, ss = 1;
        for (int e = 0; e < 4 && 4 * q + e < N4; ++e) {
            const double th = g->lo[3] + (double)(4 * q + e) * g->h[3];
            const double c = hj_flush_trig(cos(th)), sn = hj_flush_trig(sin(th));
            if (fabs(c) > bc) bc = fabs(c), sc = c >= 0 ? 1 : -1;
            if (fabs(sn) > bs) bs = fabs(sn), ss = sn >= 0 ? 1 : -1;
        }
        for (int e = 0; e < 4 && 4 * q + e < N4; ++e) {
            const double th = g->lo[3] + (double)(4 * q + e) * g->h[3];
            // lanes whose weight is exactly 0 may sit on either side
            const double c = hj_flush_trig(cos(th)), s = hj_flush_trig(sin(th));
            if (c != 0.0 && (c >= 0 ? 1 : -1) != sc) ok = false;
            if (s != 0.0 && (s >= 0 ? 1 : -1) != ss) ok = false;
        }
        tab_sign[4 * q + 0] = (float)sc;
        tab_sign[4 * q + 1] = (float)ss;
        tab_sign[4 * q + 2] = 0.f;
        tab_sign[4 * q + 3] = 0.f;
    }
    return ok;
}

}  // namespace

int hj_tiled_threads(const hj_grid *g, int ty, int tv)
{
    const int nc = consumers_of(g, ty, tv);
    return nc <= max_consumers(g->prec == HJ_Q527) ? nc + 32 : 0;
}

int hj_tiled_variant(bool fixed, int i) { return fixed ? VARIANTS_Q527[i] : VARIANTS_F32[i]; }

bool hj_tiled_setup(hj_grid *g, char *why, size_t why_len)
{
    ++g->launch_version;  // tile, tensor maps or kernel variant may change: captured step graphs are stale
    auto fail = [&](const char *m) {
        snprintf(why, why_len, "%s", m);
        return false;
    };
    if (g->prec != HJ_FP32 && g->prec != HJ_Q527) return fail("tiled kernel is FP32 or Q5.27 only");
    const bool fixed = g->prec == HJ_Q527;
    if (g->periodic != 0x8u) return fail("tiled kernel needs theta (axis 4) periodic and x, y, v not");
    if (!g->has_dyn || (g->dyn != HJ_DYN_CAR4D && g->dyn != HJ_DYN_CAR4D_STEER))
        return fail("tiled kernel needs the car dynamics");
    if (g->p4 > 256) return fail("theta rows longer than 256 points");
    if (g->nint >= (1LL << 34)) return fail("grid of 2^34 stored values or more (32-bit float4 indices)");
    EncodeTiledFn enc = get_encode_fn();
    if (!enc) return fail("cuTensorMapEncodeTiled unavailable");

    int sms = 0, maxsmem = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    cudaDeviceGetAttribute(&maxsmem, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device);

    // quad signs: tab_tiled holds v_k [n3], cos/dx1 [p4], sin/dx2 [p4], then
    // the (cos, sin) sign of each quad's dominant lane [p4]
    float *sgn = (float *)calloc((size_t)g->p4, sizeof(float));
    if (!sgn) return fail("host allocation failed");
    // the single-sided (USIGN) form also needs every speed >= 0 (a negative
    // speed flips the upwind side); otherwise the general form runs
    const bool usign = !fixed && g->lo[2] >= 0.0 && sign_uniform(g, sgn);
    cudaError_t e = cudaMemcpy(g->tab_tiled + g->n[2] + 2 * g->p4, sgn, sizeof(float) * g->p4, cudaMemcpyHostToDevice);
    free(sgn);
    if (e != cudaSuccess) return fail("sign table upload failed");
    g->tiled_usign = usign;  // a property of the grid's v and theta ranges (read by tiled_rpt)

    // tile shape: one consumer thread per (row, theta quad) (per pair of v
    // rows in the two-row form), at most the largest launch-bound class (+
    // the producer warp).  By default the rows
    // of (y, v) with the fewest halo reads per row among the shapes whose block
    // fits the largest class that runs without spills (640 consumer threads;
    // 480 in fixed point), discounted by the share of the SMs the
    // shape can keep busy (a small grid needs small tiles to fill the GPU),
    // and as many stages as fit; hj_autotune measures the candidates instead.
    const int q4 = g->p4 / 4;
    if (max_consumers(fixed) / q4 < 1) return fail("theta rows too long for one CTA");
    int ty = g->tile_req[0], tv = g->tile_req[1];
    if (ty <= 0 || tv <= 0) {
        const int cap = fixed ? VARIANTS_Q527[1] : VARIANTS_F32[2];
        double best = 1e300;
        int bty = 1, btv = 1;
        for (int a = 1; a <= 16 && a <= g->n[1]; ++a)
            for (int b = 1; b <= 16 && b <= g->n[2]; ++b) {
                if ((ty > 0 && a != ty) || (tv > 0 && b != tv)) continue;
                const int cons = consumers_of(g, a, b);
                if (cons > cap && !(a == 1 && b == 1)) continue;
                // room for the smallest ring (4 stages)
                if (4 * (size_t)make_params(g, a, b, 1, 0).stage_bytes + 2048 > (size_t)maxsmem && !(a == 1 && b == 1))
                    continue;
                // work items this shape can offer (columns x chunks of >= 4 planes)
                const double items = (double)((g->n[1] + a - 1) / a) * ((g->n[2] + b - 1) / b) *
                                     (g->n[0] / 4 > 1 ? g->n[0] / 4 : 1);
                const double busy = items < sms ? items / (sms > 0 ? sms : 1) : 1.0;
                const double c = (double)(a + 2) * (b + 2) / (a * b) / busy - 1e-6 * a * b;  // ties: more rows
                if (c < best) {
                    best = c;
                    bty = a;
                    btv = b;
                }
            }
        ty = bty;
        tv = btv;
    }
    if (tv > g->n[2]) tv = g->n[2];
    if (ty > g->n[1]) ty = g->n[1];
    while (consumers_of(g, ty, tv) > max_consumers(fixed) && ty > 1) --ty;
    while (consumers_of(g, ty, tv) > max_consumers(fixed) && tv > 1) --tv;
    int stages = g->tile_req[3];
    if (stages <= 0) {  // as many as fit in shared memory, up to MAX_STAGES
        TiledParams P1 = make_params(g, ty, tv, 1, 0);
        stages = (int)((maxsmem - 2048) / P1.stage_bytes);
        if (stages > MAX_STAGES) stages = MAX_STAGES;
    }
    if (stages < 4 || stages > MAX_STAGES) return fail("stage count out of range");
    TiledParams P = make_params(g, ty, tv, stages, 0);
    if (P.nconsumer > max_consumers(fixed)) return fail("tile needs too many threads");
    size_t smem = tiled_smem_bytes(P);
    if ((int)smem > maxsmem) return fail("tile does not fit in shared memory");
    const void *fn = (const void *)kernel_fn(fixed, g->p4 != g->n[3], usign, g->v0_bcast, false, P.nconsumer, P.rpt);
    const void *fn_track =
        (const void *)kernel_fn(fixed, g->p4 != g->n[3], usign, g->v0_bcast, true, P.nconsumer, P.rpt);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(fn_track, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return fail("cannot raise the shared-memory limit");
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, P.nconsumer + 32, smem) != cudaSuccess ||
        per_sm < 1)
        return fail("tile shape does not fit on an SM");
    const int slots = sms * per_sm;
    const int xc = g->tile_req[2] > 0 ? g->tile_req[2] : best_chunk(g, P.ncol, slots);
    P = make_params(g, ty, tv, stages, xc);

    // tensor maps, dims (p4, n3, n2, n1): V0 / buffer A / buffer B with the
    // halo box, and V0 with the halo-free box
    cuuint64_t dims[4] = {(cuuint64_t)g->p4, (cuuint64_t)g->n[2], (cuuint64_t)g->n[1], (cuuint64_t)g->n[0]};
    cuuint64_t strides[3] = {(cuuint64_t)g->p4 * 4, (cuuint64_t)g->p4 * g->n[2] * 4,
                             (cuuint64_t)g->p4 * g->n[2] * g->n[1] * 4};
    cuuint32_t box_halo[4] = {(cuuint32_t)g->p4, (cuuint32_t)(tv + 2), (cuuint32_t)(ty + 2), 1};
    cuuint32_t box_tile[4] = {(cuuint32_t)g->p4, (cuuint32_t)tv, (cuuint32_t)ty, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    void *bases[4] = {g->v0, g->buf, (char *)g->buf + (size_t)g->nint * 4, g->v0};
    for (int i = 0; i < 4; ++i) {
        CUresult r = enc(&g->tmap[i], fixed ? CU_TENSOR_MAP_DATA_TYPE_INT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                         bases[i], dims, strides,
                         i < 3 ? box_halo : box_tile, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            snprintf(why, why_len, "cuTensorMapEncodeTiled failed (%d)", (int)r);
            return false;
        }
    }
    g->tile_ty = ty;
    g->tile_tv = tv;
    g->tile_xc = P.xc;
    g->tile_stages = stages;
    g->tiled_ctas = P.nitems < slots ? P.nitems : slots;
    g->tiled_per_sm = per_sm;
    g->tiled_usign = usign;
    return true;
}

cudaError_t hj_launch_step_tiled(hj_grid *g)
{
    const TiledParams P = make_params(g, g->tile_ty, g->tile_tv, g->tile_stages, g->tile_xc);
    KernelFn fn =
        kernel_fn(g->prec == HJ_Q527, g->p4 != g->n[3], g->tiled_usign, g->v0_bcast, g->track, P.nconsumer, P.rpt);
    // a programmatic dependent of the previous launch on the stream: the
    // kernel sets up its ring while the previous step drains and waits for
    // that step's completion before it reads anything it wrote
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)g->tiled_ctas);
    cfg.blockDim = dim3((unsigned)(P.nconsumer + 32));
    cfg.dynamicSmemBytes = tiled_smem_bytes(P);
    cfg.stream = g->stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, g->tmap[0], g->tmap[1], g->tmap[2], g->tmap[3], (float *)g->buf,
                              (const void *)g->coef, (const float *)g->tab_tiled, g->qw, (const float *)g->v0xy,
                              (const void *)g->k4tab, (const double2 *)g->amax_q, g->dstate, g->geom, P, g->nint);
}
