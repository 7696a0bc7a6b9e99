// Tiled FP32 / Q5.27 HJ step kernel for sm_103a (the HBM-bound fast path).
//
// Same per-cell arithmetic as the generic kernel (one step of Algorithm 2 of
// arxiv 2012.04011 in upwind form, see hj_step_generic.cu), organised for
// bandwidth:
//   * A CTA owns a column of the grid: TY rows of y x TV rows of v x the full
//     theta row (so the periodic wrap stays inside the tile), and streams it
//     along x (the slowest axis), plane by plane.  Long columns may be split
//     into x chunks (work items) to balance the SMs.
//   * A producer warp loads, per plane, the tile plus its one-cell y/v halo
//     of V_n and the halo-free tile of V0 as two 4D TMA boxes
//     (cp.async.bulk.tensor.4d) into one stage of a shared-memory ring
//     guarded by mbarriers (full: bytes landed, empty: consumers done).
//     Out-of-range halo rows come back zero-filled and are replaced by
//     extrapolated ghosts.
//   * Each consumer thread owns one (y, v) row of the tile and one theta quad
//     (float4) for the whole kernel.  It holds planes x-1, x, x+1 in the ring
//     (x-1 and x+1 give the x neighbours), reads y/v/theta neighbours and V0
//     from the stage of plane x, and writes V_{n+1} with one float4 store.
//     Every V and V0 value is read from HBM once per step; halos are served
//     by shared memory and L2.
//   * All CTAs of a step sweep x concurrently, so y/v halo rows of
//     neighbouring columns are in L2 when they are needed.
//   * alpha^max partials (|xdot_1|, |xdot_2| over the (v, theta) states of the
//     cells each thread updates) are reduced by warp shuffles and a block
//     reduction, and the last CTA computes the next CFL step (fused; no extra
//     pass over the grid).
// The Q5.27 variant (FIXED) moves the same 4-byte values through the same
// ring and evaluates the fixed-point update of hj_q527_update per lane:
// exact integer upwind differences (ghosts by flag, as minus the difference
// on the other side), per-(v, theta) weights from the fixed-point table, and
// the FP64 coefficient table for alpha^max.
// Broadcast V0 (BCAST): when V0 depends on (x, y) only (Eq. init_V), the
// grid keeps its N1 x N2 field and the kernel reads V0 from it (one scalar
// per row and plane, an L1/L2 hit) instead of a V0 box per plane: 8
// algorithmic bytes per cell-update instead of 12.
// Every mbarrier wait is bounded by %globaltimer; on timeout the kernel
// records HJ_ERR_TIMEOUT in the device state, stops issuing work, waits
// (bounded) for its own copies in flight and returns.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "hj_scaled.cuh"
#include "hj_tma.cuh"

namespace {

constexpr int MAX_STAGES = 8;
constexpr int MAX_CONSUMERS = 768;  // consumer threads per CTA (+ one producer warp)
// Launch-bound variants: up to 384, 512, 640 or 768 consumer threads (152,
// 120, 96 or 80 registers a thread); a shape uses the smallest that holds it.
constexpr int VARIANTS[4] = {384, 512, 640, 768};

struct TiledParams {
    int ty, tv;          // tile rows along y and v
    int xc;              // planes per work item
    int q4;              // float4 per theta row (p4 / 4)
    int nconsumer;       // consumer threads (multiple of 32)
    int stages;          // shared-memory ring depth
    int ncol_v, ncol;    // tiles along v; columns in total
    int nchunk, nitems;  // x chunks per column; work items = ncol * nchunk
    int halo_box;        // floats in the V box with halo: p4 * (tv + 2) * (ty + 2)
    int halo_floats;     // its room in a stage: halo_box rounded up to 32 floats (V0 box 128-byte aligned)
    int v0_floats;       // V0 box: p4 * tv * ty (0 with the broadcast V0)
    int stage_bytes;     // (halo_floats + v0_floats) * 4 rounded up to 128
    float k3, k4, mk34;  // |xdot_3|/dx_3, |xdot_4|/dx_4, -(k3 + k4): constant-bank operands
};

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

__device__ __forceinline__ int32_t f4geti(const float4 &v, int e) { return __float_as_int(f4get(v, e)); }

// FIXED: Q5.27 values (the ring and the buffers hold int32 codes).
// PADDED: N4 is not a multiple of 4 (the last quad of a row has pad lanes).
// USIGN: cos(theta) and sin(theta) have one sign (up to negligible values)
// across every theta quad, so each thread picks its x and y upwind sides once.
// BCAST: V0 comes from the N1 x N2 field v0xy.
template <bool FIXED, bool PADDED, bool USIGN, bool BCAST, int MAXC>
__global__ void __launch_bounds__(MAXC + 32, 1) hj_step_tiled_kernel(
    const __grid_constant__ CUtensorMap map_v0, const __grid_constant__ CUtensorMap map_a,
    const __grid_constant__ CUtensorMap map_b, const __grid_constant__ CUtensorMap map_v0_tile,
    float *__restrict__ buf, const void *__restrict__ coefv, const float *__restrict__ tab,
    int32_t *__restrict__ qw, const float *__restrict__ v0xy, const void *__restrict__ k4tab, HjDevState *st,
    const HjGeom g, const TiledParams P, long long nint)
{
    const HjCoef<float> *coef = (const HjCoef<float> *)coefv;     // FP32 grids
    const HjCoef<double> *coefd = (const HjCoef<double> *)coefv;  // Q5.27 grids
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    if (st->done) return;  // uniform across the grid

    // ---- shared memory carve-up
    float *stages = (float *)smem_raw;
    uint64_t *full = (uint64_t *)(smem_raw + (size_t)P.stages * P.stage_bytes);
    uint64_t *empty = full + MAX_STAGES;
    unsigned long long *scratch = (unsigned long long *)(empty + MAX_STAGES);
    volatile int *abort_flag = (volatile int *)(scratch + 96);
    unsigned long long *deadline_p = (unsigned long long *)(scratch + 97);

    const long long n = st->n;
    const float dt = (float)st->dt;
    float *vout = buf + (n & 1) * nint;
    const CUtensorMap *map_in = (n == 0) ? &map_v0 : (((n - 1) & 1) ? &map_b : &map_a);

    const int tid = threadIdx.x;
    const int nconsumer_warps = P.nconsumer >> 5;
    if (tid == 0) {
        for (int s = 0; s < P.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], nconsumer_warps);
        }
        *abort_flag = 0;
        *deadline_p = global_ns() + HJ_WAIT_NS;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    float am1 = 0.f, am2 = 0.f;  // this thread's max |xdot_1|, |xdot_2| (non-negative)
    unsigned long long ab1 = 0ull, ab2 = 0ull;  // the same as FP64 bit patterns (FIXED)
    // convergence mode (Algorithm 2's epsilon): this thread's largest |V_{n+1} - V_n|
    const bool track = st->track;
    float dmf = 0.f;
    unsigned int dmq = 0u;  // in codes (FIXED; a change of one step is below 2^32 codes)

    if (tid >= P.nconsumer) {
        // ------------------------------------------------------------ producer
        if (tid == P.nconsumer) {
            const unsigned long long deadline = *deadline_p;
            // ring cursor: slot of the next load and the parity of its use
            int slot = 0;
            uint32_t phase = 0;
            uint32_t issued = 0;      // loads issued so far
            uint32_t used_mask = 0;   // slots that received a load
            uint32_t last_phase = 0;  // bit s: parity of the last load into slot s
            // bytes each box delivers (the exact box sizes, not the padded room)
            const uint32_t tx_halo = (uint32_t)(P.halo_box * 4), tx_v0 = (uint32_t)(P.v0_floats * 4);
            bool ok = true;
            for (int item = blockIdx.x; item < P.nitems && ok; item += gridDim.x) {
                ItemGeom it = item_geom(P, g, item);
                for (int p = it.pl0; p <= it.pl1; ++p) {
                    // the slot's previous contents must have been released
                    if (issued >= (uint32_t)P.stages && !mbar_wait(&empty[slot], phase ^ 1u, deadline)) {
                        ok = false;
                        break;
                    }
                    if (*abort_flag) {
                        ok = false;
                        break;
                    }
                    // V0 is needed on updated planes only (and never as a box with the broadcast V0)
                    const bool interior = !BCAST && p >= it.x0 && p < it.x1;
                    float *dst = stages + (size_t)slot * (P.stage_bytes / 4);
                    mbar_arrive_expect_tx(&full[slot], tx_halo + (interior ? tx_v0 : 0u));
                    tma_load_4d(dst, map_in, &full[slot], 0, it.v0 - 1, it.y0 - 1, p);
                    if (interior) tma_load_4d(dst + P.halo_floats, &map_v0_tile, &full[slot], 0, it.v0, it.y0, p);
                    used_mask |= 1u << slot;
                    last_phase = (last_phase & ~(1u << slot)) | (phase << slot);
                    ++issued;
                    if (++slot == P.stages) {
                        slot = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                st->status = HJ_ERR_TIMEOUT;
                *abort_flag = 1;
            }
            // drain: every copy this CTA issued must land before the CTA exits
            const unsigned long long drain_deadline = global_ns() + HJ_WAIT_NS;
            for (int s = 0; s < P.stages; ++s)
                if (((used_mask >> s) & 1u) && !mbar_wait(&full[s], (last_phase >> s) & 1u, drain_deadline))
                    st->status = HJ_ERR_TIMEOUT;
        }
    } else {
        // ------------------------------------------------------------ consumers
        // Thread t owns theta quad q = t % q4 of tile row r = t / q4 (row r is
        // (y0 + r / tv, v0 + r % tv)) for the whole kernel.
        const int lane = tid & 31;
        const int q = tid % P.q4;
        const int r = tid / P.q4;
        const int N1 = g.n1, N2 = g.n2, N3 = g.n3, N4 = g.n4, P4 = g.p4;
        const int srow = P.tv + 2;  // smem rows per y row
        const int jy = r / P.tv, kv = r - (r / P.tv) * P.tv;
        const bool inrow = r < P.ty * P.tv;
        const int rsm = inrow ? ((jy + 1) * srow + (kv + 1)) * P4 + 4 * q : (srow + 1) * P4;
        const int r0sm = P.halo_floats + (inrow ? (jy * P.tv + kv) * P4 + 4 * q : 0);  // V0 in the stage
        const uint32_t s1 = (uint32_t)N2 * N3 * P4;  // plane stride (the grid has < 2^31 values)

        // x and y upwind weights of this quad: xdot_1/dx_1 = v cos(th)/dx_1
        // takes V(x+1) where cos >= 0 and V(x-1) where cos < 0; likewise y.
        float wx[4], wy[4], cs[4], wxm[4], wym[4];
        bool xplus = true, yplus = true;
#pragma unroll
        for (int e = 0; e < 4 && !FIXED; ++e) {
            const float c = tab[N3 + 4 * q + e], s = tab[N3 + P4 + 4 * q + e];
            cs[e] = fabsf(c) + fabsf(s);
            if (USIGN) {
                wx[e] = fabsf(c);
                wy[e] = fabsf(s);
                wxm[e] = wym[e] = 0.f;
            } else {
                wx[e] = fmaxf(c, 0.f);
                wxm[e] = fmaxf(-c, 0.f);
                wy[e] = fmaxf(s, 0.f);
                wym[e] = fmaxf(-s, 0.f);
            }
        }
        if (USIGN && !FIXED) {  // the side of the quad's dominant lane (the host checked the others agree or vanish)
            // scalar loads: the sign table starts at float N3 + 2 P4, not 16-byte aligned in general
            xplus = tab[N3 + 2 * P4 + 4 * q] >= 0.f;
            yplus = tab[N3 + 2 * P4 + 4 * q + 1] >= 0.f;
        }
        const int lm = (4 * q - 1 + N4) % N4;  // theta index left of the quad
        const int lp = (4 * q + 4) % N4;       // right of the quad
        const int lreal = min(4, N4 - 4 * q);  // real lanes (< 4 only in a padded last quad)
        const int qtot = N3 * P4;
        int32_t qw3 = 0;  // fixed-point v weight
        if (FIXED) qw3 = qw[2 * qtot];

        // Ring cursors.  Planes are waited for and released in load order, so
        // one cursor walks the slots to wait on (with the phase parity) and
        // one walks the slots to release.
        int wslot = 0, rslot = 0;
        uint32_t wphase = 0;
        const int nst = P.stages;
        const int sfl = P.stage_bytes / 4;
        bool ok = true;
#define HJ_WAIT_NEXT(slot_out)                                   \
    do {                                                         \
        if (!mbar_wait_warp(&full[wslot], wphase, deadline_p)) { \
            slot_out = -1;                                       \
        } else {                                                 \
            slot_out = wslot;                                    \
            if (++wslot == nst) {                                \
                wslot = 0;                                       \
                wphase ^= 1u;                                    \
            }                                                    \
        }                                                        \
    } while (0)
#define HJ_RELEASE_OLDEST()                            \
    do {                                               \
        __syncwarp();                                  \
        if (lane == 0) mbar_arrive(&empty[rslot]);     \
        if (++rslot == nst) rslot = 0;                 \
    } while (0)
        for (int item = blockIdx.x; item < P.nitems && ok; item += gridDim.x) {
            const ItemGeom it = item_geom(P, g, item);
            const bool edge = it.y0 == 0 || it.y0 + P.ty >= N2 || it.v0 == 0 || it.v0 + P.tv >= N3;
            const int y = it.y0 + jy, v = it.v0 + kv;
            const bool rok = inrow && y < N2 && v < N3;
            const uint32_t rbase = rok ? ((uint32_t)y * N3 + v) * P4 + 4 * q : 0u;
            const float vk = (rok && !FIXED) ? tab[v] : 0.f;
            // theta coefficient of this row's speed (the steering car's heading
            // rate bound grows with v): (k4, -(k3 + k4)), or the fixed-point weight
            float2 k4m = make_float2(0.f, 0.f);
            int32_t qw4 = 0;
            if (rok) {
                if (FIXED) qw4 = qw[2 * qtot + HJ_QW_TAIL + v];
                else k4m = ((const float2 *)k4tab)[v];
            }
            int4 qw1 = make_int4(0, 0, 0, 0), qw2 = make_int4(0, 0, 0, 0);  // signed x / y weights of the quad
            if (FIXED && rok) {
                qw1 = *(const int4 *)(qw + v * P4 + 4 * q);
                qw2 = *(const int4 *)(qw + qtot + v * P4 + 4 * q);
            }
            // per lane: weight magnitudes, upwind sides and -(sum of the four weights)
            int32_t aw1[4], aw2[4], nsum[4];
            bool xpos[4], ypos[4];
            if (FIXED) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int32_t w1 = e == 0 ? qw1.x : e == 1 ? qw1.y : e == 2 ? qw1.z : qw1.w;
                    const int32_t w2 = e == 0 ? qw2.x : e == 1 ? qw2.y : e == 2 ? qw2.z : qw2.w;
                    xpos[e] = w1 >= 0;
                    ypos[e] = w2 >= 0;
                    aw1[e] = abs(w1);
                    aw2[e] = abs(w2);
                    nsum[e] = -(aw1[e] + aw2[e] + qw3 + qw4);
                }
            }
            float v0next = 0.f;  // broadcast V0 of the next plane (loaded one plane ahead)
            if (BCAST && rok) v0next = __ldg(v0xy + (size_t)it.x0 * N2 + y);
            // ghosts this row needs: 1 y-1, 2 y+1, 4 v-1, 8 v+1
            const uint32_t gmask = (y == 0 ? 1u : 0u) | (y == N2 - 1 ? 2u : 0u) | (v == 0 ? 4u : 0u) |
                                   (v == N3 - 1 ? 8u : 0u);

            // Planes held while plane x is updated: x-1 (if loaded), x and
            // x+1; plane x-1 is released after the update.
            int s_first, s_x;
            HJ_WAIT_NEXT(s_first);
            s_x = s_first;
            if (s_first >= 0 && it.x0 > it.pl0) HJ_WAIT_NEXT(s_x);
            if (s_first < 0 || s_x < 0) {
                ok = false;
                break;
            }
            float4 cur = *(const float4 *)(stages + (size_t)s_x * sfl + rsm);
            int s_prev = it.x0 > it.pl0 ? s_first : -1;  // slot of plane x-1, -1 at x = 0

            for (int x = it.x0; x < it.x1; ++x) {
                if (__any_sync(0xffffffffu, *abort_flag != 0)) {
                    ok = false;
                    break;
                }
                const float *sx = stages + (size_t)s_x * sfl;
                float v0s = 0.f;
                if (BCAST) {
                    v0s = v0next;
                    if (rok && x + 1 < it.x1) v0next = __ldg(v0xy + (size_t)(x + 1) * N2 + y);
                }
                // centre of plane x+1, or the extrapolated ghost past the end
                int s_n = -1;
                float4 prev, nxt;
                if (x + 1 <= N1 - 1) {
                    HJ_WAIT_NEXT(s_n);
                    if (s_n < 0) {
                        ok = false;
                        break;
                    }
                    nxt = *(const float4 *)(stages + (size_t)s_n * sfl + rsm);
                    prev = s_prev >= 0 ? *(const float4 *)(stages + (size_t)s_prev * sfl + rsm)
                                       : (FIXED ? cur : f4ghost(cur, nxt));
                } else {
                    prev = s_prev >= 0 ? *(const float4 *)(stages + (size_t)s_prev * sfl + rsm) : cur;
                    nxt = FIXED ? cur : f4ghost(cur, prev);
                }
                if (rok) {
                    const float *row = sx + rsm;
                    float4 ym = *(const float4 *)(row - srow * P4);
                    float4 yp = *(const float4 *)(row + srow * P4);
                    float4 vm = *(const float4 *)(row - P4);
                    float4 vp = *(const float4 *)(row + P4);
                    if (!FIXED && edge && gmask) {
                        // extrapolated points past the y / v ends (Sec. II-B)
                        if (gmask & 1u) ym = f4ghost(cur, yp);
                        if (gmask & 2u) yp = f4ghost(cur, ym);
                        if (gmask & 4u) vm = f4ghost(cur, vp);
                        if (gmask & 8u) vp = f4ghost(cur, vm);
                    }
                    const float *row0 = row - 4 * q;
                    const float tl = row0[lm], tr = row0[lp];
                    float t0 = 0.f;
                    if (PADDED) t0 = row0[0];
                    const float4 v0c = BCAST ? make_float4(v0s, v0s, v0s, v0s) : *(const float4 *)(sx + r0sm);
                    float4 xu = nxt, yu = yp;  // upwind x / y neighbours (USIGN)
                    if (USIGN) {
                        if (!xplus) xu = prev;
                        if (!yplus) yu = ym;
                    }
                    float4 out;
                    if constexpr (FIXED) {
                        // ghost flags: x-1 (x = 0), x+1 (x = N1-1), y-1, y+1, v-1, v+1
                        const bool gxm = s_prev < 0, gxp = x == N1 - 1;
                        const bool gym = gmask & 1u, gyp = gmask & 2u, gvm = gmask & 4u, gvp = gmask & 8u;
                        if (!(gxm || gxp || gmask)) {  // interior row: int32 operands throughout
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int32_t vc = f4geti(cur, e);
                                const int32_t tm = e == 0 ? __float_as_int(tl) : f4geti(cur, e - 1);
                                int32_t tp = e == 3 ? __float_as_int(tr) : f4geti(cur, e + 1);
                                if (PADDED && lreal < 4 && e == lreal - 1) tp = __float_as_int(t0);
                                const int32_t u1 = xpos[e] ? f4geti(nxt, e) : f4geti(prev, e);
                                const int32_t u2 = ypos[e] ? f4geti(yp, e) : f4geti(ym, e);
                                const int32_t u3 = max(f4geti(vp, e), f4geti(vm, e));
                                int32_t vn = hj_q527_update_interior(vc, f4geti(v0c, e), u1, u2, u3, max(tp, tm),
                                                                     aw1[e], aw2[e], qw3, qw4, nsum[e]);
                                if (PADDED && e >= lreal) vn = 0;
                                f4set(out, e, __int_as_float(vn));
                            }
                        } else {
                            // an extrapolated ghost on some axis (Sec. II-B): the ghost
                            // 2 V_c - V_o enters as -W on V_o and +2W on V_c, so the
                            // operands stay int32 and the sum stays exact
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int32_t vc = f4geti(cur, e);
                                const int32_t xm = f4geti(prev, e), xp = f4geti(nxt, e);
                                const int32_t ym_ = f4geti(ym, e), yp_ = f4geti(yp, e);
                                const int32_t vm_ = f4geti(vm, e), vp_ = f4geti(vp, e);
                                const int32_t tm = e == 0 ? __float_as_int(tl) : f4geti(cur, e - 1);
                                int32_t tp = e == 3 ? __float_as_int(tr) : f4geti(cur, e + 1);
                                if (PADDED && lreal < 4 && e == lreal - 1) tp = __float_as_int(t0);
                                // x, y: the upwind side, and whether it is a ghost
                                const bool hx = xpos[e] ? gxp : gxm, hy = ypos[e] ? gyp : gym;
                                const int32_t ux = (xpos[e] != hx) ? xp : xm, uy = (ypos[e] != hy) ? yp_ : ym_;
                                // v: the larger of V(v+1), V(v-1), either possibly a ghost
                                bool hv = false;
                                int32_t uv = max(vp_, vm_);
                                if (gvp) {
                                    uv = vm_;
                                    hv = vc >= vm_;
                                } else if (gvm) {
                                    uv = vp_;
                                    hv = vp_ < vc;
                                }
                                const int32_t c0 = nsum[e] + (hx ? 2 * aw1[e] : 0) + (hy ? 2 * aw2[e] : 0) +
                                                   (hv ? 2 * qw3 : 0);
                                int32_t vn = hj_q527_update_interior(vc, f4geti(v0c, e), ux, uy, uv, max(tp, tm),
                                                                     hx ? -aw1[e] : aw1[e], hy ? -aw2[e] : aw2[e],
                                                                     hv ? -qw3 : qw3, qw4, c0);
                                if (PADDED && e >= lreal) vn = 0;
                                f4set(out, e, __int_as_float(vn));
                            }
                        }
                    } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float vc = f4get(cur, e);
                        const float tm = e == 0 ? tl : f4get(cur, e - 1);
                        float tp = e == 3 ? tr : f4get(cur, e + 1);
                        if (PADDED && lreal < 4 && e == lreal - 1) tp = t0;  // wrap of a padded last quad
                        float in;
                        if (USIGN) {
                            in = wx[e] * f4get(xu, e);
                            in = fmaf(wy[e], f4get(yu, e), in);
                        } else {  // upwind differences folded into weights (no selects)
                            in = wx[e] * f4get(nxt, e);
                            in = fmaf(wxm[e], f4get(prev, e), in);
                            in = fmaf(wy[e], f4get(yp, e), in);
                            in = fmaf(wym[e], f4get(ym, e), in);
                        }
                        in = fmaf(-cs[e], vc, in);
                        // v and theta: the bang-bang control takes the larger neighbour
                        float acc = fmaf(P.k3, fmaxf(f4get(vp, e), f4get(vm, e)), k4m.y * vc);
                        acc = fmaf(k4m.x, fmaxf(tp, tm), acc);
                        acc = fmaf(vk, in, acc);
                        float vn = fminf(f4get(v0c, e), fmaf(dt, acc, vc));
                        if (PADDED && e >= lreal) vn = 0.f;
                        f4set(out, e, vn);
                    }
                    }
                    *(float4 *)(vout + (uint32_t)x * s1 + rbase) = out;
                    if (track) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            if constexpr (FIXED) {
                                const long long dd = (long long)f4geti(out, e) - f4geti(cur, e);
                                const unsigned long long ad = (unsigned long long)(dd < 0 ? -dd : dd);
                                dmq = max(dmq, (unsigned int)min(ad, 0xffffffffull));
                            } else {
                                dmf = fmaxf(dmf, fabsf(f4get(out, e) - f4get(cur, e)));
                            }
                        }
                    }
                }
                if (s_prev >= 0) HJ_RELEASE_OLDEST();  // plane x-1
                s_prev = s_x;
                s_x = s_n;
                cur = nxt;
            }
            if (!ok) break;
            // still held: plane x1-1 and, if loaded, the halo plane x1
            HJ_RELEASE_OLDEST();
            if (it.x1 <= it.pl1) HJ_RELEASE_OLDEST();
        }
#undef HJ_WAIT_NEXT
#undef HJ_RELEASE_OLDEST
        if (!ok) {
            st->status = HJ_ERR_TIMEOUT;
            *abort_flag = 1;
        }
        // alpha^max partials over the (v, theta) states of the cells this
        // thread updated (the car's xdot_1, xdot_2 depend only on v, theta)
        for (int item = blockIdx.x; item < P.nitems; item += gridDim.x) {
            const ItemGeom it = item_geom(P, g, item);
            const int y = it.y0 + jy, v = it.v0 + kv;
            if (inrow && y < N2 && v < N3)
                for (int e = 0; e < lreal; ++e) {
                    if constexpr (FIXED) {
                        const HjCoef<double> c = coefd[v * N4 + 4 * q + e];
                        const unsigned long long b1 = hj_abits(c.a1), b2 = hj_abits(c.a2);
                        ab1 = ab1 > b1 ? ab1 : b1;
                        ab2 = ab2 > b2 ? ab2 : b2;
                    } else {
                        const HjCoef<float> c = coef[v * N4 + 4 * q + e];
                        am1 = fmaxf(am1, c.a1);
                        am2 = fmaxf(am2, c.a2);
                    }
                }
        }
    }
    if constexpr (FIXED)
        hj_step_epilogue_scaled(st, g, ab1, ab2, hj_abits((double)dmq * (1.0 / HJ_Q527_SCALE)), scratch, nullptr, qw,
                                coefd, (const double *)k4tab);
    else
        hj_step_epilogue(st, g, hj_abits((double)am1), hj_abits((double)am2), hj_abits((double)dmf), scratch);
}

typedef void (*KernelFn)(const CUtensorMap, const CUtensorMap, const CUtensorMap, const CUtensorMap, float *,
                         const void *, const float *, int32_t *, const float *, const void *, HjDevState *,
                         const HjGeom, const TiledParams, long long);

template <bool FIXED, bool PADDED, bool USIGN, bool BCAST>
KernelFn kernel_fn_pu(int nconsumer)
{
    if (nconsumer <= VARIANTS[0]) return hj_step_tiled_kernel<FIXED, PADDED, USIGN, BCAST, VARIANTS[0]>;
    if (nconsumer <= VARIANTS[1]) return hj_step_tiled_kernel<FIXED, PADDED, USIGN, BCAST, VARIANTS[1]>;
    if (nconsumer <= VARIANTS[2]) return hj_step_tiled_kernel<FIXED, PADDED, USIGN, BCAST, VARIANTS[2]>;
    return hj_step_tiled_kernel<FIXED, PADDED, USIGN, BCAST, VARIANTS[3]>;
}

template <bool BCAST>
KernelFn kernel_fn_b(bool fixed, bool padded, bool usign, int nconsumer)
{
    // the fixed-point variant selects the upwind side per lane (no USIGN form)
    if (fixed)
        return padded ? kernel_fn_pu<true, true, false, BCAST>(nconsumer)
                      : kernel_fn_pu<true, false, false, BCAST>(nconsumer);
    if (padded)
        return usign ? kernel_fn_pu<false, true, true, BCAST>(nconsumer)
                     : kernel_fn_pu<false, true, false, BCAST>(nconsumer);
    return usign ? kernel_fn_pu<false, false, true, BCAST>(nconsumer)
                 : kernel_fn_pu<false, false, false, BCAST>(nconsumer);
}

KernelFn kernel_fn(bool fixed, bool padded, bool usign, bool bcast, int nconsumer)
{
    return bcast ? kernel_fn_b<true>(fixed, padded, usign, nconsumer)
                 : kernel_fn_b<false>(fixed, padded, usign, nconsumer);
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
    P.nconsumer = ((P.q4 * ty * tv + 31) / 32) * 32;
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
    const int nc = ((g->p4 / 4) * ty * tv + 31) / 32 * 32;
    return nc <= MAX_CONSUMERS ? nc + 32 : 0;
}

bool hj_tiled_setup(hj_grid *g, char *why, size_t why_len)
{
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
    if (g->nint >= (1LL << 31)) return fail("grid too large for 32-bit offsets");
    EncodeTiledFn enc = get_encode_fn();
    if (!enc) return fail("cuTensorMapEncodeTiled unavailable");

    int sms = 0, maxsmem = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    cudaDeviceGetAttribute(&maxsmem, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device);

    // quad signs: tab_tiled holds v_k [n3], cos/dx1 [p4], sin/dx2 [p4], then
    // the (cos, sin) sign of each quad's dominant lane [p4]
    float *sgn = (float *)calloc((size_t)g->p4, sizeof(float));
    if (!sgn) return fail("host allocation failed");
    const bool usign = !fixed && sign_uniform(g, sgn);
    cudaError_t e = cudaMemcpy(g->tab_tiled + g->n[2] + 2 * g->p4, sgn, sizeof(float) * g->p4, cudaMemcpyHostToDevice);
    free(sgn);
    if (e != cudaSuccess) return fail("sign table upload failed");

    // tile shape: by default 8 x 4 rows of (y, v) and as many stages as fit;
    // one consumer thread per (row, theta quad), at most MAX_CONSUMERS (+ the
    // producer warp)
    const int q4 = g->p4 / 4;
    const int max_rows = MAX_CONSUMERS / q4;
    if (max_rows < 1) return fail("theta rows too long for one CTA");
    int ty = g->tile_req[0] > 0 ? g->tile_req[0] : 8;
    int tv = g->tile_req[1] > 0 ? g->tile_req[1] : 4;
    if (tv > g->n[2]) tv = g->n[2];
    if (ty > g->n[1]) ty = g->n[1];
    while (ty * tv > max_rows && ty > 1) --ty;
    while (ty * tv > max_rows && tv > 1) --tv;
    int stages = g->tile_req[3];
    if (stages <= 0) {  // as many as fit in shared memory, up to MAX_STAGES
        TiledParams P1 = make_params(g, ty, tv, 1, 0);
        stages = (int)((maxsmem - 2048) / P1.stage_bytes);
        if (stages > MAX_STAGES) stages = MAX_STAGES;
    }
    if (stages < 4 || stages > MAX_STAGES) return fail("stage count out of range");
    TiledParams P = make_params(g, ty, tv, stages, 0);
    if (P.nconsumer > MAX_CONSUMERS) return fail("tile needs too many threads");
    size_t smem = tiled_smem_bytes(P);
    if ((int)smem > maxsmem) return fail("tile does not fit in shared memory");
    const void *fn = (const void *)kernel_fn(fixed, g->p4 != g->n[3], usign, g->v0_bcast, P.nconsumer);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
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
    KernelFn fn = kernel_fn(g->prec == HJ_Q527, g->p4 != g->n[3], g->tiled_usign, g->v0_bcast, P.nconsumer);
    fn<<<g->tiled_ctas, P.nconsumer + 32, tiled_smem_bytes(P), g->stream>>>(
        g->tmap[0], g->tmap[1], g->tmap[2], g->tmap[3], (float *)g->buf, g->coef, g->tab_tiled, g->qw,
        (const float *)g->v0xy, g->k4tab, g->dstate, g->geom, P, g->nint);
    return cudaGetLastError();
}
