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
//     (float4) for the whole kernel (two or four adjacent v rows in the
//     broadcast-V0 variant, see below).  It holds planes x-1, x, x+1 in the ring
//     (x-1 and x+1 give the x neighbours), reads y/v/theta neighbours and V0
//     from the stage of plane x, and writes V_{n+1} with one float4 store.
//     Every V and V0 value is read from HBM once per step; halos are served
//     by shared memory and L2.
//   * All CTAs of a step sweep x concurrently, so y/v halo rows of
//     neighbouring columns are in L2 when they are needed.
//   * alpha^max partials (|xdot_1|, |xdot_2| over the (v, theta) states of the
//     cells each thread updates: one FP64 pair per (v, theta quad) of each of
//     its items, from a small table) are reduced by each consumer thread at
//     the start, while the first planes are in flight, then by warp shuffles
//     and shared-memory maxima; the last CTA computes the next CFL step
//     (fused; no extra pass over the grid, no registers held in the sweep).
// The Q5.27 variant (FIXED) moves the same 4-byte values through the same
// ring and evaluates the fixed-point update of hj_q527_update per lane:
// exact integer upwind differences (ghosts by flag, as minus the difference
// on the other side), per-(v, theta) weights from the fixed-point table, and
// the FP64 coefficient table for alpha^max.
// Broadcast V0 (BCAST): when V0 depends on (x, y) only (Eq. init_V), the
// grid keeps its N1 x N2 field and the kernel reads V0 from it (one scalar
// per row and plane, an L1/L2 hit) instead of a V0 box per plane: 8
// algorithmic bytes per cell-update instead of 12.  That variant is issue-
// bound rather than HBM-bound, so in its single-sided form a thread may own
// RPT = 2 or 4 adjacent v rows of one theta quad: the ring waits, releases,
// cursors, stage addresses and the V0 load of a plane are shared by the
// rows, and the rows' v neighbours overlap (RPT + 2 row loads for the
// centres and v neighbours instead of 3 RPT).  With four rows a thread, a
// CTA can hold tiles large enough (8 x 8 rows and up) that the y/v halo
// rows, which each plane re-reads from L2, add about 1.5 instead of 1.8
// times the tile; that L2 traffic, not the arithmetic, sets the pace of this
// variant.  Each cell's arithmetic is the one-row form's, in the same order.
// Every mbarrier wait is bounded by %globaltimer; on timeout the kernel
// records HJ_ERR_TIMEOUT in the device state, stops issuing work, waits
// (bounded) for its own copies in flight and returns.
#pragma once

#include <math.h>
#include <stdio.h>
#include <string.h>

#include "hj_scaled.cuh"
#include "hj_tma.cuh"

// The kernel template lives in this header; hj_tiled_f32.cu,
// hj_tiled_f32_track.cu and hj_tiled_q527.cu each instantiate a disjoint
// part of it (so that the variants compile in parallel), and
// hj_step_tiled.cu holds the host side.
namespace hj_tiled {

constexpr int MAX_STAGES = 8;
// Launch-bound variants: a shape uses the smallest that holds its consumer
// threads.  Each of an SM's four 16K-register files holds a quarter of a
// CTA's warps (rounded up), which sets the registers a thread may use.
// FP32: up to 384, 512, 640 or 768 consumers (with the producer warp 13, 17,
// 21 or 25 warps: 128, 96, 80 or 72 registers); its 4D update compiled under
// the 80-register cap of the 640 class ran faster than under 96.  Q5.27: up
// to 352, 480, 608 or 736 (12, 16, 20 or 24 warps: 168, 128, 96 or 80
// registers), so that its 480-consumer shapes keep the registers of the
// integer update without spilling.
constexpr int VARIANTS_F32[4] = {384, 512, 640, 768};
constexpr int VARIANTS_Q527[4] = {352, 480, 608, 736};
template <bool FIXED>
constexpr int variant(int i)
{
    return FIXED ? VARIANTS_Q527[i] : VARIANTS_F32[i];
}
constexpr int max_consumers(bool fixed) { return fixed ? VARIANTS_Q527[3] : VARIANTS_F32[3]; }

struct TiledParams {
    int ty, tv;          // tile rows along y and v
    int xc;              // planes per work item
    int q4;              // float4 per theta row (p4 / 4)
    int rpt;             // v rows per consumer thread (1; 2 or 4 in the broadcast-V0 single-sided form)
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
// TRACK: convergence mode, the step also reduces max |V_{n+1} - V_n|.
// RPT: v rows per consumer thread (2 or 4 only with BCAST, USIGN, FP32, unpadded).
template <bool FIXED, bool PADDED, bool USIGN, bool BCAST, bool TRACK, int MAXC, int RPT = 1>
__global__ void __launch_bounds__(MAXC + 32, 1) hj_step_tiled_kernel(
    const __grid_constant__ CUtensorMap map_v0, const __grid_constant__ CUtensorMap map_a,
    const __grid_constant__ CUtensorMap map_b, const __grid_constant__ CUtensorMap map_v0_tile,
    float *__restrict__ buf, const void *__restrict__ coefv, const float *__restrict__ tab,
    int32_t *__restrict__ qw, const float *__restrict__ v0xy, const void *__restrict__ k4tab,
    const double2 *__restrict__ amaxq, HjDevState *st, const HjGeom g, const TiledParams P, long long nint)
{
    static_assert(RPT == 1 || ((RPT == 2 || RPT == 4) && BCAST && USIGN && !FIXED && !PADDED),
                  "several rows per thread: broadcast V0, single-sided FP32");
    const HjCoef<double> *coefd = (const HjCoef<double> *)coefv;  // Q5.27 grids: the table the weights come from
    extern __shared__ __align__(1024) unsigned char smem_raw[];

    // ---- shared memory carve-up
    float *stages = (float *)smem_raw;
    uint64_t *full = (uint64_t *)(smem_raw + (size_t)P.stages * P.stage_bytes);
    uint64_t *empty = full + MAX_STAGES;
    unsigned long long *scratch = (unsigned long long *)(empty + MAX_STAGES);
    volatile int *abort_flag = (volatile int *)(scratch + 96);
    unsigned long long *deadline_p = (unsigned long long *)(scratch + 97);
    unsigned long long *alpha_s = scratch + 98;  // the CTA's alpha^max partials (FP64 bit patterns)

    const int tid = threadIdx.x;
    const int nconsumer_warps = P.nconsumer >> 5;
    if (tid == 0) {
        for (int s = 0; s < P.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], nconsumer_warps);
        }
        *abort_flag = 0;
        *deadline_p = global_ns() + HJ_WAIT_NS;
        alpha_s[0] = 0ull;
        alpha_s[1] = 0ull;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    // Launched as a programmatic dependent of the previous step (the host sets
    // the launch attribute): everything above overlaps that step's end; from
    // here on the previous grid has completed and its V_n and finalised state
    // are visible.  Then the next step may be scheduled as SMs free up (its
    // CTAs wait here in turn).  Without such a prerequisite both are no-ops.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (st->done) return;  // uniform across the grid
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const long long n = st->n;
    const float dt = (float)st->dt;
    float *vout = buf + (n & 1) * nint;
    const CUtensorMap *map_in = (n == 0) ? &map_v0 : (((n - 1) & 1) ? &map_b : &map_a);

    // convergence mode (Algorithm 2's epsilon): this thread's largest |V_{n+1} - V_n|
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
        // (y0 + r / tv, v0 + r % tv)) for the whole kernel; with RPT > 1, of
        // the rows (y0 + r / (tv / RPT), v0 + RPT (r % (tv / RPT)) + k), k < RPT.
        const int lane = tid & 31;
        const int q = tid % P.q4;
        const int r = tid / P.q4;
        const int N1 = g.n1, N2 = g.n2, N3 = g.n3, N4 = g.n4, P4 = g.p4;
        const int srow = P.tv + 2;  // smem rows per y row
        const int tvr = RPT == 1 ? P.tv : P.tv / RPT;  // threads along v (the host makes tv a multiple of RPT)
        const int jy = r / tvr, kv = (r - jy * tvr) * RPT;
        const bool inrow = r < P.ty * tvr;
        {
            // alpha^max partials: the FP64 |xdot_1|, |xdot_2| maxima over this
            // thread's theta quad in the row it owns in each of its items (the
            // car's velocity depends on v and theta only), reduced while the
            // producer's first copies are in flight
            unsigned long long ab1 = 0ull, ab2 = 0ull;
#pragma unroll 4
            for (int item = blockIdx.x; item < P.nitems; item += gridDim.x) {
                const int col = item % P.ncol;
                const int y = (col / P.ncol_v) * P.ty + jy, v = (col % P.ncol_v) * P.tv + kv;
#pragma unroll
                for (int rr = 0; rr < RPT; ++rr)
                    if (inrow && y < g.n2 && v + rr < g.n3) {
                        const double2 am = amaxq[(v + rr) * P.q4 + q];
                        const unsigned long long b1 = hj_abits(am.x), b2 = hj_abits(am.y);
                        ab1 = ab1 > b1 ? ab1 : b1;
                        ab2 = ab2 > b2 ? ab2 : b2;
                    }
            }
            ab1 = hj_warp_max_u64(ab1);
            ab2 = hj_warp_max_u64(ab2);
            if (lane == 0) {
                atomicMax(&alpha_s[0], ab1);
                atomicMax(&alpha_s[1], ab2);
            }
        }
        const int rsm = inrow ? ((jy + 1) * srow + (kv + 1)) * P4 + 4 * q : (srow + 1) * P4;
        const int r0sm = P.halo_floats + (inrow ? (jy * P.tv + kv) * P4 + 4 * q : 0);  // V0 in the stage
        // V_{n+1} is addressed in float4 units (P4 is a multiple of 4): 32-bit
        // indices then reach 2^34 values, more than any grid the API accepts
        const uint32_t s1q = (uint32_t)N2 * N3 * (P4 / 4);  // plane stride in float4 units

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
        // Issue-bound variants (broadcast V0, fixed point) trim the per-plane
        // work: the abort flag is polled per item, and with USIGN only the
        // upwind y row is read (the other one only for an extrapolated ghost on
        // the upwind side).  The HBM-bound FP32 4D variant keeps the per-plane
        // poll and both y rows: measured faster there (0.190 vs 0.196-0.210 ms
        // per step on 128x128x64x96).
        constexpr bool LEAN = BCAST || FIXED;
        constexpr bool YONE = LEAN && USIGN && !FIXED;
        constexpr bool XLOAD = YONE;
        // (the sides are those of cos and sin: the host takes the USIGN form
        // only when every speed is >= 0; the general form flips the sides of
        // a negative-speed row, see below)
        const int yoff = yplus ? srow * P4 : -srow * P4;
        const uint32_t yghost = yplus ? 2u : 1u;
        bool wswapped = false;  // general form: the +/- weights are exchanged for a negative-speed row
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
        if (!mbar_wait_warp<BCAST || FIXED>(&full[wslot], wphase, deadline_p)) { \
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
            // a producer that gave up stops the consumers at the next item (a
            // plane that never arrives ends their bounded waits instead)
            if (LEAN && __any_sync(0xffffffffu, *abort_flag != 0)) {
                ok = false;
                break;
            }
            const ItemGeom it = item_geom(P, g, item);
            const bool edge = it.y0 == 0 || it.y0 + P.ty >= N2 || it.v0 == 0 || it.v0 + P.tv >= N3;
            const int y = it.y0 + jy, v = it.v0 + kv;
            const bool rok = inrow && y < N2 && v < N3;
            const uint32_t rbq = rok ? ((uint32_t)y * N3 + v) * (P4 / 4) + q : 0u;  // row quad, float4 units
            // xdot_1 = v cos(th), xdot_2 = v sin(th): in the general form a
            // negative speed flips the upwind sides and the weights take |v|
            float vk = (rok && !FIXED) ? tab[v] : 0.f;
            const bool vneg = !USIGN && vk < 0.f;
            if (vneg) vk = -vk;
            if (!USIGN && !FIXED && vneg != wswapped) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float tx = wx[e], ty = wy[e];
                    wx[e] = wxm[e];
                    wxm[e] = tx;
                    wy[e] = wym[e];
                    wym[e] = ty;
                }
                wswapped = vneg;
            }
            // theta coefficient of this row's speed (the steering car's heading
            // rate bound grows with v): (k4, -(k3 + k4)), or the fixed-point weight
            float2 k4m = make_float2(0.f, 0.f);
            int32_t qw4 = 0;
            if (rok) {
                if (FIXED) qw4 = qw[2 * qtot + HJ_QW_TAIL + v];
                else k4m = ((const float2 *)k4tab)[v];
            }
            // RPT > 1: rows v + k; in the grid, speed, theta coefficient
            bool rokv[RPT];
            float vkv[RPT];
            float2 k4v[RPT];
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                rokv[k] = rok && v + k < N3;
                vkv[k] = (RPT > 1 && rokv[k]) ? tab[v + k] : 0.f;
                k4v[k] = (RPT > 1 && rokv[k]) ? ((const float2 *)k4tab)[v + k] : make_float2(0.f, 0.f);
            }
            int4 qw1 = make_int4(0, 0, 0, 0), qw2 = make_int4(0, 0, 0, 0);  // signed x / y weights of the quad
            if (FIXED && rok) {
                qw1 = *(const int4 *)(qw + v * P4 + 4 * q);
                qw2 = *(const int4 *)(qw + qtot + v * P4 + 4 * q);
            }
            // per lane: weight magnitudes, upwind sides and -(sum of the four weights)
            int32_t aw1[4], aw2[4], nsum[4];
            bool xpos[4], ypos[4];
            bool wsmall = true;  // every lane's weights sum to at most 2^30 (hj_q527_update_interior32)
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
                    wsmall = wsmall && nsum[e] >= -(1 << 30);
                }
            }
            float v0next = 0.f;  // broadcast V0 of the next plane (loaded one plane ahead)
            if (BCAST && rok) v0next = __ldg(v0xy + (size_t)it.x0 * N2 + y);
            // ghosts this row needs: 1 y-1, 2 y+1, 4 v-1, 8 v+1
            const uint32_t gmask = (y == 0 ? 1u : 0u) | (y == N2 - 1 ? 2u : 0u) | (v == 0 ? 4u : 0u) |
                                   (v == N3 - 1 ? 8u : 0u);
            uint32_t gmv[RPT];  // and ghosts (RPT > 1)
#pragma unroll
            for (int k = 0; k < RPT; ++k) gmv[k] = (gmask & (k == 0 ? 7u : 3u)) | (v + k == N3 - 1 ? 8u : 0u);

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
            int s_prev = it.x0 > it.pl0 ? s_first : -1;  // slot of plane x-1, -1 at x = 0
            // XLOAD (the broadcast-V0 single-sided form): the centre and the one
            // upwind x neighbour are loaded from their stages every plane;
            // otherwise the centres of planes x-1 and x are carried in registers
            float4 cur = make_float4(0.f, 0.f, 0.f, 0.f), prevr = cur;
            if (!XLOAD) {
                cur = *(const float4 *)(stages + (size_t)s_x * sfl + rsm);
                prevr = s_prev >= 0 ? *(const float4 *)(stages + (size_t)s_first * sfl + rsm) : cur;
            }

            for (int x = it.x0; x < it.x1; ++x) {
                if (!LEAN && __any_sync(0xffffffffu, *abort_flag != 0)) {
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
                float4 prev = make_float4(0.f, 0.f, 0.f, 0.f), nxt = prev;
                if (x + 1 <= N1 - 1) {
                    HJ_WAIT_NEXT(s_n);
                    if (s_n < 0) {
                        ok = false;
                        break;
                    }
                    if (!XLOAD) {
                        nxt = *(const float4 *)(stages + (size_t)s_n * sfl + rsm);
                        prev = s_prev >= 0 ? prevr : (FIXED ? cur : f4ghost(cur, nxt));
                    }
                } else if (!XLOAD) {
                    prev = s_prev >= 0 ? prevr : cur;
                    nxt = FIXED ? cur : f4ghost(cur, prev);
                }
                if constexpr (RPT > 1) {
                    // RPT adjacent v rows of one theta quad, a rolling window
                    // along v: the centres of rows k - 1 and k + 1 are row k's
                    // v neighbours; per cell the arithmetic and its order are
                    // those of the one-row form below
                    if (rok) {
                        const float *row = sx + rsm;
                        // the upwind x plane, or past an end the one to
                        // extrapolate from (the other side, or the centre)
                        const int s_u = xplus ? s_n : s_prev, s_o = xplus ? s_prev : s_n;
                        const float *ru = stages + (size_t)(s_u >= 0 ? s_u : (s_o >= 0 ? s_o : s_x)) * sfl + rsm;
                        float4 cm = *(const float4 *)(row - P4), c = *(const float4 *)row;
                        float4 *dst = (float4 *)vout + ((uint32_t)x * s1q + rbq);
#pragma unroll
                        for (int k = 0; k < RPT; ++k) {
                            const float *rk = row + k * P4;
                            const float4 cp = *(const float4 *)(rk + P4);
                            float4 xl = *(const float4 *)(ru + k * P4);
                            if (s_u < 0) xl = f4ghost(c, xl);
                            float4 yu = *(const float4 *)(rk + yoff), vm = cm, vp = cp;
                            if (edge && (gmv[k] & (yghost | 12u))) {
                                // extrapolated points past the y / v ends (Sec. II-B)
                                if (gmv[k] & yghost) yu = f4ghost(c, *(const float4 *)(rk - yoff));
                                if (gmv[k] & 4u) vm = f4ghost(c, vp);
                                if (gmv[k] & 8u) vp = f4ghost(c, vm);
                            }
                            const float *rk0 = rk - 4 * q;
                            const float tl = rk0[lm], tr = rk0[lp];
                            float4 out;
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const float vc = f4get(c, e);
                                const float tm = e == 0 ? tl : f4get(c, e - 1), tp = e == 3 ? tr : f4get(c, e + 1);
                                float in = wx[e] * f4get(xl, e);
                                in = fmaf(wy[e], f4get(yu, e), in);
                                in = fmaf(-cs[e], vc, in);
                                float acc = fmaf(P.k3, fmaxf(f4get(vp, e), f4get(vm, e)), k4v[k].y * vc);
                                acc = fmaf(k4v[k].x, fmaxf(tp, tm), acc);
                                acc = fmaf(vkv[k], in, acc);
                                f4set(out, e, fminf(v0s, fmaf(dt, acc, vc)));
                            }
                            if (rokv[k]) {
                                dst[k * (P4 / 4)] = out;
                                if constexpr (TRACK) {
#pragma unroll
                                    for (int e = 0; e < 4; ++e) dmf = fmaxf(dmf, fabsf(f4get(out, e) - f4get(c, e)));
                                }
                            }
                            cm = c;
                            c = cp;
                        }
                    }
                } else {
                    float4 xl = make_float4(0.f, 0.f, 0.f, 0.f);  // XLOAD: the upwind x neighbour
                    if (XLOAD && rok) {
                        cur = *(const float4 *)(sx + rsm);
                        const int s_u = xplus ? s_n : s_prev;
                        if (s_u >= 0) {
                            xl = *(const float4 *)(stages + (size_t)s_u * sfl + rsm);
                        } else {  // past an end: the extrapolated point from the other side
                            const int s_o = xplus ? s_prev : s_n;
                            xl = f4ghost(cur, s_o >= 0 ? *(const float4 *)(stages + (size_t)s_o * sfl + rsm) : cur);
                        }
                    }
                    if (rok) {
                        const float *row = sx + rsm;
                        float4 ym = make_float4(0.f, 0.f, 0.f, 0.f), yp = ym, yu = ym;
                        if (YONE) {
                            yu = *(const float4 *)(row + yoff);
                        } else {
                            ym = *(const float4 *)(row - srow * P4);
                            yp = *(const float4 *)(row + srow * P4);
                        }
                        float4 vm = *(const float4 *)(row - P4);
                        float4 vp = *(const float4 *)(row + P4);
                        if (!FIXED && edge && gmask) {
                            // extrapolated points past the y / v ends (Sec. II-B)
                            if (YONE) {
                                if (gmask & yghost) yu = f4ghost(cur, *(const float4 *)(row - yoff));
                            } else {
                                if (gmask & 1u) ym = f4ghost(cur, yp);
                                if (gmask & 2u) yp = f4ghost(cur, ym);
                            }
                            if (gmask & 4u) vm = f4ghost(cur, vp);
                            if (gmask & 8u) vp = f4ghost(cur, vm);
                        }
                        const float *row0 = row - 4 * q;
                        const float tl = row0[lm], tr = row0[lp];
                        float t0 = 0.f;
                        if (PADDED) t0 = row0[0];
                        const float4 v0c = BCAST ? make_float4(v0s, v0s, v0s, v0s) : *(const float4 *)(sx + r0sm);
                        float4 xu = nxt;  // upwind x / y neighbours (USIGN)
                        if (XLOAD) xu = xl;
                        else if (USIGN && !xplus) xu = prev;
                        if (USIGN && !YONE) yu = yplus ? yp : ym;
                        float4 out;
                        if constexpr (FIXED) {
                            // ghost flags: x-1 (x = 0), x+1 (x = N1-1), y-1, y+1, v-1, v+1
                            const bool gxm = s_prev < 0, gxp = x == N1 - 1;
                            const bool gym = gmask & 1u, gyp = gmask & 2u, gvm = gmask & 4u, gvp = gmask & 8u;
                            if (!(gxm || gxp || gmask) && wsmall) {  // interior row: int32 operands throughout
    #pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    const int32_t vc = f4geti(cur, e);
                                    const int32_t tm = e == 0 ? __float_as_int(tl) : f4geti(cur, e - 1);
                                    int32_t tp = e == 3 ? __float_as_int(tr) : f4geti(cur, e + 1);
                                    if (PADDED && lreal < 4 && e == lreal - 1) tp = __float_as_int(t0);
                                    const int32_t u1 = xpos[e] ? f4geti(nxt, e) : f4geti(prev, e);
                                    const int32_t u2 = ypos[e] ? f4geti(yp, e) : f4geti(ym, e);
                                    const int32_t u3 = max(f4geti(vp, e), f4geti(vm, e));
                                    int32_t vn = hj_q527_update_interior32(vc, f4geti(v0c, e), u1, u2, u3, max(tp, tm),
                                                                           aw1[e], aw2[e], qw3, qw4, nsum[e]);
                                    if (PADDED && e >= lreal) vn = 0;
                                    f4set(out, e, __int_as_float(vn));
                                }
                            } else {
                                // an extrapolated ghost on some axis (Sec. II-B): the ghost
                                // 2 V_c - V_o enters as -W on V_o and +2W on V_c, so the
                                // operands stay int32 and the sum stays exact (this form
                                // also takes interior rows whose weights sum above 2^30)
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
                        ((float4 *)vout)[(uint32_t)x * s1q + rbq] = out;
                        if constexpr (TRACK) {
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
                }
                if (s_prev >= 0) HJ_RELEASE_OLDEST();  // plane x-1
                s_prev = s_x;
                s_x = s_n;
                if (!XLOAD) {
                    prevr = cur;
                    cur = nxt;
                }
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
    }
    // the CTA's alpha^max partials enter the block reduction through thread 0
    __syncthreads();
    const unsigned long long ab1 = tid == 0 ? alpha_s[0] : 0ull, ab2 = tid == 0 ? alpha_s[1] : 0ull;
    if constexpr (FIXED)
        hj_step_epilogue_scaled(st, g, ab1, ab2, hj_abits((double)dmq * (1.0 / HJ_Q527_SCALE)), scratch, nullptr, qw,
                                coefd, (const double *)k4tab);
    else
        hj_step_epilogue(st, g, ab1, ab2, hj_abits((double)dmf), scratch);
}

typedef void (*KernelFn)(const CUtensorMap, const CUtensorMap, const CUtensorMap, const CUtensorMap, float *,
                         const void *, const float *, int32_t *, const float *, const void *, const double2 *,
                         HjDevState *, const HjGeom, const TiledParams, long long);

// Kernel of a variant, smallest launch bound class that holds nconsumer
// consumer threads (defined in the instantiating translation units); rpt is
// the v rows per consumer thread (2 or 4 only for the broadcast-V0
// single-sided FP32 form, see TiledParams::rpt).
KernelFn select_f32(bool padded, bool usign, bool bcast, int nconsumer, int rpt);        // hj_tiled_f32.cu
KernelFn select_f32_track(bool padded, bool usign, bool bcast, int nconsumer, int rpt);  // hj_tiled_f32_track.cu
KernelFn select_q527(bool padded, bool bcast, bool track, int nconsumer);                // hj_tiled_q527.cu

template <bool FIXED, bool PADDED, bool USIGN, bool BCAST, bool TRACK, int RPT = 1>
KernelFn by_bound(int nconsumer)
{
    if (nconsumer <= variant<FIXED>(0)) return hj_step_tiled_kernel<FIXED, PADDED, USIGN, BCAST, TRACK, variant<FIXED>(0), RPT>;
    if (nconsumer <= variant<FIXED>(1)) return hj_step_tiled_kernel<FIXED, PADDED, USIGN, BCAST, TRACK, variant<FIXED>(1), RPT>;
    if (nconsumer <= variant<FIXED>(2)) return hj_step_tiled_kernel<FIXED, PADDED, USIGN, BCAST, TRACK, variant<FIXED>(2), RPT>;
    return hj_step_tiled_kernel<FIXED, PADDED, USIGN, BCAST, TRACK, variant<FIXED>(3), RPT>;
}

}  // namespace hj_tiled
