// Batched solves: many independent 4D car instances (each its own grid
// size, obstacle map V0, horizon and time loop) stepped by one persistent
// kernel that runs many batch steps per launch.  Same scheme and same
// per-cell arithmetic as the single-grid tiled kernel (one step of
// Algorithm 2 of arxiv 2012.04011 in upwind form, see hj_step_generic.cu and
// hj_step_tiled.cu).
//
// Work: every running slot's grid is cut into items (slot, y-tile, v-tile,
// x-chunk).  A CTA's producer warp takes the next item from a device-side
// queue (items are ordered slot by slot, so concurrently running CTAs share
// neighbouring columns and their halos hit L2) and streams the item's planes
// (V_n box with a one-cell y/v halo, V0 box without) through the
// shared-memory ring with TMA; the stage of an item's first plane carries the
// item's descriptor (geometry, the slot's coefficients, dt and output
// buffer), so consumers start an item from shared memory.  Consumers own one
// (row, theta quad) each, as in the single-grid kernel, and update lane pairs
// with paired FP32 multiply-adds; the tile shape of each slot is chosen so
// that its rows x quads fit the block.
//
// Time loop: each slot keeps its own FP64 state (t, dt, step count) on the
// device.  After an item, each consumer warp counts itself done; the warp
// that completes the slot's last item of a step reduces the slot's alpha^max
// over its per-speed table of |xdot_1|, |xdot_2| maxima and computes the
// slot's next CFL step (hj_finalise).  A launch runs many such steps as
// rounds of the queue (round r: the items of every slot with more than r
// steps to go), and a slot's items of its next step start as soon as its own
// step is finalised, so the slots do not wait for one another between steps
// and the GPU stays busy while the slots that finish early drop out.
//
// Slots can be added and removed between calls (the serving loop admits
// requests this way); the item list, the per-slot descriptors and the tensor
// maps live in device memory and are rewritten by stream-ordered copies.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "hj_tma.cuh"

namespace {

constexpr int B_MAX_STAGES = 8;
constexpr int B_VARIANTS[4] = {352, 480, 608, 736};
// Shapes of at most B_DUAL consumers run two CTAs per SM (10 warps each, two
// independent rings and producers per SM; each CTA gets half the SM's shared
// memory).
constexpr int B_DUAL = 288;
// Batch steps (rounds) per launch at most.
constexpr int B_MAX_ROUNDS = 1024;

struct BatchInst {
    int n1, n2, n3, n4, p4, q4;
    int ty, tv, xc;
    int nitems;  // items of this slot per step
    int halo_box, halo_floats, v0_floats;
    float k3, k4, mk34;
    long long nint;
    float *buf;                 // buffer A, then buffer B (nint floats each)
    const float *tab;           // v_k [n3], cos/dx1 [p4], sin/dx2 [p4]
    const HjCoef<float> *coef;  // [n3 * n4]
    const double2 *amaxv;       // [n3]: the largest FP64 |xdot_1|, |xdot_2| over the headings of each speed
    HjGeom geom;
};

struct BatchSlot {
    HjDevState st;
    unsigned int warps_done;  // consumer warps that finished an item of this slot in this step
    int pad_[3];
};

struct BatchItem {
    int slot, y0, v0, x0;
};

struct BatchCtl {
    unsigned int head;       // next item to hand out
    unsigned int ctas_done;  // CTAs of this launch that finished
    int nitems;
    int status;
};

struct BatchParams {
    int nconsumer;    // consumer threads per CTA (multiple of 32)
    int stages;       // ring depth
    int stage_bytes;  // ring stage room (the largest slot's V box + V0 box)
};

static __device__ __forceinline__ void tensormap_acquire(const CUtensorMap *m)
{
    // the maps live in global memory and are rewritten by the host between
    // launches when slots change
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((unsigned long long)m) : "memory");
}

// One slot's V0 conversion and first step, for the calls that set up many
// slots at once (one launch for all of them instead of one per slot).
struct SlotSetup {
    const void *src;  // caller's dense V0 (FP64 or FP32)
    float *dst;       // the slot's V0 in the internal layout
    HjDevState *st;   // the slot's time-loop state
    const HjCoef<float> *coef;
    long long nrows;  // N1 * N2 * N3
    int n4, p4, ncoef;
    double T, cfl;
    HjGeom geom;
};

// blockIdx.y = entry: dense -> padded rows (pad lanes zero), NaN / Inf flag
// into the entry's state (the state itself was reset before).
template <typename Tin>
__global__ void batch_ingest_many_kernel(const SlotSetup *__restrict__ list)
{
    const SlotSetup d = list[blockIdx.y];
    const Tin *src = (const Tin *)d.src;
    // a slot holds fewer than 2^31 values (hj_batch_add): 32-bit indices
    const uint32_t total = (uint32_t)(d.nrows * d.p4), p4 = (uint32_t)d.p4, n4 = (uint32_t)d.n4;
    int bad = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const uint32_t row = i / p4;
        const uint32_t l = i - row * p4;
        float v = 0.f;
        if (l < n4) {
            const double x = (double)src[(size_t)row * n4 + l];
            if (!isfinite(x)) bad = 1;
            v = (float)x;
        }
        d.dst[i] = v;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&d.st->nonfinite, 1);
}

// One block per entry: the solve prologue of the entry's slot.
__global__ void batch_horizon_many_kernel(const SlotSetup *__restrict__ list)
{
    __shared__ unsigned long long scratch[64];
    const SlotSetup &d = list[blockIdx.x];
    hj_prologue_block(d.st, d.geom, d.coef, d.ncoef, d.T, d.cfl, 0.0, scratch);
}

// What the consumers need of a work item, written into shared memory by the
// producer (with the item's first plane; the full barrier's arrive releases
// it), so that an item starts without a chain of dependent global loads.
struct BatchDesc {
    int item;                 // -1: no more work
    int slot;
    int y0, v0, x0, x1;       // tile origin and the item's x range [x0, x1)
    int n1, n2, n3, n4, p4, q4, ty, tv;
    int halo_floats;          // V0 box offset in a stage
    unsigned int per_step;    // consumer warps x the slot's items: finishes of one slot step
    float k3, k4, mk34, dt;   // v / theta coefficients and the slot's dt (working precision)
    float *vout;              // buffer of V_{n+1}
    const float *tab;         // v_k [n3], cos/dx1 [p4], sin/dx2 [p4]
};

// The planes of one item for one consumer thread (row r of the tile, theta
// quad q): waits for each plane, updates the thread's quad, stores V_{n+1},
// releases plane x-1.  PADDED: N4 is not a multiple of 4 (the last quad of a
// row has pad lanes: the theta wrap of its last real lane comes from lane 0
// of the row, and pad lanes are written as 0).  Returns false if a wait ran
// out.  Plane x-1 is carried in registers from the previous plane.
template <bool PADDED>
__device__ __forceinline__ bool batch_item_planes(const BatchDesc &d, int s_first, int q, int jy, int kv, bool rok,
                                                  const float *stages, int sfl, int nst, uint64_t *full,
                                                  uint64_t *empty, const unsigned long long *deadline_p, int lane,
                                                  int &wslot, uint32_t &wphase, int &rslot)
{
#define HJ_WAIT_NEXT(slot_out)                                   \
    do {                                                         \
        if (!mbar_wait_warp<true>(&full[wslot], wphase, deadline_p)) { \
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
    const int N1 = d.n1, N2 = d.n2, N3 = d.n3, N4 = d.n4, P4 = d.p4, tv = d.tv;
    const int x0 = d.x0, x1 = d.x1, pl0 = max(x0 - 1, 0), pl1 = min(x1, N1 - 1);
    const int y = d.y0 + jy, v = d.v0 + kv;
    const int srow = tv + 2;
    const int rsm = rok ? ((jy + 1) * srow + (kv + 1)) * P4 + 4 * q : (srow + 1) * P4;
    const int r0sm = d.halo_floats + (rok ? (jy * tv + kv) * P4 + 4 * q : 0);
    const uint32_t s1 = (uint32_t)N2 * N3 * P4;
    const uint32_t rbase = rok ? ((uint32_t)y * N3 + v) * P4 + 4 * q : 0u;
    const uint32_t gmask = (y == 0 ? 1u : 0u) | (y == N2 - 1 ? 2u : 0u) | (v == 0 ? 4u : 0u) |
                           (v == N3 - 1 ? 8u : 0u);
    const int lm = (4 * q - 1 + N4) % N4, lp = (4 * q + 4) % N4, lreal = min(4, N4 - 4 * q);
    const float k3 = d.k3, k4 = d.k4, mk34 = d.mk34, dt = d.dt;
    float *const vout = d.vout;
    float wx[4], wxm[4], wy[4], wym[4], cs[4];
    float vk = 0.f;
    if (rok) {
        // xdot_1 = v cos(th), xdot_2 = v sin(th): a negative speed flips the
        // upwind sides, and the weights take |v|
        vk = d.tab[v];
        const float sg = vk < 0.f ? -1.f : 1.f;
        vk = fabsf(vk);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float c = sg * d.tab[N3 + 4 * q + e], sn = sg * d.tab[N3 + P4 + 4 * q + e];
            wx[e] = fmaxf(c, 0.f);
            wxm[e] = fmaxf(-c, 0.f);
            wy[e] = fmaxf(sn, 0.f);
            wym[e] = fmaxf(-sn, 0.f);
            cs[e] = fabsf(c) + fabsf(sn);
        }
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) wx[e] = wxm[e] = wy[e] = wym[e] = cs[e] = 0.f;
    }
    // the weights as lane pairs (0, 1), (2, 3) and the constants broadcast
    const float2 wx01 = make_float2(wx[0], wx[1]), wx23 = make_float2(wx[2], wx[3]);
    const float2 wxm01 = make_float2(wxm[0], wxm[1]), wxm23 = make_float2(wxm[2], wxm[3]);
    const float2 wy01 = make_float2(wy[0], wy[1]), wy23 = make_float2(wy[2], wy[3]);
    const float2 wym01 = make_float2(wym[0], wym[1]), wym23 = make_float2(wym[2], wym[3]);
    const float2 ncs01 = make_float2(-cs[0], -cs[1]), ncs23 = make_float2(-cs[2], -cs[3]);
    const float2 k3p = make_float2(k3, k3), k4p = make_float2(k4, k4), mk34p = make_float2(mk34, mk34);
    const float2 vkp = make_float2(vk, vk), dtp = make_float2(dt, dt);
    int s_x = s_first;
    if (x0 > pl0) HJ_WAIT_NEXT(s_x);
    if (s_x < 0) return false;
    float4 cur = *(const float4 *)(stages + (size_t)s_x * sfl + rsm);
    int s_prev = x0 > pl0 ? s_first : -1;
    // centre of plane x-1, carried in registers from the previous plane
    float4 prevr = s_prev >= 0 ? *(const float4 *)(stages + (size_t)s_first * sfl + rsm) : cur;
    for (int x = x0; x < x1; ++x) {
        const float *sx = stages + (size_t)s_x * sfl;
        int s_n = -1;
        float4 prev, nxt;
        if (x + 1 <= N1 - 1) {
            HJ_WAIT_NEXT(s_n);
            if (s_n < 0) return false;
            nxt = *(const float4 *)(stages + (size_t)s_n * sfl + rsm);
            prev = s_prev >= 0 ? prevr : f4ghost(cur, nxt);
        } else {
            prev = s_prev >= 0 ? prevr : cur;
            nxt = f4ghost(cur, prev);
        }
        if (rok) {
            const float *row = sx + rsm;
            float4 ym = *(const float4 *)(row - srow * P4);
            float4 yp = *(const float4 *)(row + srow * P4);
            float4 vm = *(const float4 *)(row - P4);
            float4 vp = *(const float4 *)(row + P4);
            if (gmask) {  // extrapolated points past the y / v ends (Sec. II-B)
                if (gmask & 1u) ym = f4ghost(cur, yp);
                if (gmask & 2u) yp = f4ghost(cur, ym);
                if (gmask & 4u) vm = f4ghost(cur, vp);
                if (gmask & 8u) vp = f4ghost(cur, vm);
            }
            const float *row0 = row - 4 * q;
            const float tl = row0[lm], tr = row0[lp];
            float t0 = 0.f;
            if (PADDED) t0 = row0[0];
            const float4 v0c = *(const float4 *)(sx + r0sm);
            // theta neighbours: the larger of the two, per lane
            float tp3 = tr, tp2 = cur.w, tp1 = cur.z, tp0 = cur.y;
            if (PADDED && lreal < 4) {  // wrap of a padded last quad
                if (lreal == 1) tp0 = t0;
                if (lreal == 2) tp1 = t0;
                if (lreal == 3) tp2 = t0;
            }
            const float2 mt01 = make_float2(fmaxf(tp0, tl), fmaxf(tp1, cur.x));
            const float2 mt23 = make_float2(fmaxf(tp2, cur.y), fmaxf(tp3, cur.z));
            const float2 mv01 = make_float2(fmaxf(vp.x, vm.x), fmaxf(vp.y, vm.y));
            const float2 mv23 = make_float2(fmaxf(vp.z, vm.z), fmaxf(vp.w, vm.w));
            const float2 c01 = make_float2(cur.x, cur.y), c23 = make_float2(cur.z, cur.w);
            // lanes (0, 1) and (2, 3) in paired FP32 multiply-adds: the same
            // operations in the same order as one lane at a time, so the same bits
            float2 in01 = __fmul2_rn(wx01, make_float2(nxt.x, nxt.y));
            float2 in23 = __fmul2_rn(wx23, make_float2(nxt.z, nxt.w));
            in01 = __ffma2_rn(wxm01, make_float2(prev.x, prev.y), in01);
            in23 = __ffma2_rn(wxm23, make_float2(prev.z, prev.w), in23);
            in01 = __ffma2_rn(wy01, make_float2(yp.x, yp.y), in01);
            in23 = __ffma2_rn(wy23, make_float2(yp.z, yp.w), in23);
            in01 = __ffma2_rn(wym01, make_float2(ym.x, ym.y), in01);
            in23 = __ffma2_rn(wym23, make_float2(ym.z, ym.w), in23);
            in01 = __ffma2_rn(ncs01, c01, in01);
            in23 = __ffma2_rn(ncs23, c23, in23);
            float2 acc01 = __ffma2_rn(k3p, mv01, __fmul2_rn(mk34p, c01));
            float2 acc23 = __ffma2_rn(k3p, mv23, __fmul2_rn(mk34p, c23));
            acc01 = __ffma2_rn(k4p, mt01, acc01);
            acc23 = __ffma2_rn(k4p, mt23, acc23);
            acc01 = __ffma2_rn(vkp, in01, acc01);
            acc23 = __ffma2_rn(vkp, in23, acc23);
            const float2 u01 = __ffma2_rn(dtp, acc01, c01), u23 = __ffma2_rn(dtp, acc23, c23);
            float4 out = make_float4(fminf(v0c.x, u01.x), fminf(v0c.y, u01.y), fminf(v0c.z, u23.x),
                                     fminf(v0c.w, u23.y));
            if (PADDED && lreal < 4) {  // pad lanes hold 0
                if (lreal <= 1) out.y = 0.f;
                if (lreal <= 2) out.z = 0.f;
                out.w = 0.f;
            }
            *(float4 *)(vout + (uint32_t)x * s1 + rbase) = out;
        }
        if (s_prev >= 0) HJ_RELEASE_OLDEST();
        s_prev = s_x;
        s_x = s_n;
        prevr = cur;
        cur = nxt;
    }
    // still held: plane x1-1 and, if loaded, the halo plane x1
    HJ_RELEASE_OLDEST();
    if (x1 <= pl1) HJ_RELEASE_OLDEST();
    return true;
#undef HJ_WAIT_NEXT
#undef HJ_RELEASE_OLDEST
}

// One launch runs nrounds batch steps.  Round r holds the items of every
// slot with more than r steps to go: the first round_start[r + 1] -
// round_start[r] items of the item list (slots with more steps first), at
// queue positions round_start[r] onwards.  A slot moves to its next step as
// soon as its own step is finalised: the producer that takes an item of round
// r waits (bounded) until rounds_done[slot] (zeroed before the launch, raised
// by the slot's finalising warp after the slot's state is written and
// fenced) reaches r, then reads the slot's state.  Every item
// of the slot's round r - 1 comes earlier in the queue and needs nothing
// that a waiting producer holds, so the waits end.  Consumers make their
// stores visible to other SMs' tensor copies (a proxy fence and a release
// fence) before they count an item done; the producer acquires the finalised
// step before it issues the item's copies.
template <int MAXC, int MINB>
__global__ void __launch_bounds__(MAXC + 32, MINB)
    hj_batch_step_kernel(const BatchInst *__restrict__ insts, BatchSlot *slots, const BatchItem *__restrict__ items,
                         BatchCtl *ctl, const CUtensorMap *maps, const BatchParams BP,
                         const int *__restrict__ round_start, int *rounds_done, int nrounds)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float *stages = (float *)smem_raw;
    uint64_t *full = (uint64_t *)(smem_raw + (size_t)BP.stages * BP.stage_bytes);
    uint64_t *empty = full + B_MAX_STAGES;
    BatchDesc *desc = (BatchDesc *)(empty + B_MAX_STAGES);  // descriptor of the item whose first plane is in a stage
    volatile int *abort_flag = (volatile int *)(desc + B_MAX_STAGES);
    unsigned long long *deadline_p = (unsigned long long *)(abort_flag + 2);

    const int tid = threadIdx.x;
    const int nconsumer_warps = BP.nconsumer >> 5;
    const int nitems = ctl->nitems;
    if (tid == 0) {
        for (int s = 0; s < BP.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], nconsumer_warps);
        }
        *abort_flag = 0;
        *deadline_p = global_ns() + HJ_WAIT_NS;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    if (tid >= BP.nconsumer) {
        // ------------------------------------------------------------ producer
        if (tid == BP.nconsumer) {
            unsigned long long deadline = *deadline_p;
            int slot = 0;
            uint32_t phase = 0, issued = 0, used_mask = 0, last_phase = 0;
            bool ok = true;
            auto next_slot = [&]() -> bool {  // wait until ring slot `slot` is free
                if (issued >= (uint32_t)BP.stages && !mbar_wait(&empty[slot], phase ^ 1u, deadline)) return false;
                return *abort_flag == 0;
            };
            auto advance = [&]() {
                used_mask |= 1u << slot;
                last_phase = (last_phase & ~(1u << slot)) | (phase << slot);
                ++issued;
                if (++slot == BP.stages) {
                    slot = 0;
                    phase ^= 1u;
                }
            };
            int round = 0;
            while (ok) {
                const int gi = (int)atomicAdd(&ctl->head, 1u);
                if (gi >= nitems) break;
                while (round + 1 < nrounds && round_start[round + 1] <= gi) ++round;  // queue positions only grow
                const int item = gi - round_start[round];
                const BatchItem it = items[item];
                BatchSlot *sl = &slots[it.slot];
                // the slot's steps of the earlier rounds must be finalised
                // (bounded wait; a slot that reached its horizon has no more)
                const unsigned long long wdl = global_ns() + HJ_WAIT_NS;
                bool skip = false;
                while (*(volatile int *)&rounds_done[it.slot] < round) {
                    if (*(volatile int *)&sl->st.done) {
                        skip = true;
                        break;
                    }
                    if (global_ns() > wdl || *abort_flag) {
                        ok = false;
                        break;
                    }
                    __nanosleep(256);
                }
                if (!ok) break;
                if (skip) continue;
                __threadfence();  // acquire the slot's state and its V_n
                asm volatile("fence.proxy.async.global;" ::: "memory");
                if (*(volatile int *)&sl->st.done) continue;
                deadline = global_ns() + HJ_WAIT_NS;
                *deadline_p = deadline;  // the waits of this item: bounded per item
                const BatchInst &I = insts[it.slot];
                const long long n = *(volatile long long *)&sl->st.n;
                const CUtensorMap *m_in = &maps[4 * it.slot + (n == 0 ? 0 : 1 + (int)((n - 1) & 1))];
                const CUtensorMap *m_v0 = &maps[4 * it.slot + 3];
                tensormap_acquire(m_in);
                tensormap_acquire(m_v0);
                const int x1 = min(it.x0 + I.xc, I.n1), pl0 = max(it.x0 - 1, 0), pl1 = min(x1, I.n1 - 1);
                const uint32_t tx_halo = (uint32_t)(I.halo_box * 4), tx_v0 = (uint32_t)(I.v0_floats * 4);
                for (int p = pl0; p <= pl1; ++p) {
                    if (!next_slot()) {
                        ok = false;
                        break;
                    }
                    if (p == pl0) {  // the item's descriptor travels with its first plane
                        BatchDesc &D = desc[slot];
                        D.item = item;
                        D.slot = it.slot;
                        D.y0 = it.y0;
                        D.v0 = it.v0;
                        D.x0 = it.x0;
                        D.x1 = x1;
                        D.n1 = I.n1;
                        D.n2 = I.n2;
                        D.n3 = I.n3;
                        D.n4 = I.n4;
                        D.p4 = I.p4;
                        D.q4 = I.q4;
                        D.ty = I.ty;
                        D.tv = I.tv;
                        D.halo_floats = I.halo_floats;
                        D.per_step = (unsigned int)nconsumer_warps * (unsigned int)I.nitems;
                        D.k3 = I.k3;
                        D.k4 = I.k4;
                        D.mk34 = I.mk34;
                        D.dt = (float)*(volatile double *)&sl->st.dt;
                        D.vout = I.buf + (n & 1) * I.nint;
                        D.tab = I.tab;
                    }
                    const bool interior = p >= it.x0 && p < x1;
                    float *dst = stages + (size_t)slot * (BP.stage_bytes / 4);
                    mbar_arrive_expect_tx(&full[slot], tx_halo + (interior ? tx_v0 : 0u));
                    tma_load_4d(dst, m_in, &full[slot], 0, it.v0 - 1, it.y0 - 1, p);
                    if (interior) tma_load_4d(dst + I.halo_floats, m_v0, &full[slot], 0, it.v0, it.y0, p);
                    advance();
                }
            }
            // end of work: a stage whose descriptor says so, completed by a
            // plain arrive; it is that ring slot's last phase, so the drain
            // below waits for it (a parity wait only tells the current phase
            // from the one before)
            if (ok && next_slot()) {
                desc[slot].item = -1;
                mbar_arrive(&full[slot]);
                advance();
            } else {
                ok = false;
            }
            if (!ok) {
                ctl->status = HJ_ERR_TIMEOUT;
                *abort_flag = 1;
            }
            const unsigned long long drain_deadline = global_ns() + HJ_WAIT_NS;
            for (int s = 0; s < BP.stages; ++s)
                if (((used_mask >> s) & 1u) && !mbar_wait(&full[s], (last_phase >> s) & 1u, drain_deadline))
                    ctl->status = HJ_ERR_TIMEOUT;
        }
    } else {
        // ------------------------------------------------------------ consumers
        const int lane = tid & 31;
        int wslot = 0, rslot = 0;
        uint32_t wphase = 0;
        const int nst = BP.stages;
        const int sfl = BP.stage_bytes / 4;
        bool ok = true;
        while (ok) {
            // a producer that gave up stops the consumers at the next item (a
            // plane that never arrives ends their bounded waits instead)
            if (__any_sync(0xffffffffu, *abort_flag != 0)) {
                ok = false;
                break;
            }
            int s_first = -1;
            if (!mbar_wait_warp<true>(&full[wslot], wphase, deadline_p)) {
                ok = false;
                break;
            }
            s_first = wslot;
            if (++wslot == nst) {
                wslot = 0;
                wphase ^= 1u;
            }
            const BatchDesc d = desc[s_first];
            if (d.item < 0) break;  // no more work
            const int q = tid % d.q4, r = tid / d.q4;
            const int jy = r / d.tv, kv = r - (r / d.tv) * d.tv;
            const bool inrow = r < d.ty * d.tv;
            const bool rok = inrow && d.y0 + jy < d.n2 && d.v0 + kv < d.n3;
            ok = (d.p4 != d.n4)
                     ? batch_item_planes<true>(d, s_first, q, jy, kv, rok, stages, sfl, nst, full, empty, deadline_p,
                                               lane, wslot, wphase, rslot)
                     : batch_item_planes<false>(d, s_first, q, jy, kv, rok, stages, sfl, nst, full, empty, deadline_p,
                                                lane, wslot, wphase, rslot);
            if (!ok) break;

            // count the warp done; the warp completing the slot's step
            // reduces the slot's alpha^max over its per-speed table (every cell
            // of the slot was updated in this step, and the car's velocity
            // depends on v and theta only: the same maxima as over the cells)
            // and finalises the step
            // (this warp's stores of V_{n+1} are read by later items' tensor
            // copies on other SMs: proxy fence, then a release before the count)
            BatchSlot *sl = &slots[d.slot];
            asm volatile("fence.proxy.async.global;" ::: "memory");
            __syncwarp();
            unsigned int last = 0u;
            if (lane == 0) {
                __threadfence();
                last = atomicAdd(&sl->warps_done, 1u) + 1 == d.per_step;
            }
            if (__shfl_sync(0xffffffffu, last, 0)) {
                __threadfence();
                const BatchInst &I = insts[d.slot];
                unsigned long long a1 = 0ull, a2 = 0ull;
                for (int e = lane; e < d.n3; e += 32) {
                    const double2 am = I.amaxv[e];
                    const unsigned long long b1 = hj_abits(am.x), b2 = hj_abits(am.y);
                    a1 = a1 > b1 ? a1 : b1;
                    a2 = a2 > b2 ? a2 : b2;
                }
                a1 = hj_warp_max_u64(a1);
                a2 = hj_warp_max_u64(a2);
                if (lane == 0) {
                    atomicMax(&sl->st.alpha_bits[0], a1);
                    atomicMax(&sl->st.alpha_bits[1], a2);
                    hj_finalise(&sl->st, I.geom);
                    sl->warps_done = 0u;
                    __threadfence();
                    atomicAdd(&rounds_done[d.slot], 1);  // publish: the slot's next step may start
                }
            }
        }
        if (!ok) {
            ctl->status = HJ_ERR_TIMEOUT;
            *abort_flag = 1;
        }
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned int prev = atomicAdd(&ctl->ctas_done, 1u);
        if (prev == gridDim.x - 1) {  // last CTA: rewind the queue for the next launch
            ctl->head = 0u;
            ctl->ctas_done = 0u;
            __threadfence();
        }
    }
}
}  // namespace

// ======================================================================== host

namespace {

typedef CUresult (*BEncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

BEncodeFn batch_encode_fn()
{
    static BEncodeFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (BEncodeFn)p;
    }
    return fn;
}

typedef void (*BatchKernelFn)(const BatchInst *, BatchSlot *, const BatchItem *, BatchCtl *, const CUtensorMap *,
                              const BatchParams, const int *, int *, int);

BatchKernelFn batch_kernel(int nconsumer)
{
    if (nconsumer <= B_DUAL) return hj_batch_step_kernel<B_DUAL, 2>;
    if (nconsumer <= B_VARIANTS[0]) return hj_batch_step_kernel<B_VARIANTS[0], 1>;
    if (nconsumer <= B_VARIANTS[1]) return hj_batch_step_kernel<B_VARIANTS[1], 1>;
    if (nconsumer <= B_VARIANTS[2]) return hj_batch_step_kernel<B_VARIANTS[2], 1>;
    return hj_batch_step_kernel<B_VARIANTS[3], 1>;
}

size_t batch_smem(const BatchParams &bp)
{
    // ring, full / empty barriers, item descriptors, abort flag, deadline
    return (size_t)bp.stages * bp.stage_bytes + 2 * B_MAX_STAGES * sizeof(uint64_t) + B_MAX_STAGES * sizeof(BatchDesc) +
           2 * sizeof(int) + sizeof(unsigned long long) + 32;
}

struct SlotHost {
    bool used = false;
    int n[4] = {0, 0, 0, 0};
    double lo[4], hi[4], h[4];
    double a_max = 0, w_max = 0;
    int p4 = 0;
    long long nint = 0, ncell = 0;
    void *mem = nullptr;
    size_t bytes = 0;
    float *v0 = nullptr, *buf = nullptr, *tab = nullptr;
    HjCoef<float> *coef = nullptr;
    double2 *amaxv = nullptr;
    bool has_value = false;
    double T = 0, cfl = 0.8;
    int ty = 0, tv = 0, xc = 0;
    HjGeom geom;
};

}  // namespace

struct hj_batch {
    int max_slots = 0;
    size_t budget = 0, used_bytes = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0, sms = 0, maxsmem = 0, smem_sm = 0;
    std::vector<SlotHost> slots;
    BatchInst *d_insts = nullptr;
    BatchSlot *d_slots = nullptr;
    BatchSlot *h_slots = nullptr;  // pinned mirror
    BatchItem *d_items = nullptr;
    int items_cap = 0;
    std::vector<BatchInst> h_insts;  // host copy of d_insts (the item layout rewrites xc and nitems)
    std::vector<char> lay_active;    // slots the current item layout covers
    int lay_nitems = 0;              // source of the stream-ordered copy into d_ctl->nitems
    int lay_items = 0;               // items of one batch step in the current layout
    BatchCtl *d_ctl = nullptr;
    CUtensorMap *d_maps = nullptr;
    int nconsumer_req = 0;  // 0: automatic
    int xc_mode = 0;        // 0: automatic, k > 0: about n1 / k planes per chunk
    BatchParams bp = {0, 0, 0};
    int ctas = 0;
    bool dirty = true;
    int *d_rounds = nullptr;       // queue position of each round of a launch (B_MAX_ROUNDS + 1)
    int *d_rounds_done = nullptr;  // per slot: steps finalised in the current launch
    std::vector<int> h_rounds;     // source of the stream-ordered copy into d_rounds
    std::vector<int> lay_order;   // slot order of the current item layout
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaEvent_t ev_in = nullptr;  // own stream: orders device inputs after the legacy default stream
    SlotSetup *h_setup = nullptr;  // pinned staging of the multi-slot set-up lists (max_slots entries)
    SlotSetup *d_setup = nullptr;  // their device copy
    cudaEvent_t ev_setup = nullptr;  // the last staging copy has been read
};

namespace {

thread_local char b_err[256];

hj_status bfail(hj_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b_err, sizeof(b_err), fmt, ap);
    va_end(ap);
    hj_internal_set_error(b_err);
    return s;
}

#define HJB_CUDA(call)                                                                                   \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) {                                                                         \
            cudaGetLastError(); /* a failed call (not a sticky fault) must not fail later checks */      \
            return bfail(e_ == cudaErrorMemoryAllocation ? HJ_ERR_OOM : HJ_ERR_CUDA, "%s: %s", #call,      \
                         cudaGetErrorString(e_));                                                        \
        }                                                                                                \
    } while (0)


// Tile of one slot for a block of nc consumer threads (ty x tv <= nc / q4).
// Every item costs the whole block a pass over its planes, whether its rows
// fill the block or not (ragged last tiles along y and v), so: the fewest
// items per column sweep, then the fewest halo reads per row.
void choose_tile(const SlotHost &s, int nc, int *ty_out, int *tv_out)
{
    const int q4 = s.p4 / 4, max_rows = nc / q4;
    int bty = 1, btv = 1;
    double best = 1e300;
    for (int ty = 1; ty <= 16 && ty <= s.n[1]; ++ty)
        for (int tv = 1; tv <= 16 && tv <= s.n[2]; ++tv) {
            if (ty * tv > max_rows) continue;
            const double items = (double)((s.n[1] + ty - 1) / ty) * ((s.n[2] + tv - 1) / tv);
            const double halo = (double)(ty + 2) * (tv + 2) / (ty * tv);
            const double c = items * (1.0 + 0.02 * halo);
            if (c < best) {
                best = c;
                bty = ty;
                btv = tv;
            }
        }
    *ty_out = bty;
    *tv_out = btv;
}

hj_status upload_slot_tables(hj_batch *b, SlotHost &s)
{
    const int N3 = s.n[2], N4 = s.n[3], P4 = s.p4;
    std::vector<HjCoef<float>> c((size_t)N3 * N4);
    std::vector<float> tab((size_t)N3 + 2 * P4, 0.f);
    std::vector<double2> amax((size_t)N3, make_double2(0.0, 0.0));
    const double k3 = s.a_max / s.h[2], k4 = s.w_max / s.h[3];
    for (int k = 0; k < N3; ++k) {
        const double v = s.lo[2] + (double)k * s.h[2];
        tab[k] = (float)v;
        for (int l = 0; l < N4; ++l) {
            const double th = s.lo[3] + (double)l * s.h[3];
            const double f1 = v * hj_flush_trig(cos(th)), f2 = v * hj_flush_trig(sin(th));
            const double c1 = f1 / s.h[0], c2 = f2 / s.h[1];
            HjCoef<float> &e = c[(size_t)k * N4 + l];
            e.c1 = (float)c1;
            e.c2 = (float)c2;
            e.ks = (float)(fabs(c1) + fabs(c2) + k3 + k4);
            e.a1 = fabs(f1);
            e.a2 = fabs(f2);
            double2 &m = amax[k];  // the speed's largest |xdot_1|, |xdot_2|
            if (e.a1 > m.x) m.x = e.a1;
            if (e.a2 > m.y) m.y = e.a2;
        }
    }
    for (int l = 0; l < N4; ++l) {
        const double th = s.lo[3] + (double)l * s.h[3];
        tab[N3 + l] = (float)(hj_flush_trig(cos(th)) / s.h[0]);
        tab[N3 + P4 + l] = (float)(hj_flush_trig(sin(th)) / s.h[1]);
    }
    HJB_CUDA(cudaMemcpyAsync(s.coef, c.data(), sizeof(HjCoef<float>) * c.size(), cudaMemcpyHostToDevice, b->stream));
    HJB_CUDA(cudaMemcpyAsync(s.tab, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice, b->stream));
    HJB_CUDA(cudaMemcpyAsync(s.amaxv, amax.data(), sizeof(double2) * amax.size(), cudaMemcpyHostToDevice, b->stream));
    HJB_CUDA(cudaStreamSynchronize(b->stream));  // the host vectors go out of scope
    return HJ_OK;
}

// Item layout of the slots marked in `active` for `ctas` resident CTAs (the
// tiles chosen by rebuild): x chunks per slot, h_insts' xc and nitems
// (0 for the others), and the queue in order.  Whole columns while the
// active slots have at least one (y, v) column per CTA, else enough chunks
// (of at least 4 planes) to give every CTA an item, since a column's planes
// are streamed one after another by one CTA.  (With the steps of a launch
// overlapping, nothing is gained by cutting some columns shorter: cutting
// the queue's last slots, or the slots with the most steps, into x chunks
// measured slower, 19.6-19.7 against 19.4 ms per batch64 solve.)  Slots with
// more steps to go come first, then the longest columns.  A fixed chunk
// count (hj_batch_set_shape) replaces the automatic one.
void plan_layout(hj_batch *b, const std::vector<char> &active, const std::vector<long long> &ki, long long ctas,
                 std::vector<BatchItem> &items)
{
    items.clear();
    long long columns = 0;
    int min_n1 = 1 << 30;
    std::vector<int> order;
    for (int i = 0; i < b->max_slots; ++i) {
        b->h_insts[i].nitems = 0;
        if (!b->slots[i].used || !active[i]) continue;
        const SlotHost &s = b->slots[i];
        columns += (long long)((s.n[1] + s.ty - 1) / s.ty) * ((s.n[2] + s.tv - 1) / s.tv);
        if (s.n[0] < min_n1) min_n1 = s.n[0];
        order.push_back(i);
    }
    int nchunk = b->xc_mode > 0 ? b->xc_mode : 1;
    if (b->xc_mode == 0 && columns > 0 && columns < ctas) {
        nchunk = (int)((ctas + columns - 1) / columns);
        const int most = min_n1 / 4 > 1 ? min_n1 / 4 : 1;  // chunks of at least 4 planes
        if (nchunk > most) nchunk = most;
    }
    // slots with more steps to go first (a launch's later rounds are then a
    // prefix of the list), then the longest columns first
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        if (ki[a] != ki[c]) return ki[a] > ki[c];
        return b->slots[a].n[0] > b->slots[c].n[0];
    });
    std::vector<int> slot_chunks(b->max_slots, nchunk);
    for (int i : order) {
        SlotHost &s = b->slots[i];
        s.xc = (s.n[0] + slot_chunks[i] - 1) / slot_chunks[i];
        if (s.xc < 4) s.xc = s.n[0] < 4 ? s.n[0] : 4;
        const int ncv = (s.n[2] + s.tv - 1) / s.tv, ncy = (s.n[1] + s.ty - 1) / s.ty;
        const int nch = (s.n[0] + s.xc - 1) / s.xc;
        b->h_insts[i].xc = s.xc;
        b->h_insts[i].nitems = ncv * ncy * nch;
        for (int c = 0; c < nch; ++c)
            for (int yt = 0; yt < ncy; ++yt)
                for (int vt = 0; vt < ncv; ++vt) items.push_back({i, yt * s.ty, vt * s.tv, c * s.xc});
    }
    b->lay_active = active;
    b->lay_order = order;
}

// Resident CTAs of a block of nc consumers (before the occupancy query).
long long resident_ctas(const hj_batch *b, int nc) { return (long long)b->sms * (nc <= B_DUAL ? 2 : 1); }

// Rebuild the per-slot descriptors, tensor maps and item list after slots or
// the kernel shape changed.
hj_status rebuild(hj_batch *b)
{
    BEncodeFn enc = batch_encode_fn();
    if (!enc) return bfail(HJ_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    // block size: the request, else the smallest variant that gives every
    // slot at least 32 rows
    int nc = b->nconsumer_req;
    if (nc <= 0) {
        nc = B_VARIANTS[0];
        for (auto &s : b->slots)
            if (s.used) {
                const int need = (s.p4 / 4) * 32;
                while (nc < need && nc < B_VARIANTS[3]) nc += 128;
            }
    }
    b->h_insts.assign(b->max_slots, BatchInst());
    std::vector<BatchInst> &insts = b->h_insts;
    std::vector<CUtensorMap> maps((size_t)4 * b->max_slots);
    memset(insts.data(), 0, sizeof(BatchInst) * insts.size());
    memset(maps.data(), 0, sizeof(CUtensorMap) * maps.size());
    std::vector<BatchItem> items;
    int stage_bytes = 128;
    int max_cons = 32;
    std::vector<char> all(b->max_slots, 0);
    for (int i = 0; i < b->max_slots; ++i) {
        SlotHost &s = b->slots[i];
        if (!s.used) continue;
        choose_tile(s, nc, &s.ty, &s.tv);
        all[i] = 1;
    }
    plan_layout(b, all, std::vector<long long>(b->max_slots, 1), resident_ctas(b, nc), items);
    for (int i = 0; i < b->max_slots; ++i) {
        if (!all[i]) continue;
        SlotHost &s = b->slots[i];
        BatchInst &I = insts[i];
        I.n1 = s.n[0];
        I.n2 = s.n[1];
        I.n3 = s.n[2];
        I.n4 = s.n[3];
        I.p4 = s.p4;
        I.q4 = s.p4 / 4;
        I.ty = s.ty;
        I.tv = s.tv;
        I.halo_box = s.p4 * (s.tv + 2) * (s.ty + 2);
        I.halo_floats = (I.halo_box + 31) / 32 * 32;
        I.v0_floats = s.p4 * s.ty * s.tv;
        I.k3 = (float)(s.a_max / s.h[2]);
        I.k4 = (float)(s.w_max / s.h[3]);
        I.mk34 = (float)(-(s.a_max / s.h[2] + s.w_max / s.h[3]));
        I.nint = s.nint;
        I.buf = s.buf;
        I.tab = s.tab;
        I.coef = s.coef;
        I.amaxv = s.amaxv;
        I.geom = s.geom;
        const int sb = ((I.halo_floats + I.v0_floats) * 4 + 127) / 128 * 128;
        if (sb > stage_bytes) stage_bytes = sb;
        const int cons = ((I.q4 * s.ty * s.tv) + 31) / 32 * 32;
        if (cons > max_cons) max_cons = cons;
        // tensor maps: V0 / A / B with the halo box, V0 with the tile box
        cuuint64_t dims[4] = {(cuuint64_t)s.p4, (cuuint64_t)s.n[2], (cuuint64_t)s.n[1], (cuuint64_t)s.n[0]};
        cuuint64_t strides[3] = {(cuuint64_t)s.p4 * 4, (cuuint64_t)s.p4 * s.n[2] * 4,
                                 (cuuint64_t)s.p4 * s.n[2] * s.n[1] * 4};
        cuuint32_t box_halo[4] = {(cuuint32_t)s.p4, (cuuint32_t)(s.tv + 2), (cuuint32_t)(s.ty + 2), 1};
        cuuint32_t box_tile[4] = {(cuuint32_t)s.p4, (cuuint32_t)s.tv, (cuuint32_t)s.ty, 1};
        cuuint32_t estr[4] = {1, 1, 1, 1};
        void *bases[4] = {s.v0, s.buf, s.buf + s.nint, s.v0};
        for (int m = 0; m < 4; ++m) {
            CUresult r = enc(&maps[4 * i + m], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, bases[m], dims, strides,
                             m < 3 ? box_halo : box_tile, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return bfail(HJ_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for slot %d", (int)r, i);
        }
    }
    BatchParams bp;
    bp.nconsumer = max_cons;
    bp.stage_bytes = stage_bytes;
    // two CTAs per SM for the smallest shapes: each gets half of the SM's
    // shared memory, less the 1 KB the runtime reserves per block
    const int smem_cta = max_cons <= B_DUAL ? b->smem_sm / 2 - 1024 : b->maxsmem;
    bp.stages = (int)((smem_cta - 4096) / stage_bytes);
    if (bp.stages > B_MAX_STAGES) bp.stages = B_MAX_STAGES;
    if (bp.stages < 4) return bfail(HJ_ERR_UNSUPPORTED, "a slot's tile does not fit four ring stages");
    // device copies
    // room for the layouts of the advance loop's later phases too (at most
    // about four items per resident CTA beyond this layout's count)
    const int need = (int)items.size() + 4 * (int)resident_ctas(b, nc) + 64;
    if (need > b->items_cap) {
        if (b->d_items) cudaFree(b->d_items);
        b->d_items = nullptr;
        b->items_cap = 0;
        const int cap = need + (int)items.size();
        HJB_CUDA(cudaMalloc(&b->d_items, sizeof(BatchItem) * cap));
        b->items_cap = cap;
    }
    HJB_CUDA(cudaStreamSynchronize(b->stream));
    if (!items.empty())
        HJB_CUDA(cudaMemcpy(b->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice));
    HJB_CUDA(cudaMemcpy(b->d_insts, insts.data(), sizeof(BatchInst) * insts.size(), cudaMemcpyHostToDevice));
    HJB_CUDA(cudaMemcpy(b->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice));
    BatchCtl ctl = {0u, 0u, (int)items.size(), HJ_OK};
    HJB_CUDA(cudaMemcpy(b->d_ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice));
    b->lay_items = (int)items.size();
    if (bp.nconsumer != b->bp.nconsumer || bp.stages != b->bp.stages || bp.stage_bytes != b->bp.stage_bytes) {
        b->bp = bp;
        BatchKernelFn fn = batch_kernel(bp.nconsumer);
        const size_t smem = batch_smem(bp);
        HJB_CUDA(cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        HJB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)fn, bp.nconsumer + 32, smem));
        if (per_sm < 1) return bfail(HJ_ERR_UNSUPPORTED, "batch kernel shape does not fit on an SM");
        b->ctas = b->sms * per_sm;
    }
    b->dirty = false;
    return HJ_OK;
}

// Item layout of the slots with ki > 0, ordered by ki (steps to go), for a
// launch.  The item list, the per-slot descriptors and the item count go to
// the device by copies queued on the batch's stream, so they take effect
// after every launch queued before.  A no-op when the layout covers the same
// slots in the same order.
hj_status apply_layout(hj_batch *b, const std::vector<long long> &ki)
{
    std::vector<char> active(b->max_slots, 0);
    for (int i = 0; i < b->max_slots; ++i) active[i] = b->slots[i].used && ki[i] > 0;
    std::vector<int> order;
    for (int i = 0; i < b->max_slots; ++i)
        if (active[i]) order.push_back(i);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        if (ki[a] != ki[c]) return ki[a] > ki[c];
        return b->slots[a].n[0] > b->slots[c].n[0];
    });
    if (active == b->lay_active && order == b->lay_order) return HJ_OK;
    std::vector<BatchItem> items;
    plan_layout(b, active, ki, b->ctas, items);
    if ((int)items.size() > b->items_cap)
        return bfail(HJ_ERR_CUDA, "batch item layout of %d items exceeds its buffer (%d)", (int)items.size(),
                     b->items_cap);
    // pageable sources: each copy has taken its data when the call returns
    if (!items.empty())
        HJB_CUDA(cudaMemcpyAsync(b->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice,
                                 b->stream));
    HJB_CUDA(cudaMemcpyAsync(b->d_insts, b->h_insts.data(), sizeof(BatchInst) * b->h_insts.size(),
                             cudaMemcpyHostToDevice, b->stream));
    b->lay_items = (int)items.size();
    return HJ_OK;
}

// k batch steps (k <= B_MAX_ROUNDS) as one launch: every slot i takes
// min(ki[i], k) of them (round r holds the slots with ki > r, a prefix of
// the layout).
hj_status run_rounds(hj_batch *b, const std::vector<long long> &ki, long long k)
{
    if (k <= 0) return HJ_OK;
    if (k > B_MAX_ROUNDS) return bfail(HJ_ERR_INVALID_ARG, "at most %d batch steps per launch", B_MAX_ROUNDS);
    hj_status s = apply_layout(b, ki);
    if (s != HJ_OK) return s;
    // round r: the items of the slots with ki > r (a prefix of the layout)
    std::vector<long long> per_slot(b->max_slots, 0);
    for (int i = 0; i < b->max_slots; ++i) per_slot[i] = b->h_insts[i].nitems;
    b->h_rounds.assign((size_t)k + 1, 0);
    long long pos = 0;
    for (long long r = 0; r < k; ++r) {
        b->h_rounds[r] = (int)pos;
        for (int i : b->lay_order)
            if (ki[i] > r) pos += per_slot[i];
    }
    if (pos >= (1LL << 31)) return bfail(HJ_ERR_INVALID_ARG, "too many work items in one launch");
    b->h_rounds[k] = (int)pos;
    HJB_CUDA(cudaMemcpyAsync(b->d_rounds, b->h_rounds.data(), sizeof(int) * (k + 1), cudaMemcpyHostToDevice,
                             b->stream));
    HJB_CUDA(cudaMemsetAsync(b->d_rounds_done, 0, sizeof(int) * b->max_slots, b->stream));
    b->lay_nitems = (int)pos;
    HJB_CUDA(cudaMemcpyAsync((char *)b->d_ctl + offsetof(BatchCtl, nitems), &b->lay_nitems, sizeof(int),
                             cudaMemcpyHostToDevice, b->stream));
    BatchKernelFn fn = batch_kernel(b->bp.nconsumer);
    fn<<<b->ctas, b->bp.nconsumer + 32, batch_smem(b->bp), b->stream>>>(b->d_insts, b->d_slots, b->d_items, b->d_ctl,
                                                                        b->d_maps, b->bp, b->d_rounds,
                                                                        b->d_rounds_done, (int)k);
    HJB_CUDA(cudaGetLastError());
    return HJ_OK;
}

// Steps to go of every slot: ceil((T - t) / dt) (exact while dt stays
// constant, as with the car's fixed alpha^max; the advance loop re-plans
// otherwise), 0 for a slot that is not running.
std::vector<long long> steps_to_go(const hj_batch *b)
{
    std::vector<long long> ki(b->max_slots, 0);
    for (int i = 0; i < b->max_slots; ++i) {
        if (!b->slots[i].used) continue;
        const HjDevState &h = b->h_slots[i].st;
        if (h.done || h.status != HJ_OK) continue;
        ki[i] = 1;
        if (!h.last && h.dt > 0) {
            const double r = ceil((h.T - h.t) / h.dt);
            ki[i] = r > 1 ? (r < 1e9 ? (long long)r : 1000000000LL) : 1;
        }
    }
    return ki;
}

hj_status pull_slots(hj_batch *b)
{
    HJB_CUDA(cudaMemcpyAsync(b->h_slots, b->d_slots, sizeof(BatchSlot) * b->max_slots, cudaMemcpyDeviceToHost,
                             b->stream));
    HJB_CUDA(cudaStreamSynchronize(b->stream));
    return HJ_OK;
}

hj_status push_slot(hj_batch *b, int i)
{
    HJB_CUDA(cudaMemcpyAsync(&b->d_slots[i], &b->h_slots[i], sizeof(BatchSlot), cudaMemcpyHostToDevice, b->stream));
    HJB_CUDA(cudaStreamSynchronize(b->stream));
    return HJ_OK;
}

// Queue the host mirror of slot i to the device without waiting: every later
// host read of the mirror comes after a stream synchronisation, and the
// mirror entry is not written again before then.
hj_status push_slot_async(hj_batch *b, int i)
{
    HJB_CUDA(cudaMemcpyAsync(&b->d_slots[i], &b->h_slots[i], sizeof(BatchSlot), cudaMemcpyHostToDevice, b->stream));
    return HJ_OK;
}

// Whether the ingest queued on the stream saw a NaN or Inf in slot i's V0
// (waits for the stream).
hj_status pull_nonfinite(hj_batch *b, int i, bool *bad)
{
    HJB_CUDA(cudaMemcpyAsync(&b->h_slots[i].st.nonfinite, &b->d_slots[i].st.nonfinite, sizeof(int),
                             cudaMemcpyDeviceToHost, b->stream));
    HJB_CUDA(cudaStreamSynchronize(b->stream));
    *bad = b->h_slots[i].st.nonfinite != 0;
    return HJ_OK;
}

hj_status check_slot(const hj_batch *b, int slot)
{
    if (!b) return bfail(HJ_ERR_INVALID_ARG, "batch is NULL");
    if (slot < 0 || slot >= b->max_slots || !b->slots[slot].used)
        return bfail(HJ_ERR_INVALID_ARG, "slot %d is not in use", slot);
    return HJ_OK;
}

}  // namespace

extern "C" {

hj_status hj_batch_create(int32_t max_slots, size_t memory_budget, void *cuda_stream, hj_batch **out)
{
    hj_internal_set_error("");
    if (!out) return bfail(HJ_ERR_INVALID_ARG, "out is NULL");
    if (max_slots < 1 || max_slots > 4096) return bfail(HJ_ERR_INVALID_ARG, "max_slots must be in [1, 4096]");
    hj_batch *b = new (std::nothrow) hj_batch();
    if (!b) return bfail(HJ_ERR_OOM, "host allocation failed");
    b->max_slots = max_slots;
    b->slots.resize(max_slots);
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->maxsmem, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&b->smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, b->device);
    size_t free_b = 0, total_b = 0;
    if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
    b->budget = memory_budget > 0 ? memory_budget : (size_t)(0.9 * (double)free_b);
    if (e == cudaSuccess && cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else if (e == cudaSuccess) {
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        b->own_stream = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->d_insts, sizeof(BatchInst) * max_slots);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_slots, sizeof(BatchSlot) * max_slots);
    if (e == cudaSuccess) e = cudaHostAlloc(&b->h_slots, sizeof(BatchSlot) * max_slots, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(&b->h_setup, sizeof(SlotSetup) * max_slots, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_setup, sizeof(SlotSetup) * max_slots);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_setup, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ctl, sizeof(BatchCtl));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_rounds, sizeof(int) * (B_MAX_ROUNDS + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_rounds_done, sizeof(int) * max_slots);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_maps, sizeof(CUtensorMap) * 4 * max_slots);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreate(&b->ev[i]);
    if (e == cudaSuccess && b->own_stream) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) {
        memset(b->h_slots, 0, sizeof(BatchSlot) * max_slots);
        for (int i = 0; i < max_slots; ++i) b->h_slots[i].st.done = 1;
        e = cudaMemcpy(b->d_slots, b->h_slots, sizeof(BatchSlot) * max_slots, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemset(b->d_insts, 0, sizeof(BatchInst) * max_slots);
    if (e == cudaSuccess) e = cudaMemset(b->d_ctl, 0, sizeof(BatchCtl));
    if (e != cudaSuccess) {
        cudaGetLastError();  // the failed allocation must not fail later launch checks
        hj_status s = bfail(e == cudaErrorMemoryAllocation ? HJ_ERR_OOM : HJ_ERR_CUDA, "hj_batch_create: %s",
                            cudaGetErrorString(e));
        hj_batch_destroy(b);
        return s;
    }
    *out = b;
    return HJ_OK;
}

void hj_batch_destroy(hj_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto &s : b->slots)
        if (s.mem) cudaFree(s.mem);
    if (b->d_insts) cudaFree(b->d_insts);
    if (b->d_slots) cudaFree(b->d_slots);
    if (b->h_slots) cudaFreeHost(b->h_slots);
    if (b->h_setup) cudaFreeHost(b->h_setup);
    if (b->d_setup) cudaFree(b->d_setup);
    if (b->ev_setup) cudaEventDestroy(b->ev_setup);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_ctl) cudaFree(b->d_ctl);
    if (b->d_rounds) cudaFree(b->d_rounds);
    if (b->d_rounds_done) cudaFree(b->d_rounds_done);
    if (b->d_maps) cudaFree(b->d_maps);
    for (int i = 0; i < 2; ++i)
        if (b->ev[i]) cudaEventDestroy(b->ev[i]);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

// Device memory of one slot: V0, buffers A|B (contiguous), coefficient
// table, tiled tables; each section 256-byte aligned.
static void slot_layout(const int32_t n[4], size_t *v0_b, size_t *ab_b, size_t *coef_b, size_t *tab_b,
                        size_t *amax_b)
{
    const long long p4 = (n[3] + 3) / 4 * 4;
    const long long nint = (long long)n[0] * n[1] * n[2] * p4;
    *v0_b = ((size_t)nint * 4 + 255) / 256 * 256;
    *ab_b = ((size_t)nint * 8 + 255) / 256 * 256;
    *coef_b = ((size_t)n[2] * n[3] * sizeof(HjCoef<float>) + 255) / 256 * 256;
    *tab_b = (((size_t)n[2] + 2 * (size_t)p4) * 4 + 255) / 256 * 256;
    *amax_b = ((size_t)n[2] * sizeof(double2) + 255) / 256 * 256;
}

size_t hj_batch_slot_bytes(const int32_t n[4])
{
    if (!n) return 0;
    for (int d = 0; d < 4; ++d)
        if (n[d] < 1) return 0;
    size_t a, b2, c, t, am;
    slot_layout(n, &a, &b2, &c, &t, &am);
    return a + b2 + c + t + am;
}

hj_status hj_batch_add(hj_batch *b, const int32_t n[4], const double lo[4], const double hi[4], const double params[2],
                       int32_t *slot_out)
{
    hj_internal_set_error("");
    if (!b || !n || !lo || !hi || !params || !slot_out) return bfail(HJ_ERR_INVALID_ARG, "NULL argument");
    for (int d = 0; d < 4; ++d) {
        if (n[d] < 3) return bfail(HJ_ERR_INVALID_ARG, "N%d = %d < 3", d + 1, n[d]);
        if (!isfinite(lo[d]) || !isfinite(hi[d]) || !(hi[d] > lo[d]))
            return bfail(HJ_ERR_INVALID_ARG, "axis %d bounds must be finite with hi > lo", d + 1);
    }
    if (!isfinite(params[0]) || !isfinite(params[1]) || params[0] < 0 || params[1] < 0)
        return bfail(HJ_ERR_INVALID_ARG, "a_max and w_max must be finite and >= 0");
    const int p4 = (n[3] + 3) / 4 * 4;
    if (p4 > 256) return bfail(HJ_ERR_UNSUPPORTED, "theta rows longer than 256 points");
    if ((p4 / 4) > B_VARIANTS[3]) return bfail(HJ_ERR_UNSUPPORTED, "theta rows too long");
    const long long nint = (long long)n[0] * n[1] * n[2] * p4;
    if (nint >= (1LL << 31)) return bfail(HJ_ERR_UNSUPPORTED, "grid too large for a batch slot");
    int slot = -1;
    for (int i = 0; i < b->max_slots; ++i)
        if (!b->slots[i].used) {
            slot = i;
            break;
        }
    if (slot < 0) return bfail(HJ_ERR_OOM, "all %d slots are in use", b->max_slots);
    const size_t bytes = hj_batch_slot_bytes(n);
    if (b->used_bytes + bytes > b->budget)
        return bfail(HJ_ERR_OOM, "slot needs %zu bytes; %zu of the %zu-byte budget are in use", bytes, b->used_bytes,
                     b->budget);
    int cur = -1;
    HJB_CUDA(cudaGetDevice(&cur));
    if (cur != b->device) HJB_CUDA(cudaSetDevice(b->device));
    SlotHost s;
    s.used = true;
    for (int d = 0; d < 4; ++d) {
        s.n[d] = n[d];
        s.lo[d] = lo[d];
        s.hi[d] = hi[d];
        s.h[d] = (hi[d] - lo[d]) / (double)(d == 3 ? n[d] : n[d] - 1);  // theta periodic, the rest not
    }
    s.a_max = params[0];
    s.w_max = params[1];
    s.p4 = p4;
    s.nint = nint;
    s.ncell = (long long)n[0] * n[1] * n[2] * n[3];
    HJB_CUDA(cudaMalloc(&s.mem, bytes));
    s.bytes = bytes;
    size_t sz_v0, sz_ab, sz_coef, sz_tab, sz_amax;
    slot_layout(n, &sz_v0, &sz_ab, &sz_coef, &sz_tab, &sz_amax);
    char *m = (char *)s.mem;
    s.v0 = (float *)m;
    s.buf = (float *)(m + sz_v0);  // A, then B at buf + nint
    s.coef = (HjCoef<float> *)(m + sz_v0 + sz_ab);
    s.tab = (float *)(m + sz_v0 + sz_ab + sz_coef);
    s.amaxv = (double2 *)(m + sz_v0 + sz_ab + sz_coef + sz_tab);
    memset(&s.geom, 0, sizeof(s.geom));
    s.geom.n1 = n[0];
    s.geom.n2 = n[1];
    s.geom.n3 = n[2];
    s.geom.n4 = n[3];
    s.geom.p4 = p4;
    s.geom.periodic = 0x8;
    s.geom.mode3 = s.geom.mode4 = HJ_AXIS_CONTROL;
    for (int d = 0; d < 4; ++d) s.geom.h[d] = s.h[d];
    s.geom.alpha3 = s.a_max;
    s.geom.alpha4 = s.w_max;
    s.geom.k3 = s.a_max / s.h[2];
    s.geom.k4 = s.w_max / s.h[3];
    b->slots[slot] = s;
    hj_status st = upload_slot_tables(b, b->slots[slot]);
    if (st != HJ_OK) {
        cudaFree(s.mem);
        b->slots[slot] = SlotHost();
        return st;
    }
    b->used_bytes += bytes;
    memset(&b->h_slots[slot], 0, sizeof(BatchSlot));
    b->h_slots[slot].st.done = 1;  // no horizon yet
    if ((st = push_slot(b, slot)) != HJ_OK) return st;
    b->dirty = true;
    *slot_out = slot;
    return HJ_OK;
}

hj_status hj_batch_remove(hj_batch *b, int32_t slot)
{
    hj_internal_set_error("");
    hj_status s = check_slot(b, slot);
    if (s != HJ_OK) return s;
    HJB_CUDA(cudaStreamSynchronize(b->stream));
    memset(&b->h_slots[slot], 0, sizeof(BatchSlot));
    b->h_slots[slot].st.done = 1;
    if ((s = push_slot(b, slot)) != HJ_OK) return s;
    cudaFree(b->slots[slot].mem);
    b->used_bytes -= b->slots[slot].bytes;
    b->slots[slot] = SlotHost();
    b->dirty = true;
    return HJ_OK;
}

// Checks a slot's V0 arguments.
static hj_status ingest_check(hj_batch *b, int32_t slot, const void *src, size_t count)
{
    hj_status s = check_slot(b, slot);
    if (s != HJ_OK) return s;
    if (!src) return bfail(HJ_ERR_INVALID_ARG, "v0 is NULL");
    if (count != (size_t)b->slots[slot].ncell)
        return bfail(HJ_ERR_INVALID_ARG, "count %zu != %lld", count, b->slots[slot].ncell);
    return HJ_OK;
}

// Queues a slot's V0 ingest (reset state, staging copy, conversion kernel
// with its NaN / Inf flag) on the batch's stream, without waiting.
static hj_status ingest_queue(hj_batch *b, int32_t slot, const void *src, hj_precision type, bool on_host)
{
    SlotHost &sl = b->slots[slot];
    // (every call of the batch API returns with its stream work done or with
    // a synchronisation after its last use of the host mirror, so the mirror
    // entry is free to rewrite; the reset state is queued, not waited for)
    memset(&b->h_slots[slot], 0, sizeof(BatchSlot));
    b->h_slots[slot].st.done = 1;  // until a horizon is set
    b->h_slots[slot].st.status = HJ_OK;
    hj_status s;
    if ((s = push_slot_async(b, slot)) != HJ_OK) return s;
    const void *dsrc = src;
    if (on_host) {  // stage the FP64 array in the slot's A|B region (2 nint floats >= ncell doubles)
        HJB_CUDA(cudaMemcpyAsync(sl.buf, src, sizeof(double) * (size_t)sl.ncell, cudaMemcpyHostToDevice, b->stream));
        dsrc = sl.buf;
    }
    int *flag = &b->d_slots[slot].st.nonfinite;
    HJB_CUDA(hj_launch_ingest_f32(dsrc, type, sl.v0, sl.n[3], sl.p4, (long long)sl.n[0] * sl.n[1] * sl.n[2], flag,
                                  b->stream));
    return HJ_OK;
}

// A batch on its own (non-blocking) stream reads a caller's device arrays
// only after the work already queued on the legacy default stream.
static hj_status order_after_default_stream(hj_batch *b)
{
    if (b->own_stream) {
        HJB_CUDA(cudaEventRecord(b->ev_in, cudaStreamLegacy));
        HJB_CUDA(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    }
    return HJ_OK;
}

static hj_status batch_ingest(hj_batch *b, int32_t slot, const void *src, hj_precision type, bool on_host,
                              size_t count)
{
    hj_status s = ingest_check(b, slot, src, count);
    if (s != HJ_OK) return s;
    SlotHost &sl = b->slots[slot];
    if (!on_host && (s = order_after_default_stream(b)) != HJ_OK) return s;
    if ((s = ingest_queue(b, slot, src, type, on_host)) != HJ_OK) return s;
    bool bad = false;
    if ((s = pull_nonfinite(b, slot, &bad)) != HJ_OK) return s;
    if (bad) {
        sl.has_value = false;
        return bfail(HJ_ERR_INVALID_ARG, "V0 contains NaN or Inf");
    }
    sl.has_value = true;
    return HJ_OK;
}

hj_status hj_batch_set_initial_value_xy(hj_batch *b, int32_t slot, const double *v0_xy, size_t count)
{
    hj_internal_set_error("");
    hj_status s = check_slot(b, slot);
    if (s != HJ_OK) return s;
    SlotHost &sl = b->slots[slot];
    if (!v0_xy) return bfail(HJ_ERR_INVALID_ARG, "v0_xy is NULL");
    const long long nxy = (long long)sl.n[0] * sl.n[1];
    if (count != (size_t)nxy) return bfail(HJ_ERR_INVALID_ARG, "count %zu != N1*N2 = %lld", count, nxy);
    memset(&b->h_slots[slot], 0, sizeof(BatchSlot));
    b->h_slots[slot].st.done = 1;
    if ((s = push_slot_async(b, slot)) != HJ_OK) return s;
    HJB_CUDA(cudaMemcpyAsync(sl.buf, v0_xy, sizeof(double) * (size_t)nxy, cudaMemcpyHostToDevice, b->stream));
    HJB_CUDA(hj_launch_ingest_xy_f32((const double *)sl.buf, sl.v0, sl.n[2], sl.n[3], sl.p4, nxy,
                                     &b->d_slots[slot].st.nonfinite, b->stream));
    bool bad = false;
    if ((s = pull_nonfinite(b, slot, &bad)) != HJ_OK) return s;
    if (bad) {
        sl.has_value = false;
        return bfail(HJ_ERR_INVALID_ARG, "V0 contains NaN or Inf");
    }
    sl.has_value = true;
    return HJ_OK;
}

hj_status hj_batch_set_initial_value(hj_batch *b, int32_t slot, const double *v0, size_t count)
{
    hj_internal_set_error("");
    return batch_ingest(b, slot, v0, HJ_FP64, true, count);
}

hj_status hj_batch_set_initial_value_device(hj_batch *b, int32_t slot, const void *v0, hj_precision dtype,
                                            size_t count)
{
    hj_internal_set_error("");
    if (dtype != HJ_FP64 && dtype != HJ_FP32) return bfail(HJ_ERR_INVALID_ARG, "unknown dtype");
    return batch_ingest(b, slot, v0, dtype, false, count);
}

hj_status hj_batch_set_initial_values_device(hj_batch *b, int32_t nslots, const int32_t *slots,
                                             const void *const *v0, hj_precision dtype, const size_t *counts)
{
    hj_internal_set_error("");
    if (!b) return bfail(HJ_ERR_INVALID_ARG, "batch is NULL");
    if (nslots < 0 || (nslots > 0 && (!slots || !v0 || !counts)))
        return bfail(HJ_ERR_INVALID_ARG, "nslots must be >= 0 with non-NULL slots, v0 and counts");
    if (dtype != HJ_FP64 && dtype != HJ_FP32) return bfail(HJ_ERR_INVALID_ARG, "unknown dtype");
    hj_status s;
    for (int32_t k = 0; k < nslots; ++k)  // every argument first: nothing is queued for a bad call
        if ((s = ingest_check(b, slots[k], v0[k], counts[k])) != HJ_OK) return s;
    if (nslots == 0) return HJ_OK;
    if ((s = order_after_default_stream(b)) != HJ_OK) return s;
    // reset the slots' states: the mirror entries, pushed as runs of
    // consecutive slots
    for (int32_t k = 0; k < nslots; ++k) {
        memset(&b->h_slots[slots[k]], 0, sizeof(BatchSlot));
        b->h_slots[slots[k]].st.done = 1;  // until a horizon is set
    }
    std::vector<int32_t> sorted(slots, slots + nslots);
    std::sort(sorted.begin(), sorted.end());
    sorted.erase(std::unique(sorted.begin(), sorted.end()), sorted.end());
    for (size_t a = 0; a < sorted.size();) {
        size_t c = a + 1;
        while (c < sorted.size() && sorted[c] == sorted[c - 1] + 1) ++c;
        HJB_CUDA(cudaMemcpyAsync(&b->d_slots[sorted[a]], &b->h_slots[sorted[a]], sizeof(BatchSlot) * (c - a),
                                 cudaMemcpyHostToDevice, b->stream));
        a = c;
    }
    // one conversion launch for all the slots
    HJB_CUDA(cudaEventSynchronize(b->ev_setup));  // the previous list has been copied
    long long most = 1;
    for (int32_t k = 0; k < nslots; ++k) {
        const SlotHost &sl = b->slots[slots[k]];
        SlotSetup &e = b->h_setup[k];
        e.src = v0[k];
        e.dst = sl.v0;
        e.st = &b->d_slots[slots[k]].st;
        e.nrows = (long long)sl.n[0] * sl.n[1] * sl.n[2];
        e.n4 = sl.n[3];
        e.p4 = sl.p4;
        if (e.nrows * e.p4 > most) most = e.nrows * e.p4;
    }
    HJB_CUDA(cudaMemcpyAsync(b->d_setup, b->h_setup, sizeof(SlotSetup) * nslots, cudaMemcpyHostToDevice, b->stream));
    HJB_CUDA(cudaEventRecord(b->ev_setup, b->stream));
    long long bx = (most + 255) / 256;
    if (bx > 1024) bx = 1024;
    const dim3 grid((unsigned)bx, (unsigned)nslots);
    if (dtype == HJ_FP64) batch_ingest_many_kernel<double><<<grid, 256, 0, b->stream>>>(b->d_setup);
    else batch_ingest_many_kernel<float><<<grid, 256, 0, b->stream>>>(b->d_setup);
    HJB_CUDA(cudaGetLastError());
    // one synchronisation for every slot's NaN / Inf check
    if ((s = pull_slots(b)) != HJ_OK) return s;
    int first_bad = -1;
    for (int32_t k = 0; k < nslots; ++k) {
        const bool bad = b->h_slots[slots[k]].st.nonfinite != 0;
        b->slots[slots[k]].has_value = !bad;
        if (bad && first_bad < 0) first_bad = slots[k];
    }
    if (first_bad >= 0) return bfail(HJ_ERR_INVALID_ARG, "slot %d: V0 contains NaN or Inf", first_bad);
    return HJ_OK;
}

hj_status hj_batch_set_horizon(hj_batch *b, int32_t slot, double T, double cfl)
{
    hj_internal_set_error("");
    hj_status s = check_slot(b, slot);
    if (s != HJ_OK) return s;
    if (!isfinite(T) || T < 0) return bfail(HJ_ERR_INVALID_ARG, "T must be finite and >= 0");
    if (!isfinite(cfl) || !(cfl > 0) || cfl > 1) return bfail(HJ_ERR_INVALID_ARG, "cfl must be in (0, 1]");
    SlotHost &sl = b->slots[slot];
    if (!sl.has_value) return bfail(HJ_ERR_STATE, "slot %d has no initial value", slot);
    sl.T = T;
    sl.cfl = cfl;
    // queued on the batch's stream (ordered before the next batch step); the
    // calls that read slot states synchronise first
    HJB_CUDA(hj_launch_prologue_f32(&b->d_slots[slot].st, sl.geom, sl.coef, sl.n[2] * sl.n[3], T, cfl, b->stream));
    return HJ_OK;
}

hj_status hj_batch_set_horizons(hj_batch *b, int32_t nslots, const int32_t *slots, const double *T, const double *cfl)
{
    hj_internal_set_error("");
    if (!b) return bfail(HJ_ERR_INVALID_ARG, "batch is NULL");
    if (nslots < 0 || (nslots > 0 && (!slots || !T || !cfl)))
        return bfail(HJ_ERR_INVALID_ARG, "nslots must be >= 0 with non-NULL slots, T and cfl");
    hj_status s;
    for (int32_t k = 0; k < nslots; ++k) {  // every argument first: nothing is queued for a bad call
        if ((s = check_slot(b, slots[k])) != HJ_OK) return s;
        if (!isfinite(T[k]) || T[k] < 0) return bfail(HJ_ERR_INVALID_ARG, "slot %d: T must be finite and >= 0", slots[k]);
        if (!isfinite(cfl[k]) || !(cfl[k] > 0) || cfl[k] > 1)
            return bfail(HJ_ERR_INVALID_ARG, "slot %d: cfl must be in (0, 1]", slots[k]);
        if (!b->slots[slots[k]].has_value) return bfail(HJ_ERR_STATE, "slot %d has no initial value", slots[k]);
    }
    if (nslots == 0) return HJ_OK;
    HJB_CUDA(cudaEventSynchronize(b->ev_setup));  // the previous list has been copied
    for (int32_t k = 0; k < nslots; ++k) {
        SlotHost &sl = b->slots[slots[k]];
        sl.T = T[k];
        sl.cfl = cfl[k];
        SlotSetup &e = b->h_setup[k];
        e.st = &b->d_slots[slots[k]].st;
        e.geom = sl.geom;
        e.coef = sl.coef;
        e.ncoef = sl.n[2] * sl.n[3];
        e.T = T[k];
        e.cfl = cfl[k];
    }
    // one launch, one block per slot (queued; ordered before the next batch step)
    HJB_CUDA(cudaMemcpyAsync(b->d_setup, b->h_setup, sizeof(SlotSetup) * nslots, cudaMemcpyHostToDevice, b->stream));
    HJB_CUDA(cudaEventRecord(b->ev_setup, b->stream));
    batch_horizon_many_kernel<<<nslots, 256, 0, b->stream>>>(b->d_setup);
    HJB_CUDA(cudaGetLastError());
    return HJ_OK;
}

hj_status hj_batch_advance(hj_batch *b, int64_t max_steps, hj_batch_stats *stats)
{
    hj_internal_set_error("");
    if (!b) return bfail(HJ_ERR_INVALID_ARG, "batch is NULL");
    if (max_steps < 0) return bfail(HJ_ERR_INVALID_ARG, "max_steps must be >= 0");
    hj_status s;
    if (b->dirty && (s = rebuild(b)) != HJ_OK) return s;
    long long taken = 0, launches = 0;
    bool started = false;
    if ((s = pull_slots(b)) != HJ_OK) return s;
    HJB_CUDA(cudaEventRecord(b->ev[0], b->stream));
    while (taken < max_steps) {
        // batch steps until the slowest unfinished slot reaches its horizon,
        // up to B_MAX_ROUNDS per launch; each slot takes its own steps to go
        const std::vector<long long> ki = steps_to_go(b);
        long long k = 0;
        for (long long v : ki) k = v > k ? v : k;
        if (k == 0) break;
        if (k > max_steps - taken) k = max_steps - taken;
        if (k > B_MAX_ROUNDS) k = B_MAX_ROUNDS;
        if ((s = run_rounds(b, ki, k)) != HJ_OK) return s;
        started = true;
        launches += 1;
        taken += k;
        if ((s = pull_slots(b)) != HJ_OK) return s;
        BatchCtl ctl;
        HJB_CUDA(cudaMemcpy(&ctl, b->d_ctl, sizeof(ctl), cudaMemcpyDeviceToHost));
        if (ctl.status != HJ_OK)
            return bfail((hj_status)ctl.status, "device reported %s", hj_status_string((hj_status)ctl.status));
    }
    HJB_CUDA(cudaEventRecord(b->ev[1], b->stream));
    HJB_CUDA(cudaEventSynchronize(b->ev[1]));
    int active = 0, finished = 0;
    for (int i = 0; i < b->max_slots; ++i) {
        if (!b->slots[i].used) continue;
        const HjDevState &h = b->h_slots[i].st;
        if (h.status != HJ_OK)
            return bfail((hj_status)h.status, "slot %d: device reported %s", i, hj_status_string((hj_status)h.status));
        if (!h.done) ++active;
        else if (b->slots[i].has_value && b->slots[i].T > 0 && h.t >= b->slots[i].T) ++finished;
    }
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->steps = taken;
        stats->launches = launches;
        stats->active = active;
        stats->finished = finished;
        float ms = 0.f;
        if (started) cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]);
        stats->device_ms = ms;
        stats->nconsumer = b->bp.nconsumer;
        stats->ctas = b->ctas;
        stats->items = b->lay_items;
    }
    return HJ_OK;
}

hj_status hj_batch_get_slot_info(const hj_batch *bc, int32_t slot, hj_batch_slot_info *info)
{
    hj_internal_set_error("");
    hj_batch *b = (hj_batch *)bc;
    hj_status s = check_slot(b, slot);
    if (s != HJ_OK) return s;
    if (!info) return bfail(HJ_ERR_INVALID_ARG, "info is NULL");
    if ((s = pull_slots(b)) != HJ_OK) return s;
    const SlotHost &sl = b->slots[slot];
    const HjDevState &h = b->h_slots[slot].st;
    memset(info, 0, sizeof(*info));
    for (int d = 0; d < 4; ++d) info->n[d] = sl.n[d];
    info->steps = h.n;
    info->t = h.t;
    info->T = sl.T;
    info->dt_last = h.dt_prev;
    info->done = h.done;
    info->has_value = sl.has_value;
    info->tile[0] = sl.ty;
    info->tile[1] = sl.tv;
    info->tile[2] = sl.xc;
    info->device_bytes = sl.bytes;
    return HJ_OK;
}

static hj_status batch_read(hj_batch *b, int32_t slot, void *out, hj_precision dtype, bool to_host, size_t count)
{
    hj_status s = check_slot(b, slot);
    if (s != HJ_OK) return s;
    const SlotHost &sl = b->slots[slot];
    if (!out) return bfail(HJ_ERR_INVALID_ARG, "out is NULL");
    if (count != (size_t)sl.ncell) return bfail(HJ_ERR_INVALID_ARG, "count %zu != %lld", count, sl.ncell);
    if (!sl.has_value) return bfail(HJ_ERR_STATE, "slot %d has no initial value", slot);
    if ((s = pull_slots(b)) != HJ_OK) return s;
    const long long n = b->h_slots[slot].st.n;
    const float *src = n == 0 ? sl.v0 : sl.buf + ((n - 1) & 1) * sl.nint;
    const long long nrows = (long long)sl.n[0] * sl.n[1] * sl.n[2];
    if (!to_host) {
        if (b->own_stream) {  // the caller's array may still be in use on the legacy default stream
            HJB_CUDA(cudaEventRecord(b->ev_in, cudaStreamLegacy));
            HJB_CUDA(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
        }
        HJB_CUDA(hj_launch_readback_f32(src, out, dtype, sl.n[3], sl.p4, 0, nrows, b->stream));
        HJB_CUDA(cudaStreamSynchronize(b->stream));
        return HJ_OK;
    }
    // convert into the free buffer in chunks of rows, copy each out
    float *freebuf = n == 0 ? sl.buf : sl.buf + (n & 1) * sl.nint;
    const size_t free_bytes = (n == 0 ? 2 : 1) * (size_t)sl.nint * 4;
    const long long per = (long long)(free_bytes / (sizeof(double) * (size_t)sl.n[3]));
    for (long long r0 = 0; r0 < nrows; r0 += per) {
        const long long nr = nrows - r0 < per ? nrows - r0 : per;
        HJB_CUDA(hj_launch_readback_f32(src, freebuf, HJ_FP64, sl.n[3], sl.p4, r0, nr, b->stream));
        HJB_CUDA(cudaMemcpyAsync((double *)out + r0 * sl.n[3], freebuf, sizeof(double) * (size_t)(nr * sl.n[3]),
                                 cudaMemcpyDeviceToHost, b->stream));
    }
    HJB_CUDA(cudaStreamSynchronize(b->stream));
    return HJ_OK;
}

hj_status hj_batch_read_value(hj_batch *b, int32_t slot, double *out, size_t count)
{
    hj_internal_set_error("");
    return batch_read(b, slot, out, HJ_FP64, true, count);
}

hj_status hj_batch_read_value_device(hj_batch *b, int32_t slot, void *out_device, hj_precision dtype, size_t count)
{
    hj_internal_set_error("");
    if (dtype != HJ_FP64 && dtype != HJ_FP32) return bfail(HJ_ERR_INVALID_ARG, "unknown dtype");
    return batch_read(b, slot, out_device, dtype, false, count);
}

hj_status hj_batch_set_shape(hj_batch *b, int32_t nconsumer, int32_t chunks)
{
    hj_internal_set_error("");
    if (!b) return bfail(HJ_ERR_INVALID_ARG, "batch is NULL");
    if (nconsumer != 0 && (nconsumer < 128 || nconsumer > B_VARIANTS[3] || nconsumer % 32 != 0))
        return bfail(HJ_ERR_INVALID_ARG, "nconsumer must be 0 or a multiple of 32 in [128, %d]", B_VARIANTS[3]);
    if (chunks < 0 || chunks > 64) return bfail(HJ_ERR_INVALID_ARG, "chunks must be in [0, 64]");
    HJB_CUDA(cudaStreamSynchronize(b->stream));
    b->nconsumer_req = nconsumer;
    b->xc_mode = chunks;
    b->dirty = true;
    return HJ_OK;
}

hj_status hj_batch_autotune(hj_batch *b, int32_t steps_per_trial, int32_t *best_nconsumer, int32_t *best_chunks,
                            double *best_ms_per_step)
{
    hj_internal_set_error("");
    if (!b) return bfail(HJ_ERR_INVALID_ARG, "batch is NULL");
    if (steps_per_trial < 1) return bfail(HJ_ERR_INVALID_ARG, "steps_per_trial must be >= 1");
    hj_status s;
    if ((s = pull_slots(b)) != HJ_OK) return s;
    for (int i = 0; i < b->max_slots; ++i)
        if (b->slots[i].used && (b->h_slots[i].st.n != 0 || !b->slots[i].has_value))
            return bfail(HJ_ERR_STATE, "autotune needs every slot right after its initial value (slot %d)", i);
    std::vector<BatchSlot> saved(b->h_slots, b->h_slots + b->max_slots);
    const int keep_nc = b->nconsumer_req, keep_ch = b->xc_mode;
    double best = 1e300;
    int best_nc = keep_nc, best_ch = keep_ch;
    const int ncs[5] = {B_DUAL, B_VARIANTS[0], B_VARIANTS[1], B_VARIANTS[2], B_VARIANTS[3]};
    const int chs[4] = {0, 1, 2, 4};
    for (int a = 0; a < 5; ++a)
        for (int c = 0; c < 4; ++c) {
            b->nconsumer_req = ncs[a];
            b->xc_mode = chs[c];
            b->dirty = true;
            if ((s = rebuild(b)) != HJ_OK) {
                if (s == HJ_ERR_UNSUPPORTED) continue;
                break;
            }
            // trial: every slot from its initial value with an unreachable horizon
            for (int i = 0; i < b->max_slots; ++i)
                if (b->slots[i].used)
                    hj_launch_prologue_f32(&b->d_slots[i].st, b->slots[i].geom, b->slots[i].coef,
                                           b->slots[i].n[2] * b->slots[i].n[3], 1e300, 0.8, b->stream);
            // (the trial's steps: every slot takes each of them)
            std::vector<long long> all(b->max_slots, 0);
            for (int i = 0; i < b->max_slots; ++i) all[i] = b->slots[i].used ? (1LL << 40) : 0;
            if ((s = run_rounds(b, all, 2)) != HJ_OK) break;
            cudaEventRecord(b->ev[0], b->stream);
            const int kt = steps_per_trial > B_MAX_ROUNDS ? B_MAX_ROUNDS : steps_per_trial;
            if ((s = run_rounds(b, all, kt)) != HJ_OK) break;
            cudaEventRecord(b->ev[1], b->stream);
            cudaEventSynchronize(b->ev[1]);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]);
            const double per = ms / kt;
            if (per < best) {
                best = per;
                best_nc = ncs[a];
                best_ch = chs[c];
            }
            // put the states back
            memcpy(b->h_slots, saved.data(), sizeof(BatchSlot) * b->max_slots);
            HJB_CUDA(cudaMemcpyAsync(b->d_slots, b->h_slots, sizeof(BatchSlot) * b->max_slots, cudaMemcpyHostToDevice,
                                     b->stream));
            HJB_CUDA(cudaStreamSynchronize(b->stream));
        }
    memcpy(b->h_slots, saved.data(), sizeof(BatchSlot) * b->max_slots);
    cudaMemcpyAsync(b->d_slots, b->h_slots, sizeof(BatchSlot) * b->max_slots, cudaMemcpyHostToDevice, b->stream);
    cudaStreamSynchronize(b->stream);
    b->nconsumer_req = best < 1e300 ? best_nc : keep_nc;
    b->xc_mode = best < 1e300 ? best_ch : keep_ch;
    b->dirty = true;
    hj_status r = rebuild(b);
    if (s == HJ_OK) s = r;
    if (best_nconsumer) *best_nconsumer = b->nconsumer_req;
    if (best_chunks) *best_chunks = b->xc_mode;
    if (best_ms_per_step) *best_ms_per_step = best < 1e300 ? best : 0.0;
    return s;
}

}  // extern "C"

// Internal (not in the C ABI): pull every slot's state once, then read the
// host copy.
hj_status hj_batch_refresh(hj_batch *b)
{
    if (!b) return bfail(HJ_ERR_INVALID_ARG, "batch is NULL");
    return pull_slots(b);
}

bool hj_batch_cached_done(const hj_batch *b, int32_t slot, int64_t *steps)
{
    if (!b || slot < 0 || slot >= b->max_slots) return false;
    if (steps) *steps = b->h_slots[slot].st.n;
    return b->h_slots[slot].st.done != 0;
}
