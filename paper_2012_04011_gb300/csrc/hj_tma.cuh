// Shared device helpers of the TMA-fed step kernels: mbarrier waits bounded
// by %globaltimer, 4D tensor copies, float4 lane access.
#pragma once

#include "hj_device.cuh"

constexpr unsigned long long HJ_WAIT_NS = 4000000000ull;  // 4 s per wait: far beyond any healthy wait

static __device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

static __device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
static __device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
static __device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
static __device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
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
// The same try with a suspend-time hint: the thread may sleep until the phase
// completes or HJ_TRY_WAIT_NS pass, so a waiting warp spins a few times per
// wait instead of many, leaving issue slots to the warps that compute (the
// issue-bound kernels gain; the HBM-bound 4D FP32 step, whose warps mostly
// wait on memory, measured slower with it).
constexpr uint32_t HJ_TRY_WAIT_NS = 20000u;
static __device__ __forceinline__ bool mbar_try_wait_hint(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(HJ_TRY_WAIT_NS)
        : "memory");
    return ok != 0;
}
static __device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase with the given parity; false if the deadline passed.
static __device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned long long deadline)
{
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() > deadline) return false;
    }
    return true;
}
// Warp-uniform version for consumer warps: every lane observes the phase,
// and the timeout decision is the same for the whole warp.  The deadline is
// read (from shared memory) only when the phase is not complete yet.
template <bool HINT = false>
static __device__ __forceinline__ bool mbar_wait_warp(uint64_t *bar, uint32_t parity, const unsigned long long *deadline)
{
    while (true) {
        bool done = HINT ? mbar_try_wait_hint(bar, parity) : mbar_try_wait(bar, parity);
        if (__all_sync(0xffffffffu, done)) return true;
        bool late = global_ns() > *deadline;
        if (__any_sync(0xffffffffu, late)) return false;
    }
}
static __device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1, int c2,
                                            int c3)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

static __device__ __forceinline__ float f4get(const float4 &v, int e)
{
    return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}
static __device__ __forceinline__ void f4set(float4 &v, int e, float x)
{
    if (e == 0) v.x = x;
    else if (e == 1) v.y = x;
    else if (e == 2) v.z = x;
    else v.w = x;
}
static __device__ __forceinline__ float4 f4ghost(const float4 &c, const float4 &o)
{
    return make_float4(2.f * c.x - o.x, 2.f * c.y - o.y, 2.f * c.z - o.z, 2.f * c.w - o.w);
}

