// Grid-wide barrier of the resident step kernel (hj_step_generic.cu), which
// runs many time steps in one cooperative launch: every CTA is resident at
// once (cudaLaunchCooperativeKernel checks the grid against the occupancy),
// so a CTA that waits for the others never blocks one that has not started.
//
// One counter, zeroed before the launch, counts arrivals: barrier b of the
// launch (b = 0, 1, ...) is complete when it reaches nblocks * (b + 1).
// Thread 0 of every CTA adds its arrival with acquire-release semantics and
// waits with acquire loads, so the writes of every CTA before the barrier
// are visible to every CTA after it.  Each wait is bounded by %globaltimer:
// after limit_ns the CTA gives up and the barrier returns false (the kernel
// then records HJ_ERR_TIMEOUT and returns), so no failure can leave the GPU
// spinning.
#pragma once

#include "hj_tma.cuh"

__device__ __forceinline__ unsigned int hj_ld_acquire_u32(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned int hj_atom_add_acq_rel_u32(unsigned int *p, unsigned int x)
{
    unsigned int old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(x) : "memory");
    return old;
}

// Every thread of every CTA calls it with the same target.  Writes made by
// any thread of any CTA before the barrier are visible to every thread after
// it (to loads that bypass L1: ld.global.cg, atomics).  s_ok is a shared int
// of the CTA.
__device__ __forceinline__ bool hj_grid_sync(unsigned int *count, unsigned int target, unsigned long long limit_ns,
                                             int *s_ok)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (hj_atom_add_acq_rel_u32(count, 1u) + 1u < target) {
            const unsigned long long deadline = global_ns() + limit_ns;
            while (hj_ld_acquire_u32(count) < target) {
                if (global_ns() > deadline) {
                    ok = 0;
                    break;
                }
            }
        }
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}
