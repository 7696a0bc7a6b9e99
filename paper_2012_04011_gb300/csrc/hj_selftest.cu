// Self-test of the bounded device-side waits (failure detection without a
// GPU fault).  Every mbarrier wait of the step kernels gives up at a
// deadline read from %globaltimer and records HJ_ERR_TIMEOUT instead of
// spinning forever.  This kernel exercises exactly that path: one producer
// thread initialises an mbarrier that expects one arrival and never
// arrives; the consumer warps wait on it with the same warp-uniform bounded
// waits (mbar_wait_warp, with and without the suspend-time hint) as the step
// kernels, give up at the deadline and
// record the status.  Nothing faults, traps or hangs; the context stays
// usable.  The grid-barrier self-test does the same for the resident step
// kernel's barrier (hj_grid_sync): two co-resident CTAs wait for a third
// arrival that never comes.
//
// Also here: the FP64 fused multiply-add throughput probe that the FP64
// roofline of the FP64 step kernel and of the query kernel is measured
// against (GB300's FP64 rate is a small fraction of its FP32 rate, so the
// measured figure, not a nominal one, is the denominator).
#include "hj_resident.cuh"

namespace {

// Written only when a chain sum is negative, which the probe's inputs never
// give; the store keeps every chain live without a buffer from the caller.
__device__ double g_fma_sink;

constexpr int FMA_CHAINS = 8;

// Each thread runs FMA_CHAINS independent DFMA chains x <- x a + b of iters
// steps (a < 1, b > 0: the chains stay in [0, 1]).
__global__ void __launch_bounds__(256) fp64_fma_probe_kernel(long long iters, double a, double b)
{
    double x[FMA_CHAINS];
#pragma unroll
    for (int j = 0; j < FMA_CHAINS; ++j) x[j] = (double)((threadIdx.x + 7 * j) & 255) * (1.0 / 512.0);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < FMA_CHAINS; ++j) x[j] = fma(x[j], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < FMA_CHAINS; ++j) s += x[j];
    if (s < 0.0) g_fma_sink = s;
}

__global__ void wait_selftest_kernel(unsigned long long limit_ns, int *status, unsigned long long *waited_ns)
{
    __shared__ __align__(8) uint64_t bar;
    __shared__ unsigned long long deadline;
    __shared__ unsigned long long t0;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);  // one arrival expected; nothing arrives
        t0 = global_ns();
        deadline = t0 + limit_ns;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // warp 0 waits as the HBM-bound step kernels do, warp 1 with the
    // suspend-time hint of the issue-bound ones
    const bool ok = (threadIdx.x >> 5) & 1 ? mbar_wait_warp<true>(&bar, 0u, &deadline)
                                           : mbar_wait_warp<false>(&bar, 0u, &deadline);
    if (!ok && (threadIdx.x & 31) == 0) atomicExch(status, (int)HJ_ERR_TIMEOUT);
    __syncthreads();
    if (threadIdx.x == 0) *waited_ns = global_ns() - t0;
}

// Two CTAs, a barrier that expects three arrivals.
__global__ void barrier_selftest_kernel(HjResidentSync *sync, unsigned long long limit_ns, int *status,
                                        unsigned long long *waited_ns)
{
    __shared__ int s_ok;
    const unsigned long long t0 = global_ns();
    const bool ok = hj_grid_sync(&sync->count, gridDim.x + 1u, limit_ns, &s_ok);
    if (threadIdx.x == 0) {
        if (!ok) atomicExch(status, (int)HJ_ERR_TIMEOUT);
        atomicMax(waited_ns, global_ns() - t0);
    }
}

typedef void (*SelftestLaunch)(unsigned long long limit_ns, int *status, unsigned long long *waited_ns, void *scratch,
                               cudaError_t *err);

// Runs one self-test kernel with a device status word, waited time and
// scratch area; copies the results back.
hj_status run_selftest(int64_t limit_ns, int32_t *status, int64_t *waited_ns, SelftestLaunch launch)
{
    hj_internal_set_error("");
    if (!status) {
        hj_internal_set_error("status is NULL");
        return HJ_ERR_INVALID_ARG;
    }
    if (limit_ns < 1000000 || limit_ns > 2000000000) {
        hj_internal_set_error("limit_ns must be in [1 ms, 2 s]");
        return HJ_ERR_INVALID_ARG;
    }
    char *d = nullptr;
    const size_t bytes = 16 + sizeof(HjResidentSync);
    cudaError_t e = cudaMalloc(&d, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();  // the failed allocation must not fail later launch checks
        hj_internal_set_error(cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? HJ_ERR_OOM : HJ_ERR_CUDA;
    }
    int *d_status = (int *)d;
    unsigned long long *d_waited = (unsigned long long *)(d + 8);
    e = cudaMemset(d, 0, bytes);
    if (e == cudaSuccess) launch((unsigned long long)limit_ns, d_status, d_waited, d + 16, &e);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int h_status = -1;
    unsigned long long h_waited = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&h_waited, d_waited, sizeof(h_waited), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        hj_internal_set_error(cudaGetErrorString(e));
        return HJ_ERR_CUDA;
    }
    *status = h_status;
    if (waited_ns) *waited_ns = (int64_t)h_waited;
    return HJ_OK;
}

void launch_wait(unsigned long long limit_ns, int *status, unsigned long long *waited_ns, void *, cudaError_t *err)
{
    wait_selftest_kernel<<<1, 64>>>(limit_ns, status, waited_ns);
    *err = cudaGetLastError();
}

void launch_barrier(unsigned long long limit_ns, int *status, unsigned long long *waited_ns, void *scratch,
                    cudaError_t *err)
{
    HjResidentSync *sync = (HjResidentSync *)scratch;
    void *args[] = {&sync, &limit_ns, &status, &waited_ns};
    *err = cudaLaunchCooperativeKernel((const void *)barrier_selftest_kernel, 2, 64, args, 0, 0);
}

}  // namespace

extern "C" hj_status hj_barrier_selftest(int64_t limit_ns, int32_t *status, int64_t *waited_ns)
{
    return run_selftest(limit_ns, status, waited_ns, launch_barrier);
}

extern "C" hj_status hj_wait_selftest(int64_t limit_ns, int32_t *status, int64_t *waited_ns)
{
    return run_selftest(limit_ns, status, waited_ns, launch_wait);
}

extern "C" hj_status hj_fp64_fma_probe(int64_t iters, int32_t blocks_per_sm, void *cuda_stream, int64_t *fma_out)
{
    hj_internal_set_error("");
    if (iters < 1 || iters > (1LL << 40) || blocks_per_sm < 1 || blocks_per_sm > 64) {
        hj_internal_set_error("iters must be in [1, 2^40] and blocks_per_sm in [1, 64]");
        return HJ_ERR_INVALID_ARG;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        hj_internal_set_error(cudaGetErrorString(e));
        return HJ_ERR_CUDA;
    }
    const int blocks = sms * blocks_per_sm, threads = 256;
    // a = 1 - 2^-20, b = 2^-20: every chain moves toward 1 and stays in [0, 1]
    fp64_fma_probe_kernel<<<blocks, threads, 0, (cudaStream_t)cuda_stream>>>((long long)iters, 1.0 - 0x1p-20,
                                                                            0x1p-20);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        hj_internal_set_error(cudaGetErrorString(e));
        return HJ_ERR_CUDA;
    }
    if (fma_out) *fma_out = (int64_t)blocks * threads * FMA_CHAINS * iters;
    return HJ_OK;
}
