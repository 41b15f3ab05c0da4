// Self-tests of the device-side failure detection: one block whose threads
// wait, with a short bound, on an mbarrier phase that nothing completes --
// the same bounded wait (bounded_wait) that the TMA-fed single-pass kernels
// use -- or one thread that waits on a progress counter nothing advances --
// the bounded wait (bounded_progress_wait) of the fused in-place form.  The
// wait must give up, report ELBM_ERR_TIMEOUT through the status word, and
// leave the context usable.
#include <cstdio>

#include "fused_aa.cuh"

namespace {

__global__ void __launch_bounds__(32) k_selftest_wait(int* status, unsigned long long limit_ns)
{
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        elbm::mbar_init(elbm::smem_u32(&bar), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // nothing arrives on the barrier, so phase 0 never completes
    (void)elbm::bounded_wait(elbm::smem_u32(&bar), 0u, &abort_flag, status, limit_ns);
}

// One thread waits for a counter (zeroed, never advanced) to reach 1.
__global__ void __launch_bounds__(32) k_selftest_counter(const unsigned long long* counter, int* status,
                                                         unsigned long long limit_ns)
{
    if (threadIdx.x == 0) (void)elbm::bounded_progress_wait(counter, 1ull, status, elbm::globaltimer_ns(), limit_ns);
}

// Run one self-test kernel (which = 0 mbarrier wait, 1 progress-counter wait)
// with bound limit_ms; ELBM_ERR_TIMEOUT when it gave up as designed.
int selftest(int which, int limit_ms, void* stream)
{
    elbm::set_error(ELBM_OK, "");
    if (limit_ms < 1 || limit_ms > 2000) return elbm::set_error(ELBM_ERR_ARG, "limit_ms must be in 1..2000");
    (void)cudaGetLastError();  // a stale error of an earlier call is not this call's
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* status = nullptr;
    unsigned long long* counter = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&status, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (e == cudaSuccess && which == 1) e = cudaMallocAsync((void**)&counter, sizeof(unsigned long long), st);
    if (e == cudaSuccess && which == 1) e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
        const unsigned long long limit_ns = 1000000ull * (unsigned long long)limit_ms;
        if (which == 0) k_selftest_wait<<<1, 32, 0, st>>>(status, limit_ns);
        else k_selftest_counter<<<1, 32, 0, st>>>(counter, status, limit_ns);
        e = cudaGetLastError();
    }
    int host = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (status) cudaFreeAsync(status, st);
    if (counter) cudaFreeAsync(counter, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return elbm::set_error(ELBM_ERR_CUDA, cudaGetErrorString(e));
    if (host == ELBM_ERR_TIMEOUT) return elbm::set_error(ELBM_ERR_TIMEOUT, "the bounded wait gave up as designed");
    char msg[96];
    std::snprintf(msg, sizeof msg, "the bounded wait did not report a timeout (status %d)", host);
    return elbm::set_error(ELBM_ERR_STATE, msg);
}

}  // namespace

extern "C" int elbm_selftest_counter_timeout(int limit_ms, void* stream) { return selftest(1, limit_ms, stream); }

extern "C" int elbm_selftest_wait_timeout(int limit_ms, void* stream) { return selftest(0, limit_ms, stream); }
