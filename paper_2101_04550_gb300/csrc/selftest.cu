// Self-test of the device-side failure detection: one block whose threads
// wait, with a short bound, on an mbarrier phase that nothing completes --
// the same bounded wait (bounded_wait) that the TMA-fed single-pass kernels
// use.  The wait must give up, report ELBM_ERR_TIMEOUT through the status
// word, and leave the context usable.
#include <cstdio>

#include "single_pass_tma.cuh"

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

}  // namespace

extern "C" int elbm_selftest_wait_timeout(int limit_ms, void* stream)
{
    elbm::set_error(ELBM_OK, "");
    if (limit_ms < 1 || limit_ms > 2000) return elbm::set_error(ELBM_ERR_ARG, "limit_ms must be in 1..2000");
    (void)cudaGetLastError();  // a stale error of an earlier call is not this call's
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* status = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&status, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        k_selftest_wait<<<1, 32, 0, st>>>(status, 1000000ull * (unsigned long long)limit_ms);
        e = cudaGetLastError();
    }
    int host = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (status) cudaFreeAsync(status, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return elbm::set_error(ELBM_ERR_CUDA, cudaGetErrorString(e));
    if (host == ELBM_ERR_TIMEOUT) return elbm::set_error(ELBM_ERR_TIMEOUT, "the bounded wait gave up as designed");
    char msg[96];
    std::snprintf(msg, sizeof msg, "the bounded wait did not report a timeout (status %d)", host);
    return elbm::set_error(ELBM_ERR_STATE, msg);
}
