// Allocation-free step entry point (elbm_step_noalloc, declared in include/elbm.h).
//
// For callers that cannot allocate device memory themselves: a host
// application that manages all device memory through its own pool, a plugin
// running inside a framework that forbids allocations on its worker threads,
// or code running at a point where cudaMalloc, which may synchronise the
// device, is not allowed.
// They pass their own population buffer; the only scratch the two-pass step
// needs -- the anomaly field, three floats per node -- lives in a file-scope
// device array of fixed size that every GPU loading this library holds until
// the process exits.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>

#include "step_kernels.cuh"

namespace {

constexpr int kNoallocMaxNodes = 1 << 18;  // 262144 nodes, e.g. 64^3 or 512^2
constexpr int kMaxDevices = 64;

// Anomaly field of the allocation-free step, shared by every call on a device.
static __device__ __align__(256) float g_noalloc_q[3 * kNoallocMaxNodes];

// Device address of g_noalloc_q, looked up once per device (the host-side
// symbol is only a stand-in and must never be passed to a kernel).  The
// address lives as long as the device's primary context: after a
// cudaDeviceReset it is stale, and this entry point must not be used on that
// device again in the same process.
float* g_q_addr[kMaxDevices] = {};
std::mutex g_q_lock;

int noalloc_fail(int code, const char* msg) { return elbm::set_error(code, msg); }

// Even-layout restore after an odd number of in-place steps: slot (opp(i), y)
// holds f_i(y + c_i) and slot (i, y + c_i) holds f_opp(i)(y), so swapping the
// two for every y and every i before the rest population puts each population
// back at its own node.
template <int D>
__global__ void __launch_bounds__(elbm::kBlock) k_aa_to_own(elbm::StepParams p)
{
    using namespace elbm;
    constexpr int Q = Lat<D>::Q;
    const int cell = blockIdx.x * kBlock + threadIdx.x;
    if (cell >= p.N) return;
    const Node n = make_node<D>(p, cell);
    float* f = static_cast<float*>(p.f);
#pragma unroll
    for (int i = 0; i < (Q - 1) / 2; ++i) {
        const int a = (Q - 1 - i) * p.N + cell;
        const int b = i * p.N + n.at(cx_of(i), cy_of(i), cz_of<D>(i));
        const float t = f[a];
        f[a] = f[b];
        f[b] = t;
    }
}

}  // namespace

extern "C" int elbm_step_noalloc(int lattice, int nx, int ny, int nz, const double* stretch, double T,
                                 double nu, float* f, int nsteps, void* stream)
{
    elbm::set_error(ELBM_OK, "");
    if (lattice != ELBM_D2Q9 && lattice != ELBM_D3Q27) return noalloc_fail(ELBM_ERR_ARG, "lattice must be 9 or 27");
    const int D = lattice == ELBM_D2Q9 ? 2 : 3;
    if (!f) return noalloc_fail(ELBM_ERR_ARG, "population buffer is NULL");
    if (nsteps < 0) return noalloc_fail(ELBM_ERR_ARG, "nsteps must be >= 0");
    if (nx < 3 || ny < 3 || (D == 2 && nz != 1) || (D == 3 && nz < 3))
        return noalloc_fail(ELBM_ERR_ARG, "need nx, ny >= 3 and nz == 1 (D2Q9) or nz >= 3 (D3Q27)");
    const long long N = (long long)nx * ny * nz;
    if (N > kNoallocMaxNodes)
        return noalloc_fail(ELBM_ERR_ARG, "grid larger than the 262144 nodes the allocation-free step supports");
    double lam[3] = {1.0, 1.0, 1.0};
    if (stretch)
        for (int a = 0; a < D; ++a) lam[a] = stretch[a];
    double lmin2 = 1e300;
    for (int a = 0; a < D; ++a) {
        if (!(lam[a] > 0.0) || !std::isfinite(lam[a])) return noalloc_fail(ELBM_ERR_ARG, "stretch must be finite and > 0");
        lmin2 = std::min(lmin2, lam[a] * lam[a]);
    }
    if (!(T > 0.0) || !std::isfinite(T)) return noalloc_fail(ELBM_ERR_ARG, "T must be finite and > 0");
    if (T >= lmin2) return noalloc_fail(ELBM_ERR_UNREALIZABLE, "T >= min lam^2: rest population not positive");
    if (!(nu > 0.0) || !std::isfinite(nu)) return noalloc_fail(ELBM_ERR_ARG, "nu must be finite and > 0");

    // An error still pending from the caller's earlier CUDA work is the
    // caller's: report it and leave it in place rather than clear it, so that
    // the error checks below see only this call's own launches.
    const cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess) {
        char msg[256];
        std::snprintf(msg, sizeof msg, "a CUDA error from earlier work is pending (left in place): %s",
                      cudaGetErrorString(pending));
        return noalloc_fail(ELBM_ERR_CUDA, msg);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return noalloc_fail(ELBM_ERR_CUDA, "no usable current device");
    float* q = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_q_lock);
        if (!g_q_addr[dev]) {
            float* ptr = nullptr;
            e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_q);
            if (e != cudaSuccess || !ptr) return noalloc_fail(ELBM_ERR_CUDA, "cudaGetSymbolAddress of the scratch failed");
            g_q_addr[dev] = ptr;
        }
        q = g_q_addr[dev];
    }

    // A solver description on the stack: FP32 unshifted storage, rest baseline.
    elbm::Solver s;
    s.lattice = lattice;
    s.D = D;
    s.Q = lattice;
    s.nx = nx;
    s.ny = ny;
    s.nz = nz;
    s.N = N;
    s.storage = ELBM_F32;
    for (int a = 0; a < 3; ++a) s.lam[a] = lam[a];
    s.T = T;
    s.nu = nu;
    s.omega = 1.0 / (nu / T + 0.5);  // Eq. nu with R = 1, delta t = 1
    s.stream = (cudaStream_t)stream;
    s.f = f;
    s.q = q;
    long long launches = 0;
    for (int k = 0; k < nsteps && e == cudaSuccess; ++k)
        e = (D == 2) ? elbm::step_two_pass_impl<2>(s, k & 1, &launches)
                     : elbm::step_two_pass_impl<3>(s, k & 1, &launches);
    if (e == cudaSuccess && (nsteps & 1)) {
        elbm::StepParams p;
        elbm::fill_params(s, p);
        const dim3 grid((unsigned)((N + elbm::kBlock - 1) / elbm::kBlock));
        if (D == 2) k_aa_to_own<2><<<grid, elbm::kBlock, 0, s.stream>>>(p);
        else k_aa_to_own<3><<<grid, elbm::kBlock, 0, s.stream>>>(p);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return noalloc_fail(ELBM_ERR_CUDA, cudaGetErrorString(e));
    return ELBM_OK;
}
