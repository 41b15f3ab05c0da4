// Instantiation of the step kernels and their launchers for the D3Q27 lattice.
#include "step_kernels.cuh"
#include "single_pass_tmem.cuh"
#include "graph_step.cuh"
#include "batch.cuh"
#include "batch_single.cuh"
#include "fused_aa.cuh"

namespace elbm {
template cudaError_t step_two_pass_impl<3>(const Solver&, int, long long*);
template cudaError_t step_single_impl<3>(const Solver&, void*, long long*);
template cudaError_t build_step_graph_impl<3>(const Solver&, int, cudaGraphExec_t*, int*);
template cudaError_t batch_enqueue_impl<3>(int, int, int, int, const void*, int, cudaStream_t, long long*);
template cudaError_t init_impl<3>(const Solver&, const void*, const void*, int, long long*);
template cudaError_t moments_impl<3>(const Solver&, void*, void*, int, long long*);
template cudaError_t get_populations_impl<3>(const Solver&, void*, int, long long*);
template cudaError_t set_populations_impl<3>(const Solver&, const void*, int, long long*);
template cudaError_t reduce_impl<3>(const Solver&, long long*);
template cudaError_t mode_sums_impl<3>(const Solver&, const double*, const double*, long long*);
template cudaError_t field_sums_impl<3>(const Solver&, const void*, const void*, int, long long*);
// Geometry the TMEM single pass takes (the arrays' 16-byte alignment aside).
bool single_tmem_geometry(const Solver& s)
{
    return s.D == 3 && s.nx % kTileX == 0 && s.ny % kTmTileY == 0 && (s.nx * (int)storage_bytes(s.storage)) % 16 == 0;
}
// The fused in-place form (fused_aa.cuh): whether it takes s (D3Q27,
// periodic, unforced, extended or product-form equilibrium, every tile column
// co-resident), and one step of it at AA parity `parity`.
bool fused_available(const Solver& s)
{
    const bool bounded = s.walls_y || s.g[0] != 0.0 || s.g[1] != 0.0 || s.g[2] != 0.0;
    if (s.D != 3 || bounded || s.eq_mode == 2) return false;
    int bx = 0, by = 0;
    bool ok = false;
    ELBM_DISPATCH_STORAGE(s.storage, { ok = fused_fits<ST>(s, &bx, &by); });
    return ok;
}

cudaError_t step_fused_impl(const Solver& s, int parity, unsigned long long* progress, unsigned long long epoch,
                            long long* launches)
{
    StepParams p;
    fill_params(s, p);
    p.parity = parity;
    const dim3 grid((unsigned)((s.nx + kFuTileX - 1) / kFuTileX), (unsigned)((s.ny + kFuTileY - 1) / kFuTileY));
    void* args[] = {&p, &progress, &epoch};
    cudaError_t e = cudaSuccess;
    ELBM_DISPATCH_STORAGE(s.storage, {
        const void* fn = parity == 0 ? (const void*)k_fused_aa<ST, 0> : (const void*)k_fused_aa<ST, 1>;
        e = cudaLaunchCooperativeKernel(fn, grid, dim3(kFuBlock), args, kFuSmemBytes, s.stream);
    });
    if (e == cudaSuccess) ++*launches;
    return e;
}

// Single-pass kernel a step of s launches (the arrays are 16-byte aligned, as
// the stream-ordered allocator returns them): 1 TMEM (32 x 16 tiles), 2 TMA
// (32 x 8 tiles), 3 cp.async-staged; 4 the D2Q9 row march.  Walls and the
// body force run in the TMEM kernel only.
int single_pass_variant(const Solver& s)
{
    if (s.D == 2) return 4;
    if (single_tmem_geometry(s)) return 1;
    const bool fast = s.nx % kTileX == 0 && s.ny % kTileY == 0 && (s.nx * (int)storage_bytes(s.storage)) % 16 == 0;
    return fast ? 2 : 3;
}
}  // namespace elbm
