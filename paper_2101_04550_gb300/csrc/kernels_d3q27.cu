// Instantiation of the step kernels and their launchers for the D3Q27 lattice.
#include "step_kernels.cuh"
#include "single_pass_tmem.cuh"
#include "graph_step.cuh"
#include "batch.cuh"

namespace elbm {
template cudaError_t step_two_pass_impl<3>(const Solver&, int, long long*);
template cudaError_t step_single_impl<3>(const Solver&, void*, long long*);
template cudaError_t build_step_graph_impl<3>(const Solver&, int, cudaGraphExec_t*, int*);
template cudaError_t batch_enqueue_impl<3>(int, int, int, int, cudaStream_t, long long*);
template cudaError_t batch_upload_impl<3>(int, const BatchMember*, int, cudaStream_t);
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
}  // namespace elbm
