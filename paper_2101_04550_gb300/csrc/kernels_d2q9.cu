// Instantiation of the step kernels and their launchers for the D2Q9 lattice.
#include "step_kernels.cuh"
#include "single_pass_d2q9.cuh"
#include "graph_step.cuh"
#include "batch.cuh"

namespace elbm {
template cudaError_t step_two_pass_impl<2>(const Solver&, int, long long*);
// the single pass of the D2Q9 lattice (single_pass_d2q9.cuh)
template <>
cudaError_t step_single_impl<2>(const Solver& s, void* dst, long long* launches)
{
    return step_single_d2q9(s, dst, launches);
}
template cudaError_t build_step_graph_impl<2>(const Solver&, int, cudaGraphExec_t*, int*);
template cudaError_t batch_enqueue_impl<2>(int, int, int, int, const void*, int, cudaStream_t, long long*);
template cudaError_t init_impl<2>(const Solver&, const void*, const void*, int, long long*);
template cudaError_t moments_impl<2>(const Solver&, void*, void*, int, long long*);
template cudaError_t get_populations_impl<2>(const Solver&, void*, int, long long*);
template cudaError_t set_populations_impl<2>(const Solver&, const void*, int, long long*);
template cudaError_t reduce_impl<2>(const Solver&, long long*);
template cudaError_t mode_sums_impl<2>(const Solver&, const double*, const double*, long long*);
template cudaError_t field_sums_impl<2>(const Solver&, const void*, const void*, int, long long*);
}  // namespace elbm
