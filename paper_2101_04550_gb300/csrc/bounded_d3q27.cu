// Instantiation of the step with walls and body force for the D3Q27 lattice.
#include "bounded_step.cuh"

namespace elbm {
template cudaError_t step_bounded_impl<3>(const Solver&, int, long long*);
}  // namespace elbm
