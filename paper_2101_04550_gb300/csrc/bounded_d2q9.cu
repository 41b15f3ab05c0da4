// Instantiation of the step with walls and body force for the D2Q9 lattice.
#include "bounded_step.cuh"

namespace elbm {
template cudaError_t step_bounded_impl<2>(const Solver&, int, long long*);
}  // namespace elbm
