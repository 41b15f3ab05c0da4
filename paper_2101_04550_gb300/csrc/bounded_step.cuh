// The in-place two-pass step with walls and body force (the turbulent channel
// setup of Sec. III.E): half-way bounce-back below y = 0 and above y = ny-1,
// the anomaly's ghost value beyond a wall in the central difference of
// Eq. Paastar1, and the exact-difference body-force increment.  The same
// kernels as the periodic step, instantiated with BC = true, which reads the
// wall and force switches from the parameter block; kept in their own
// translation units so that the periodic kernels compile without them.
#pragma once
#include "step_kernels.cuh"

namespace elbm {

template <int D>
cudaError_t step_bounded_impl(const Solver& s, int parity, long long* launches)
{
    StepParams p;
    fill_params(s, p);
    p.parity = parity;
    const dim3 grid((unsigned)((s.N + kBlock - 1) / kBlock));
    ELBM_DISPATCH_STORAGE(s.storage, {
        if (p.eq_mode == 2) {
            if (parity == 0) k_collide<D, ST, 0, true, true><<<grid, kBlock, 0, s.stream>>>(p);
            else k_collide<D, ST, 1, true, true><<<grid, kBlock, 0, s.stream>>>(p);
        } else if (parity == 0) {
            if (p.eq_mode == 0) { k_anomaly<D, ST, 0, true><<<grid, kBlock, 0, s.stream>>>(p); ++*launches; }
            k_collide<D, ST, 0, false, true><<<grid, kBlock, 0, s.stream>>>(p);
        } else {
            if (p.eq_mode == 0) { k_anomaly<D, ST, 1, true><<<grid, kBlock, 0, s.stream>>>(p); ++*launches; }
            k_collide<D, ST, 1, false, true><<<grid, kBlock, 0, s.stream>>>(p);
        }
        ++*launches;
    });
    return cudaGetLastError();
}

}  // namespace elbm
