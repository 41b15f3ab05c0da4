// Batched form of the extended LBGK step: many grids of one lattice and one
// storage mode -- of any sizes, stretches, temperatures and viscosities --
// advance together, two launches per step for the whole batch.
//
// The batch keeps a device table of members.  A launch covers the blocks of
// every member back to back; a block belongs to exactly one member, copies that
// member's parameter block into shared memory and runs the per-node code of the
// two-pass form (anomaly pass, then collide pass), so every member's result is
// bit-identical to stepping it alone.  Each member keeps its own streaming
// parity: in step k of a launch sequence it is (parity_0 + k) mod 2.
#pragma once
#include "step_kernels.cuh"

namespace elbm {

// Member owning block b in a launch of block size BS: members are sorted by
// their first block.
template <int BS>
__device__ __forceinline__ int batch_member_of(const BatchMember* m, int nm, int b)
{
    int lo = 0, hi = nm - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (m[mid].block_begin[BS == 128 ? 0 : 1] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The owning member's parameter block, copied to shared memory; -1 for the
// blocks beyond the batch's current total (launches are sized for the
// batch's capacity, so that membership changes need no new launch sequence).
template <int BS>
__device__ __forceinline__ int batch_prologue(const BatchHeader* h, StepParams& sp, int& parity)
{
    if ((int)blockIdx.x >= h->blocks[BS == 128 ? 0 : 1]) return -1;
    const BatchMember* members = h->members;
    const int nm = h->count;
    __shared__ int s_member;
    if (threadIdx.x == 0) s_member = batch_member_of<BS>(members, nm, blockIdx.x);
    __syncthreads();
    const int k = s_member;
    const int words = (int)(sizeof(StepParams) / sizeof(int));
    for (int w = threadIdx.x; w < words; w += BS)
        reinterpret_cast<int*>(&sp)[w] = reinterpret_cast<const int*>(&members[k].p)[w];
    parity = members[k].parity;
    __syncthreads();
    return (blockIdx.x - members[k].block_begin[BS == 128 ? 0 : 1]) * BS + threadIdx.x;
}

template <int D, int ST, int BS>
__global__ void __launch_bounds__(BS) k_batch_anomaly(const BatchHeader* h, int step)
{
    __shared__ StepParams sp;
    int parity0;
    const int cell = batch_prologue<BS>(h, sp, parity0);
    if (cell < 0 || cell >= sp.N || sp.eq_mode != 0) return;
    const Node n = make_node<D>(sp, cell);
    float g[Lat<D>::Q];
    if (((parity0 + step) & 1) == 0) gather<D, ST, 0>(sp, n, g);
    else gather<D, ST, 1>(sp, n, g);
    float drho, j[3];
    moments<D>(sp, g, drho, j);
    const float inv_rho = 1.0f / (sp.rho_ref + drho);
#pragma unroll
    for (int a = 0; a < D; ++a) sp.q[a * sp.N + cell] = anomaly(sp, a, j[a], j[a] * inv_rho);
}

template <int D, int ST, int BS>
__global__ void __launch_bounds__(BS, 4 * kBlock / BS) k_batch_collide(const BatchHeader* h, int step)
{
    __shared__ StepParams sp;
    __shared__ unsigned stage[Lat<D>::Q * BS];
    int parity0;
    const int cell = batch_prologue<BS>(h, sp, parity0);
    if (cell < 0 || cell >= sp.N) return;
    if (((parity0 + step) & 1) == 0) collide_staged<D, ST, 0, BS>(sp, cell, stage + threadIdx.x);
    else collide_staged<D, ST, 1, BS>(sp, cell, stage + threadIdx.x);
}

// Enqueue `nsteps` batched steps on `stream`: for step k, the anomaly pass and
// the collide pass over every member (block size BS, grids of `blocks`
// blocks, at least the batch's current total).
template <int D>
cudaError_t batch_enqueue_impl(int storage, int block_size, const BatchHeader* h, int blocks, int nsteps,
                               cudaStream_t stream, long long* launches)
{
    for (int k = 0; k < nsteps; ++k) {
        ELBM_DISPATCH_STORAGE(storage, {
            if (block_size == 128) {
                k_batch_anomaly<D, ST, 128><<<blocks, 128, 0, stream>>>(h, k);
                k_batch_collide<D, ST, 128><<<blocks, 128, 0, stream>>>(h, k);
            } else {
                k_batch_anomaly<D, ST, 256><<<blocks, 256, 0, stream>>>(h, k);
                k_batch_collide<D, ST, 256><<<blocks, 256, 0, stream>>>(h, k);
            }
        });
        *launches += 2;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace elbm
