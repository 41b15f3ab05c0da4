// Batched form of the extended LBGK step: many grids of one lattice and one
// storage mode -- of any sizes, stretches, temperatures and viscosities --
// advance together, two launches per step for the whole batch.
//
// The batch keeps a table of its members in device memory of its own.  A
// launch covers the blocks of every member back to back; a block belongs to
// exactly one member, copies that member's record (parameter block, first
// blocks, parity) from the table into shared memory and runs the per-node
// code of the two-pass form (anomaly pass, then collide pass) on it, so every
// member's result is bit-identical to stepping it alone.  Each member keeps
// its own streaming parity: in step k of a launch sequence it is
// (parity_0 + k) mod 2.
#pragma once
#include "step_kernels.cuh"

namespace elbm {

// Member owning block b in a launch of block size BS: members are sorted by
// their first block.
template <int BS>
__device__ __forceinline__ int batch_member_of(const BatchMember* table, int count, int b)
{
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (table[mid].block_begin[BS == 128 ? 0 : 1] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The record of the member owning this block, copied into shared memory `rec`
// (every thread of the block takes part; ends with a block barrier).
template <int BS>
__device__ __forceinline__ void load_member(const BatchMember* table, int count, BatchMember& rec)
{
    __shared__ int s_member;
    if (threadIdx.x == 0) s_member = batch_member_of<BS>(table, count, blockIdx.x);
    __syncthreads();
    const unsigned* src = reinterpret_cast<const unsigned*>(table + s_member);
    unsigned* dst = reinterpret_cast<unsigned*>(&rec);
    for (int k = threadIdx.x; k < (int)(sizeof(BatchMember) / 4); k += BS) dst[k] = src[k];
    __syncthreads();
}

template <int D, int ST, int BS>
__global__ void __launch_bounds__(BS) k_batch_anomaly(const BatchMember* __restrict__ table, int count, int step)
{
    __shared__ __align__(16) BatchMember m;
    load_member<BS>(table, count, m);
    const StepParams& sp = m.p;
    const int cell = (blockIdx.x - m.block_begin[BS == 128 ? 0 : 1]) * BS + threadIdx.x;
    if (cell >= sp.N || sp.eq_mode != 0) return;
    const Node n = make_node<D>(sp, cell);
    float g[Lat<D>::Q];
    if (((m.parity + step) & 1) == 0) gather<D, ST, 0>(sp, n, g);
    else gather<D, ST, 1>(sp, n, g);
    float drho, j[3];
    moments<D>(sp, g, drho, j);
    const float inv_rho = 1.0f / (sp.rho_ref + drho);
#pragma unroll
    for (int a = 0; a < D; ++a) sp.q[a * sp.N + cell] = anomaly(sp, a, j[a], j[a] * inv_rho);
}

template <int D, int ST, int BS>
__global__ void __launch_bounds__(BS, 4 * kBlock / BS) k_batch_collide(const BatchMember* __restrict__ table, int count,
                                                                       int step)
{
    __shared__ __align__(16) BatchMember m;
    __shared__ unsigned stage[Lat<D>::Q * BS];
    load_member<BS>(table, count, m);
    const int cell = (blockIdx.x - m.block_begin[BS == 128 ? 0 : 1]) * BS + threadIdx.x;
    if (cell >= m.p.N) return;
    if (((m.parity + step) & 1) == 0) collide_staged<D, ST, 0, BS>(m.p, cell, stage + threadIdx.x);
    else collide_staged<D, ST, 1, BS>(m.p, cell, stage + threadIdx.x);
}

// Enqueue `nsteps` batched steps on `stream`: for step k, the anomaly pass and
// the collide pass over every member of the device table `table` (count
// members), `blocks` blocks of block_size threads.
template <int D>
cudaError_t batch_enqueue_impl(int storage, int block_size, int blocks, int nsteps, const void* table, int count,
                               cudaStream_t stream, long long* launches)
{
    const BatchMember* t = static_cast<const BatchMember*>(table);
    for (int k = 0; k < nsteps; ++k) {
        ELBM_DISPATCH_STORAGE(storage, {
            if (block_size == 128) {
                k_batch_anomaly<D, ST, 128><<<blocks, 128, 0, stream>>>(t, count, k);
                k_batch_collide<D, ST, 128><<<blocks, 128, 0, stream>>>(t, count, k);
            } else {
                k_batch_anomaly<D, ST, 256><<<blocks, 256, 0, stream>>>(t, count, k);
                k_batch_collide<D, ST, 256><<<blocks, 256, 0, stream>>>(t, count, k);
            }
        });
        *launches += 2;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace elbm
