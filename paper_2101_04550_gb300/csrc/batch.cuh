// Batched form of the extended LBGK step: many grids of one lattice and one
// storage mode -- of any sizes, stretches, temperatures and viscosities --
// advance together, two launches per step for the whole batch.
//
// The batch keeps a table of members in constant memory.  A launch covers the
// blocks of every member back to back; a block belongs to exactly one member,
// reads that member's parameter block from the constant table and runs the
// per-node code of the two-pass form (anomaly pass, then collide pass), so
// every member's result is bit-identical to stepping it alone.  Each member keeps its own streaming
// parity: in step k of a launch sequence it is (parity_0 + k) mod 2.
#pragma once
#include "step_kernels.cuh"

namespace elbm {

// Member tables, one per storage mode, in constant memory: the kernels read a
// member's parameters as constant-bank operands, as the single-grid kernels
// do.  The batch uploads its table before each launch sequence; one live
// batch per (lattice, storage) kind uses a table at a time.
__constant__ BatchMember c_batch_f32[kBatchMax];
__constant__ BatchMember c_batch_f32s[kBatchMax];
__constant__ BatchMember c_batch_f16[kBatchMax];
__constant__ BatchMember c_batch_bf16[kBatchMax];
__constant__ int c_batch_count[4];

template <int ST>
__device__ __forceinline__ const BatchMember* batch_table()
{
    if (ST == ELBM_F32) return c_batch_f32;
    if (ST == ELBM_F32_SHIFT) return c_batch_f32s;
    if (ST == ELBM_F16_SHIFT) return c_batch_f16;
    return c_batch_bf16;
}

// Member owning block b in a launch of block size BS: members are sorted by
// their first block.
template <int ST, int BS>
__device__ __forceinline__ int batch_member_of(int b)
{
    const BatchMember* m = batch_table<ST>();
    int lo = 0, hi = c_batch_count[ST] - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (m[mid].block_begin[BS == 128 ? 0 : 1] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int D, int ST, int BS>
__global__ void __launch_bounds__(BS) k_batch_anomaly(int step)
{
    __shared__ int s_member;
    if (threadIdx.x == 0) s_member = batch_member_of<ST, BS>(blockIdx.x);
    __syncthreads();
    const BatchMember& m = batch_table<ST>()[s_member];
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
__global__ void __launch_bounds__(BS, 4 * kBlock / BS) k_batch_collide(int step)
{
    __shared__ int s_member;
    __shared__ unsigned stage[Lat<D>::Q * BS];
    if (threadIdx.x == 0) s_member = batch_member_of<ST, BS>(blockIdx.x);
    __syncthreads();
    const BatchMember& m = batch_table<ST>()[s_member];
    const int cell = (blockIdx.x - m.block_begin[BS == 128 ? 0 : 1]) * BS + threadIdx.x;
    if (cell >= m.p.N) return;
    if (((m.parity + step) & 1) == 0) collide_staged<D, ST, 0, BS>(m.p, cell, stage + threadIdx.x);
    else collide_staged<D, ST, 1, BS>(m.p, cell, stage + threadIdx.x);
}

// Copy a member table (and its count) into the constant table of `storage`.
template <int D>
cudaError_t batch_upload_impl(int storage, const BatchMember* table, int n, cudaStream_t stream)
{
    if (n > kBatchMax) return cudaErrorInvalidValue;
    const void* sym = storage == ELBM_F32 ? (const void*)&c_batch_f32
                    : storage == ELBM_F32_SHIFT ? (const void*)&c_batch_f32s
                    : storage == ELBM_F16_SHIFT ? (const void*)&c_batch_f16 : (const void*)&c_batch_bf16;
    cudaError_t e = cudaMemcpyToSymbolAsync(sym, table, n * sizeof(BatchMember), 0, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyToSymbolAsync(c_batch_count, &n, sizeof(int), storage * sizeof(int), cudaMemcpyHostToDevice, stream);
    return e;
}

// Enqueue `nsteps` batched steps on `stream`: for step k, the anomaly pass and
// the collide pass over every member, `blocks` blocks of block_size threads.
template <int D>
cudaError_t batch_enqueue_impl(int storage, int block_size, int blocks, int nsteps, cudaStream_t stream,
                               long long* launches)
{
    for (int k = 0; k < nsteps; ++k) {
        ELBM_DISPATCH_STORAGE(storage, {
            if (block_size == 128) {
                k_batch_anomaly<D, ST, 128><<<blocks, 128, 0, stream>>>(k);
                k_batch_collide<D, ST, 128><<<blocks, 128, 0, stream>>>(k);
            } else {
                k_batch_anomaly<D, ST, 256><<<blocks, 256, 0, stream>>>(k);
                k_batch_collide<D, ST, 256><<<blocks, 256, 0, stream>>>(k);
            }
        });
        *launches += 2;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace elbm
