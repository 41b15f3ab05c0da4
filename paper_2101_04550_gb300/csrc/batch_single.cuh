// Flattened single-pass batch: one launch per step advances every member of
// a batch whose grids the TMEM single pass takes (x a multiple of 32 nodes,
// y of 16), whatever their sizes and parameters.
//
// The launch's blocks walk a work list of (member, tile column, z range)
// items kept in device memory.  A block copies its member's parameter block
// (the StepParams of the solo kernel, for the member's current source array)
// from the member table into shared memory and runs the tile body of the solo
// kernel (tmem_tile_step) with the member's tensor maps, which also live in
// the table.  The per-node arithmetic is the solo kernel's, so every member's
// result is bit-identical to stepping it alone; the tile and the segment of
// planes a block takes only decide which block computes which node and which
// ring anomaly it recomputes, and the anomaly of a node is the same function
// of its populations wherever it is computed.
#pragma once
#include "single_pass_tmem.cuh"

namespace elbm {

// One member as the kernel reads it.  params[a] is the member's parameter
// block with array a as the source (params[a].f = array a); maps[a] are the
// tensor maps of array a (tile box, ring-row box).  Before step 0 of a launch
// sequence the member's state sits in array `phase`; step k reads array
// (phase + k) & 1 and writes the other.
struct alignas(128) SpMember {
    CUtensorMap maps[2][2];
    StepParams params[2];
    int phase;
};
static_assert(sizeof(SpMember) % 128 == 0, "member records keep the tensor maps 64-byte aligned");

// Make the tensor map at `map` (device memory written before this launch)
// visible to the tensor-map proxy of the calling thread.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* map)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
                 : "memory");
}

// Work item: x = member, y = x0, z = y0, w = z0 | (z1 << 16).
template <int ST, bool BC, bool FX>
__global__ void __launch_bounds__(kTmThreads, 1)
    k_single_pass_tmem_batch(const SpMember* __restrict__ members, const int4* __restrict__ work, int step)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) StepParams sp;
    const int4 w = work[blockIdx.x];
    const SpMember* m = members + w.x;
    const int a = (m->phase + step) & 1;
    const unsigned* src = reinterpret_cast<const unsigned*>(&m->params[a]);
    unsigned* dstw = reinterpret_cast<unsigned*>(&sp);
    for (int k = threadIdx.x; k < (int)(sizeof(StepParams) / 4); k += kTmThreads) dstw[k] = src[k];
    if (threadIdx.x == kTmConsumers) {  // lane 0 of the loading warp issues every TMA load of the block
        tensormap_acquire(&m->maps[a][0]);
        tensormap_acquire(&m->maps[a][1]);
    }
    __syncthreads();
    tmem_tile_step<ST, BC, FX>(&m->maps[a][0], &m->maps[a][1], sp, m->params[a ^ 1].f, w.y, w.z, w.w & 0xffff,
                               w.w >> 16, smem_raw);
}

template <int ST, bool BC, bool FX>
cudaError_t sp_batch_launch(const SpMember* members, const int4* work, int nwork, int nsteps, cudaStream_t st)
{
    const int smem = TmemLayout<ST>::bytes;
    cudaError_t e = set_smem_limit_once<k_single_pass_tmem_batch<ST, BC, FX>>(smem);
    for (int k = 0; k < nsteps && e == cudaSuccess; ++k) {
        k_single_pass_tmem_batch<ST, BC, FX><<<nwork, kTmThreads, smem, st>>>(members, work, k);
        e = cudaGetLastError();
    }
    return e;
}

size_t sp_member_bytes() { return sizeof(SpMember); }

// Fill the member record of solver s (host memory, sp_member_bytes() bytes)
// with s->f as array 0 and s->f2 as array 1 (phase 0); encode_maps = false
// keeps the tensor maps already in the record (same arrays).
cudaError_t sp_member_fill(const Solver& s, void* record, bool encode_maps)
{
    SpMember* m = static_cast<SpMember*>(record);
    if (!single_tmem_geometry(s) || !s.f || !s.f2) return cudaErrorInvalidValue;
    for (int a = 0; a < 2; ++a) {
        void* arr = a == 0 ? s.f : s.f2;
        fill_params(s, m->params[a]);
        m->params[a].f = arr;
        m->params[a].parity = 0;
        if (encode_maps) {
            const cudaError_t e = encode_population_maps(s, arr, kTmTileY, &m->maps[a][0], &m->maps[a][1]);
            if (e != cudaSuccess) return e;
        }
    }
    m->phase = 0;
    return cudaSuccess;
}

void sp_member_set_phase(void* record, int phase) { static_cast<SpMember*>(record)->phase = phase; }

// bc: some member has walls or a body force; fx: no member's force has a y
// or z component (the lighter force increment).
cudaError_t sp_batch_enqueue(int storage, bool bc, bool fx, const void* members, const void* work, int nwork,
                             int nsteps, cudaStream_t st, long long* launches)
{
    if (nwork <= 0 || nsteps <= 0) return cudaSuccess;
    const SpMember* m = static_cast<const SpMember*>(members);
    const int4* w = static_cast<const int4*>(work);
    cudaError_t e = cudaSuccess;
    ELBM_DISPATCH_STORAGE(storage, {
        e = !bc ? sp_batch_launch<ST, false, false>(m, w, nwork, nsteps, st)
            : fx ? sp_batch_launch<ST, true, true>(m, w, nwork, nsteps, st)
                 : sp_batch_launch<ST, true, false>(m, w, nwork, nsteps, st);
    });
    if (e == cudaSuccess) *launches += nsteps;
    return e;
}

}  // namespace elbm
