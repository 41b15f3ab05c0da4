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

// One member as the kernels read it.  params[a] is the member's parameter
// block with array a as the source (params[a].f = array a); maps16[a] and
// maps8[a] are the tensor maps of array a (tile box of 16 or 8 rows, ring-row
// box) for the TMEM and the TMA kernel (each encoded where the grid's rows
// allow that tile height).  Before step 0 of a launch sequence the member's
// state sits in array `phase`; step k reads array (phase + k) & 1 and writes
// the other.
struct alignas(128) SpMember {
    CUtensorMap maps16[2][2];
    CUtensorMap maps8[2][2];
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
        tensormap_acquire(&m->maps16[a][0]);
        tensormap_acquire(&m->maps16[a][1]);
    }
    __syncthreads();
    tmem_tile_step<ST, BC, FX>(&m->maps16[a][0], &m->maps16[a][1], sp, m->params[a ^ 1].f, w.y, w.z, w.w & 0xffff,
                               w.w >> 16, smem_raw);
}

// The same over 32 x 8 tile columns with the TMA kernel's tile body
// (periodic, unforced members; two blocks per SM).
template <int ST>
__global__ void __launch_bounds__(kTmaThreads, 2)
    k_single_pass_tma_batch(const SpMember* __restrict__ members, const int4* __restrict__ work, int step)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) StepParams sp;
    const int4 w = work[blockIdx.x];
    const SpMember* m = members + w.x;
    const int a = (m->phase + step) & 1;
    const unsigned* src = reinterpret_cast<const unsigned*>(&m->params[a]);
    unsigned* dstw = reinterpret_cast<unsigned*>(&sp);
    for (int k = threadIdx.x; k < (int)(sizeof(StepParams) / 4); k += kTmaThreads) dstw[k] = src[k];
    if (threadIdx.x == kBlock) {  // lane 0 of the producer warp issues every TMA load of the block
        tensormap_acquire(&m->maps8[a][0]);
        tensormap_acquire(&m->maps8[a][1]);
    }
    __syncthreads();
    tma_tile_step<ST>(&m->maps8[a][0], &m->maps8[a][1], sp, m->params[a ^ 1].f, w.y, w.z, w.w & 0xffff, w.w >> 16,
                      smem_raw);
}

template <int ST>
cudaError_t sp_batch_launch_tma(const SpMember* members, const int4* work, int nwork, int nsteps, cudaStream_t st)
{
    const int smem = TmaLayout<ST>::bytes;
    cudaError_t e = set_smem_limit_once<k_single_pass_tma_batch<ST>>(smem);
    for (int k = 0; k < nsteps && e == cudaSuccess; ++k) {
        k_single_pass_tma_batch<ST><<<nwork, kTmaThreads, smem, st>>>(members, work, k);
        e = cudaGetLastError();
    }
    return e;
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

// Whether the flattened TMA (32 x 8) batch kernel takes solver s: the TMA
// kernel's geometry, periodic and unforced.
bool sp_tma_member(const Solver& s)
{
    const bool bounded = s.walls_y || s.g[0] != 0.0 || s.g[1] != 0.0 || s.g[2] != 0.0;
    return s.D == 3 && !bounded && s.nx % kTileX == 0 && s.ny % kTileY == 0 &&
           (s.nx * (int)storage_bytes(s.storage)) % 16 == 0;
}

// Fill the member record of solver s (host memory, sp_member_bytes() bytes)
// with s->f as array 0 and s->f2 as array 1 (phase 0); encode_maps = false
// keeps the tensor maps already in the record (same arrays).
cudaError_t sp_member_fill(const Solver& s, void* record, bool encode_maps)
{
    SpMember* m = static_cast<SpMember*>(record);
    const bool tmem = single_tmem_geometry(s), tma = sp_tma_member(s);
    if ((!tmem && !tma) || !s.f || !s.f2) return cudaErrorInvalidValue;
    for (int a = 0; a < 2; ++a) {
        void* arr = a == 0 ? s.f : s.f2;
        fill_params(s, m->params[a]);
        m->params[a].f = arr;
        m->params[a].parity = 0;
        if (encode_maps) {
            cudaError_t e = cudaSuccess;
            if (tmem) e = encode_population_maps(s, arr, kTmTileY, &m->maps16[a][0], &m->maps16[a][1]);
            if (e == cudaSuccess && tma) e = encode_population_maps(s, arr, kTileY, &m->maps8[a][0], &m->maps8[a][1]);
            if (e != cudaSuccess) return e;
        }
    }
    m->phase = 0;
    return cudaSuccess;
}

void sp_member_set_phase(void* record, int phase) { static_cast<SpMember*>(record)->phase = phase; }

// tile_y 16: the TMEM kernel, bc: some member has walls or a body force, fx:
// no member's force has a y or z component (the lighter force increment);
// tile_y 8: the TMA kernel (periodic, unforced members only).
cudaError_t sp_batch_enqueue(int storage, int tile_y, bool bc, bool fx, const void* members, const void* work,
                             int nwork, int nsteps, cudaStream_t st, long long* launches)
{
    if (nwork <= 0 || nsteps <= 0) return cudaSuccess;
    const SpMember* m = static_cast<const SpMember*>(members);
    const int4* w = static_cast<const int4*>(work);
    cudaError_t e = cudaSuccess;
    ELBM_DISPATCH_STORAGE(storage, {
        e = tile_y == kTileY ? sp_batch_launch_tma<ST>(m, w, nwork, nsteps, st)
            : !bc            ? sp_batch_launch<ST, false, false>(m, w, nwork, nsteps, st)
            : fx             ? sp_batch_launch<ST, true, true>(m, w, nwork, nsteps, st)
                             : sp_batch_launch<ST, true, false>(m, w, nwork, nsteps, st);
    });
    if (e == cudaSuccess) *launches += nsteps;
    return e;
}

}  // namespace elbm
