// Persistent, in-place (AA) pipelined form of the extended LBGK step.
//
// The correction term needs the anomaly Q~_aaa of the neighbours at the same
// time level (Eq. Paastar1), i.e. post-streaming moments of nodes whose
// population slots other thread blocks overwrite when they collide.  The
// two-pass form separates the passes by a kernel boundary and so reads the
// populations twice from HBM.  Here the grid is cut along its slowest axis
// (z for D3Q27, y for D2Q9) into chunks, and every chunk has an anomaly phase
// A(c) (read populations, write q) and a collide phase C(c) (re-read
// populations, read q of chunks c-1..c+1, relax, write populations in place).
// Phases are issued in the order
//     A(K-1), A(0), ..., A(L), C(0), A(L+1), C(1), A(L+2), ...
// so that A(c) runs L chunks ahead of C(c) and the re-read of chunk c hits L2.
//
// One launch advances one time step.  Work is split into warp-sized tiles,
// numbered in phase order.  A collide tile of chunk c waits (bounded) for the
// anomaly phases of chunks c-1, c and c+1 to be complete; with the phase order
// above those tiles have smaller numbers.  This covers every hazard of the
// in-place slots and of the q field: the anomaly phase of c reads the slot set
// of c before the collide phase of c rewrites it, slot sets of distinct nodes
// are disjoint, and q of chunks c-1..c+1 is complete before C(c) reads it.
// The kernel boundary orders consecutive steps.  Every wait is bounded by a
// wall-clock limit after which the kernel records ELBM_ERR_TIMEOUT in the
// status word and all warps return.
#pragma once
#include <algorithm>

#include "step_kernels.cuh"

namespace elbm {

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s per wait

// Resident blocks per SM the pipelined kernel is compiled for (register cap
// 65536 / (256 * ELBM_PIPE_MIN_BLOCKS)).
#ifndef ELBM_PIPE_MIN_BLOCKS
#define ELBM_PIPE_MIN_BLOCKS ELBM_COLLIDE_MIN_BLOCKS
#endif
// Nodes per lane in one (warp-sized) tile of the pipelined kernel.
#ifndef ELBM_PIPE_TILE_CPT
#define ELBM_PIPE_TILE_CPT 8
#endif

// Layout of the sync words (the first 2 + 2K are reset by the host before
// every launch): [0] unused, [1] abort flag, [2 .. 2+K) anomaly-phase
// completions per chunk, [2+K .. 2+2K) unused, then 2 words per phase of the
// step: (type, chunk).
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void fence_acquire() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Bounded wait until the three counters a, b, c are all >= target; the three
// loads are issued together and one fence then orders the block's later reads
// after the producers' releases.  False if it gave up (timeout or abort).
__device__ __forceinline__ bool wait3_ge(const StepParams& p, const unsigned* a, const unsigned* b,
                                         const unsigned* c, unsigned target)
{
    unsigned long long t0 = 0;
    volatile unsigned* abort_flag = p.sync + 1;
    for (int it = 0;; ++it) {
        const unsigned va = ld_relaxed(a), vb = ld_relaxed(b), vc = ld_relaxed(c);
        if (va >= target && vb >= target && vc >= target) {
            fence_acquire();
            return true;
        }
        if (it == 0) t0 = globaltimer();
        else if (*abort_flag) return false;
        if (globaltimer() - t0 > kWaitLimitNs) {
            atomicExch(p.sync + 1, 1u);
            atomicCAS(p.status, 0, ELBM_ERR_TIMEOUT);
            return false;
        }
        __nanosleep(32);
    }
}

// One time step (streaming parity PAR) over the whole grid.  Every warp is an
// independent worker with a static share of the tiles: warp w of W processes
// tiles w, w + W, w + 2W, ... in issue order.  Lane 0 waits for a tile's
// dependencies; after __syncwarp() it publishes the tile's completion with a
// release add.  No block-wide barrier and no ticket atomic is needed.  The
// kernel is launched cooperatively, so all W warps are resident; the warp that
// owns the oldest unfinished tile has finished all its earlier tiles and that
// tile only waits for older ones, so it never waits and the step completes.
template <int D, int ST, int PAR>
__global__ void __launch_bounds__(kBlock, ELBM_PIPE_MIN_BLOCKS) k_pipelined(StepParams p)
{
    __shared__ unsigned stage[Lat<D>::Q * kBlock];
    const int lane = threadIdx.x & 31;
    const int K = p.nchunks, T = p.tiles_per_chunk;
    unsigned* done_a = p.sync + 2;
    const unsigned* order = p.sync + 2 + 2 * K;
    const int layer = (D == 3) ? p.plane : p.nx;
    const int chunk_cells = p.chunk_planes * layer;
    const int total = 2 * K * T;
    const int W = gridDim.x * (kBlock / 32);

    for (int t = blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5); t < total; t += W) {
        const int tile = t % T;
        const int ph = t / T;
        const int type = (int)order[2 * ph];  // 0 anomaly phase, 1 collide phase
        const int c = (int)order[2 * ph + 1];
        if (type == 1) {
            int ok = 1;
            if (lane == 0) {
                const int cm = (c == 0) ? K - 1 : c - 1, cp = (c == K - 1) ? 0 : c + 1;
                ok = wait3_ge(p, done_a + cm, done_a + c, done_a + cp, (unsigned)T);
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            __syncwarp();  // the other lanes' reads are ordered after lane 0's acquire
        }

        const int c_begin = c * chunk_cells;
        const int c_end = min(p.N, c_begin + chunk_cells);
        const int t_begin = c_begin + tile * p.tile_cells;
        const int t_end = min(c_end, t_begin + p.tile_cells);
        if (type == 0) {
#pragma unroll 1
            for (int cell = t_begin + lane; cell < t_end; cell += 32) {
                const Node n = make_node<D>(p, cell);
                float g[Lat<D>::Q];
                gather<D, ST, PAR>(p, n, g);
                float drho, j[3];
                moments<D>(p, g, drho, j);
                const float inv_rho = 1.0f / (p.rho_ref + drho);
#pragma unroll
                for (int a = 0; a < D; ++a) p.q[a * p.N + cell] = anomaly(p, a, j[a], j[a] * inv_rho);
            }
        } else {
#pragma unroll 1
            for (int cell = t_begin + lane; cell < t_end; cell += 32)
                collide_staged<D, ST, PAR>(p, cell, stage + threadIdx.x);
        }
        if (type == 0) {  // collide completions are not waited on within a step
            __syncwarp();
            if (lane == 0) red_release_add(done_a + c, 1u);
        }
    }
}

// Largest resident grid of the pipelined kernel (blocks).
template <int D>
int pipelined_grid_impl(const Solver& s)
{
    int per_sm = 0;
    cudaError_t e = cudaSuccess;
    ELBM_DISPATCH_STORAGE(s.storage, {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pipelined<D, ST, 0>, kBlock, 0);
    });
    if (e != cudaSuccess) return 0;
    return per_sm * s.num_sms;
}

// Choose the chunking and the size of the sync buffer.
// Chunks hold enough layers for about 64k nodes, so that one phase spreads
// over the whole GPU while L + 2 chunks of populations stay well inside L2;
// L is chosen so that the blocks in flight (about one tile each) rarely reach
// a tile whose dependencies are unfinished.
template <int D>
PipeGeom pipelined_geometry_impl(const Solver& s)
{
    PipeGeom g{};
    const int layer = (D == 3) ? s.nx * s.ny : s.nx;
    const int nlayers = (D == 3) ? s.nz : s.ny;
    g.grid = pipelined_grid_impl<D>(s);
    g.chunk_planes = std::max(1, std::min(nlayers, (65536 + layer - 1) / layer));
    g.nchunks = (nlayers + g.chunk_planes - 1) / g.chunk_planes;
    g.tile_cells = ELBM_PIPE_TILE_CPT * 32;
    const int chunk_cells = g.chunk_planes * layer;
    g.tiles_per_chunk = (chunk_cells + g.tile_cells - 1) / g.tile_cells;
    // tiles in flight: one per resident warp
    const int warps = g.grid * (kBlock / 32);
    const int L = (warps + 2 * g.tiles_per_chunk - 1) / (2 * g.tiles_per_chunk) + 1;
    g.lookahead = (g.nchunks >= 3) ? std::max(1, std::min(L, g.nchunks - 2)) : 0;
    g.sync_words = 2 + 2 * (size_t)g.nchunks + 4 * (size_t)g.nchunks;
    return g;
}

template <int D>
cudaError_t step_pipelined_impl(const Solver& s, int parity, int nsteps, long long* launches)
{
    const PipeGeom& g = s.pipe;
    if (g.grid <= 0 || s.sync == nullptr) return cudaErrorInvalidConfiguration;
    StepParams p;
    fill_params(s, p);
    p.chunk_planes = g.chunk_planes;
    p.nchunks = g.nchunks;
    p.tile_cells = g.tile_cells;
    p.tiles_per_chunk = g.tiles_per_chunk;
    p.nsteps = 1;
    p.lookahead = g.lookahead;
    for (int k = 0; k < nsteps; ++k) {
        p.parity = (parity + k) & 1;
        cudaError_t e = cudaMemsetAsync(s.sync, 0, (2 + 2 * (size_t)g.nchunks) * sizeof(unsigned), s.stream);
        if (e != cudaSuccess) return e;
        void* args[] = {&p};
        ELBM_DISPATCH_STORAGE(s.storage, {
            const void* fn = (p.parity == 0) ? (const void*)k_pipelined<D, ST, 0> : (const void*)k_pipelined<D, ST, 1>;
            e = cudaLaunchCooperativeKernel(fn, dim3(g.grid), dim3(kBlock), args, 0, s.stream);
        });
        if (e != cudaSuccess) return e;
        ++*launches;
    }
    return cudaGetLastError();
}

}  // namespace elbm
