// Fused in-place step (one population array, AA pattern) of the D3Q27
// lattice: one launch per step, each population read from DRAM once.
//
// The two-pass form reads every node's populations twice -- once for the
// anomaly Q~ (Eq. Deviation) of the whole grid, once more to collide --
// because the central difference of Eq. Paastar1 needs the anomaly of the face
// neighbours at the same time level.  Here a block owns a 32 x 8 tile column
// and marches along z with the anomaly one plane ahead of the collision; each
// thread copies its node's populations (its AA read slots) into a column of a
// shared-memory stage with cp.async two planes before it collides them, and
// reads them from there for both the anomaly and the collision:
//   iteration z:  start the copy of plane z+2 (into the stage of plane z-1,
//                 collided last iteration); wait for the copy of plane z+1;
//                 its moments and anomaly: write Q~_xxx, Q~_yyy of plane z+1
//                 to the anomaly field (Q~_zzz goes to a ring of registers);
//                 publish "planes 0..z+1 done"; wait until the four
//                 face-neighbouring tile columns have published plane z
//                 (done an iteration earlier, so the wait rarely blocks);
//                 collide plane z from its stage (Eqs. Paastar1, 27eqext,
//                 LBGK), scattering to the AA write slots.
// A population is read from DRAM once, and the copy of a plane runs while the
// block collides the plane before it.  Publishing and waiting belong to a
// ninth warp: the consumers signal "anomaly of plane z+1 written" and wait
// for "neighbours have plane z" through shared-memory mbarriers and never
// stop at a block-wide barrier; the progress warp releases the block's
// counter once they have written, and acquires the neighbours' counters
// before it lets them collide.
// The z difference of plane 0 needs Q~_zzz of plane nz-1, which a prologue
// computes first (from the same, still untouched slots); the z difference of
// plane nz-1 needs Q~_zzz of plane 0, kept from before plane 0 was collided
// (its slots hold the next time level by then).
//
// Why blocks cannot race on populations: in the AA pattern a node reads and
// writes one slot set and the slot sets of distinct nodes are disjoint, so a
// block only ever touches the slot sets of its own nodes.  The one value that
// crosses blocks is the anomaly: its writer publishes a per-block progress
// counter with release semantics after the block's writes, the reader
// acquires its neighbours' counters before reading.  The counters grow
// monotonically over launches (epoch * (nz + 2) + planes done), so they
// never need resetting.  All blocks of a launch are co-resident (cooperative
// launch); every wait is bounded in time and, when it gives up, sets
// ELBM_ERR_TIMEOUT in the status word and stops the block.
//
// Staged copies cannot go stale: the slots a node reads in a step are the
// ones it writes, and only its own collision writes them.  The per-node
// arithmetic is the two-pass form's (staged gather, moments, anomaly,
// relax_streamed, scatter through the AA slots), so the results agree bit for
// bit.
#pragma once
#include "single_pass_tma.cuh"

namespace elbm {

constexpr int kFuTileX = 32, kFuTileY = 8;
constexpr int kFuThreads = kFuTileX * kFuTileY;

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Wait until *counter >= need (acquire), bounded: gives up once
// globaltimer - t0 exceeds limit_ns, then stores ELBM_ERR_TIMEOUT in *status
// and returns false.
__device__ __forceinline__ bool bounded_progress_wait(const unsigned long long* counter, unsigned long long need,
                                                      int* status, unsigned long long t0,
                                                      unsigned long long limit_ns)
{
    for (unsigned it = 0; ld_acquire_u64(counter) < need; ++it) {
        if ((it & 63) == 63 && globaltimer_ns() - t0 > limit_ns) {
            atomicExch(status, ELBM_ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

// Planes the anomaly runs ahead of the collision, and the shared-memory
// stage: a column of 27 words per consumer thread for each plane between its
// anomaly and its collision, plus the one being fetched.
constexpr int kFuLookahead = 1;
constexpr int kFuBufs = kFuLookahead + 2;
constexpr int kFuStageWords = kFuBufs * 27 * kFuThreads;
constexpr int kFuSmemBytes = (kFuStageWords + kFuBufs * kFuThreads) * 4;
// block: the consumer threads (one node each) + one warp that publishes the
// block's progress and acquires the neighbours'
constexpr int kFuBlock = kFuThreads + 32;

template <int ST, int PAR>
__global__ void __launch_bounds__(kFuBlock, 2)
    k_fused_aa(const __grid_constant__ StepParams p, unsigned long long* progress, unsigned long long epoch)
{
    static_assert(kFuLookahead == 1, "the cp.async group count below assumes one plane of look-ahead");
    constexpr int D = 3;
    extern __shared__ __align__(16) unsigned fu_smem[];
    unsigned* stage = fu_smem;                  // [kFuBufs][27][kFuThreads]
    unsigned* hmask = fu_smem + kFuStageWords;  // [kFuBufs][kFuThreads]: bit i, population i in the upper half
    // published(k & 1): the consumers wrote the anomaly of planes 0..k (count
    // kFuThreads); ready(z & 1): the four neighbouring tile columns have
    // released plane z (count 1).  Two of each suffice: the consumers arrive
    // on published(k+2) only after passing ready(k), which the progress warp
    // signals after observing published(k); it signals ready(z+2) only after
    // observing published(z+2), which the consumers arrive on after passing
    // ready(z).
    __shared__ __align__(8) unsigned long long s_bar[4];
    __shared__ int s_abort;
    const uint32_t bar0 = smem_u32(s_bar);
    auto published = [&](int k) { return bar0 + 8u * (k & 1); };
    auto ready = [&](int z) { return bar0 + 8u * (2 + (z & 1)); };
    volatile int* abort_flag = &s_abort;
    if (threadIdx.x == 0) {
        mbar_init(published(0), kFuThreads);
        mbar_init(published(1), kFuThreads);
        mbar_init(ready(0), 1);
        mbar_init(ready(1), 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int bx = blockIdx.x, by = blockIdx.y, nbx = gridDim.x, nby = gridDim.y;
    const unsigned long long base = epoch * (unsigned long long)(p.nz + 2);

    if (threadIdx.x >= kFuThreads) {
        // ------------------------------------------------ progress warp
        // publication k = "planes 0..k of the anomaly written" is released
        // as counter value base + k + 1, after the consumers' arrivals on
        // published(k); ready(z) is signalled once all four neighbours have
        // released plane z.  Acquiring plane z comes before waiting for the
        // block's own publication z + 1, so that the consumers, who publish
        // z + 1 before they need plane z, never wait on their own release.
        const int lane = threadIdx.x & 31;
        const int me = by * nbx + bx;
        const int nb[4] = {by * nbx + (bx == 0 ? nbx - 1 : bx - 1), by * nbx + (bx == nbx - 1 ? 0 : bx + 1),
                           (by == 0 ? nby - 1 : by - 1) * nbx + bx, (by == nby - 1 ? 0 : by + 1) * nbx + bx};
        auto release = [&](int k) {
            if (!bounded_wait(published(k), (unsigned)(k >> 1) & 1u, abort_flag, p.status, kTmaWaitNs)) return false;
            if (lane == 0) st_release_u64(progress + me, base + (unsigned long long)(k + 1));
            return true;
        };
        if (!__all_sync(0xffffffffu, release(0))) return;
        for (int z = 0; z < p.nz; ++z) {
            bool ok = true;
            if (lane < 4) {
                ok = bounded_progress_wait(progress + nb[lane], base + (unsigned long long)(z + 1), p.status,
                                           globaltimer_ns(), kTmaWaitNs);
                if (!ok) *abort_flag = 1;
            }
            if (!__all_sync(0xffffffffu, ok)) return;
            if (lane == 0) mbar_arrive(ready(z));
            if (z + 1 < p.nz && !__all_sync(0xffffffffu, release(z + 1))) return;
        }
        return;
    }
    // ------------------------------------------------------ consumers
    const int tx = threadIdx.x % kFuTileX, ty = threadIdx.x / kFuTileX;
    const int gx = bx * kFuTileX + tx, gy = by * kFuTileY + ty;
    const bool active = gx < p.nx && gy < p.ny;
    float* qx = p.q;
    float* qy = p.q + p.N;
    // node (gx, gy, z); inactive threads of a ragged tile take a valid node and do nothing with it
    auto node_at = [&](int z) { return make_node<D>(p, (active ? gx + gy * p.nx : 0) + z * p.plane); };
    // copy the own node's populations at plane z (its AA read slots) into its stage column
    auto stage_plane = [&](int z) {
        const Node n = node_at(z);
        unsigned* c = stage + (z % kFuBufs) * 27 * kFuThreads + threadIdx.x;
        unsigned h = 0;
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            const int idx = read_slot<D>(n, p.N, i, PAR);
            h |= (unsigned)(idx & 1) << i;
            cp_async4(c + i * kFuThreads, stage_src<ST>(p, idx));
        }
        hmask[(z % kFuBufs) * kFuThreads + threadIdx.x] = h;
    };
    // population i of the own node at plane z, from the stage
    auto staged = [&](int z) {
        const unsigned* c = stage + (z % kFuBufs) * 27 * kFuThreads + threadIdx.x;
        const unsigned h = hmask[(z % kFuBufs) * kFuThreads + threadIdx.x];
        return [=, &p](int i) { return stage_value<ST>(p, ld_stage(c + i * kFuThreads), (int)((h >> i) & 1u), i); };
    };
    // anomaly of the own node at plane z from the stage: Q~_xxx, Q~_yyy to the field, Q~_zzz returned
    auto anomaly_staged = [&](int z) {
        float drho, j[3];
        moments_of<D>(p, staged(z), drho, j);
        const float inv = 1.0f / (p.rho_ref + drho);
        const int cell = gx + gy * p.nx + z * p.plane;
        qx[cell] = anomaly(p, 0, j[0], j[0] * inv);
        qy[cell] = anomaly(p, 1, j[1], j[1] * inv);
        return anomaly(p, 2, j[2], j[2] * inv);
    };
    // ring[k]: Q~_zzz of the own node at plane z - 1 + k, k = 0 .. 2
    float ring[3] = {0.f, 0.f, 0.f};
    if (active) {
        // plane -1 (periodic: nz-1), straight from its slots, which no collision has touched yet
        const Node n = node_at(p.nz - 1);
        float g[27], drho, j[3];
        gather<D, ST, PAR>(p, n, g);
        moments<D>(p, g, drho, j);
        const float inv = 1.0f / (p.rho_ref + drho);
        ring[0] = anomaly(p, 2, j[2], j[2] * inv);
    }
    // planes 0 and 1 into the stage (always two cp.async groups, so that the
    // "all but the newest group" waits below name the right plane)
    stage_plane(0);
    cp_async_commit();
    if (p.nz > 1) stage_plane(1);
    cp_async_commit();
    cp_async_wait_prior();  // plane 0 is in
    if (active) ring[1] = anomaly_staged(0);
    mbar_arrive(published(0));
    const float qz_first = ring[1];  // plane 0, before it is collided
    for (int z = 0; z < p.nz; ++z) {
        const int za = z + 1;
        // --------------- fetch plane z + 2 into the stage of plane z - 1 (collided)
        if (za + 1 < p.nz) stage_plane(za + 1);
        cp_async_commit();
        cp_async_wait_prior();  // plane z + 1 is in
        // ----------------------------- anomaly of plane z + 1, published
        float qa = qz_first;
        if (za < p.nz) {
            if (active) qa = anomaly_staged(za);
            mbar_arrive(published(za));
        }
        ring[2] = qa;
        // --------------- wait until the neighbouring columns have plane z
        if (!bounded_wait(ready(z), (unsigned)(z >> 1) & 1u, abort_flag, p.status, kTmaWaitNs)) break;
        // ------------------------- collide plane z (from its stage column)
        if (active) {
            const Node n = node_at(z);
            auto gv = staged(z);
            float drho, j[3];
            moments_of<D>(p, gv, drho, j);
            float d[3] = {0.f, 0.f, 0.f};
            if (p.eq_mode == 0) {
                d[0] = (__ldcg(qx + n.at(1, 0, 0)) - __ldcg(qx + n.at(-1, 0, 0))) * p.inv_2lam[0];
                d[1] = (__ldcg(qy + n.at(0, 1, 0)) - __ldcg(qy + n.at(0, -1, 0))) * p.inv_2lam[1];
                d[2] = (ring[2] - ring[0]) * p.inv_2lam[2];
            }
            using S = Storage<ST>;
            typename S::T* f = static_cast<typename S::T*>(p.f);
            const int cell_o = opaque(n.cell);
            auto put = [&](int i, float v) {
                const int slot = (PAR == 0) ? (26 - i) * p.N + cell_o : write_slot<D>(n, p.N, i, PAR);
                S::store(f + slot, S::shifted ? v : fmaf(p.bw[i], p.rho_ref, v));
            };
            relax_streamed<D>(p, gv, put, drho, j, d);
        }
        ring[0] = ring[1];
        ring[1] = ring[2];
    }
    cp_async_wait_all();  // no copy may still be in flight when the block retires
}

// Whether the fused form takes solver s and how many of its blocks fit the GPU at once.
template <int ST>
bool fused_fits(const Solver& s, int* blocks_x, int* blocks_y)
{
    *blocks_x = (s.nx + kFuTileX - 1) / kFuTileX;
    *blocks_y = (s.ny + kFuTileY - 1) / kFuTileY;
    int per_sm = 0;
    if (set_smem_limit_once<k_fused_aa<ST, 0>>(kFuSmemBytes) != cudaSuccess ||
        set_smem_limit_once<k_fused_aa<ST, 1>>(kFuSmemBytes) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_aa<ST, 0>, kFuBlock, kFuSmemBytes) !=
            cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return (long long)per_sm * s.num_sms >= (long long)*blocks_x * *blocks_y;
}

}  // namespace elbm
