// Single-pass step with two population arrays: TMA-fed, warp-specialised, with
// the populations parked in tensor memory (TMEM) between their two uses.
//
// The per-node arithmetic is that of single_pass.cuh (bit-identical results).
// A block of five warpgroups owns a tile of 32 x 16 columns and marches
// through kSegPlanes z planes:
//   * the first warp of warpgroup 4 loads plane k of the tile with one 4-D
//     TMA box (x 32, y 16, z 1, population 27) into a ring of tile buffers in
//     shared memory, and the ring of nodes around the tile -- two TMA row
//     boxes and two columns of 16 nodes by cp.async -- into a ring of two
//     buffers; one mbarrier per buffer ("full") tracks both kinds of copy.
//     With 16-bit storage its other three warps compute the anomaly of the
//     ring (the row below, the row above, the two columns); with FP32 storage
//     they idle (TMEM lane quarters follow a warp's rank within its
//     warpgroup, so the consumers must make whole warpgroups) and the
//     consumers share the ring out;
//   * the 16 warps of warpgroups 0..3 each own one tile row.  For plane k a
//     thread reads its node's 27 populations from shared memory once, hands
//     the buffer back ("empty" mbarrier), parks the values in its TMEM lane,
//     computes the anomaly Q~ of its node (FP32 storage: and of a share of the
//     ring, the duty rotating over the warps from plane to plane), publishes it ("qready")
//     and relaxes plane k-1 -- with the values parked one plane earlier --
//     once every warp has published the anomaly of plane k-1 (the central
//     difference of Eq. Paastar1 needs the face neighbours), pushing the 27
//     results with coalesced stores.
// Shared memory is kept small on purpose: an SM's shared memory and its L1
// cache are carved from one array, and the step rate grew as the footprint
// shrank.  A tile buffer comes back as soon as it has been read, and the
// relaxation of the previous plane covers the next load, so FP32 storage runs
// fastest with a single buffer; 16-bit storage (half the bytes, more
// arithmetic per byte) with two.  There is no block-wide barrier in the loop.
// Every wait is bounded (2 s, or as soon as another thread of the block gave
// up); a wait that gives up sets ELBM_ERR_TIMEOUT in the status word, and the
// block winds down: the loader waits, again bounded, for the copies in flight,
// and the TMEM is freed by the warp that allocated it.
#pragma once
#include "single_pass_tma.cuh"

namespace elbm {

constexpr int kTmTileY = 16;                      // tile rows (one consumer warp each)
constexpr int kTmConsumers = kTileX * kTmTileY;   // 512 threads
constexpr int kTmThreads = kTmConsumers + 128;    // + the loading warpgroup
constexpr uint32_t kTmTmemCols = 256;             // 2 plane slots x 4 warps per lane quarter x 32

template <int ST>
struct TmemLayout {
    using T = typename Storage<ST>::T;
    static constexpr int es = (int)sizeof(T);
    static constexpr int ntile = es == 4 ? 1 : 2;                    // tile buffers
    // threads that compute the ring's anomaly apart from the consumers: for
    // 16-bit storage (issue-bound) the three spare warps of the loading
    // warpgroup; for FP32 (latency-bound) the consumers share it out
    static constexpr int ring_threads = es == 4 ? 0 : 96;
    static constexpr int tile_bytes = 27 * kTmTileY * kTileX * es;   // one plane of the tile
    static constexpr int row_box_bytes = 27 * kTileX * es;           // one ring row, all populations
    static constexpr int row_stride = (row_box_bytes + 127) / 128 * 128;
    static constexpr int ncol = 2 * kTmTileY;                        // ring column nodes
    static constexpr int cols_bytes = 27 * ncol * 4;                 // as 4-byte words
    static constexpr int qx_bytes = kTmTileY * (kTileX + 2) * 4;
    static constexpr int qy_bytes = (kTmTileY + 2) * kTileX * 4;
    static constexpr int off_tile = 0;                               // [ntile] planes
    static constexpr int off_rows = off_tile + ntile * tile_bytes;   // [2 slots][2 sides]
    static constexpr int off_cols = off_rows + 4 * row_stride;       // [2 slots]
    static constexpr int off_qx = off_cols + 2 * cols_bytes;         // [kTmaQSlots]
    static constexpr int off_qy = off_qx + kTmaQSlots * qx_bytes;
    static constexpr int off_bar = (off_qy + kTmaQSlots * qy_bytes + 7) / 8 * 8;
    // mbarriers, in this order: full and empty per tile buffer, full and empty
    // per ring buffer, one per anomaly slot
    static constexpr int bar_full_t = 0, bar_empty_t = ntile, bar_full_r = 2 * ntile, bar_empty_r = 2 * ntile + 2;
    static constexpr int bar_qready = 2 * ntile + 4;
    static constexpr int nbar = bar_qready + kTmaQSlots;
    static constexpr int off_abort = off_bar + 8 * nbar;
    static constexpr int off_tmem = off_abort + 4;
    static constexpr int bytes = off_abort + 16 + 128;               // + slack for aligning the base
    static_assert(tile_bytes % 128 == 0, "tile boxes must keep 128-byte alignment");
};

// One tile column of a single-pass step: the 32 x 16 columns at (x0, y0),
// planes z0 .. z1-1, from p.f into dst; every thread of the block takes part.
// tm_tile / tm_row are the tensor maps of p.f (kernel parameters, or device
// memory made visible to the tensor-map proxy).  smem_raw is the block's
// dynamic shared memory (TmemLayout<ST>::bytes).
// BC: walls (half-way bounce-back below y = 0 and above y = ny-1, with the
// anomaly's negated ghost value in the central difference) and the body force,
// read from the parameter block as in the two-pass kernels; with neither set
// in p it computes the same bits as BC = false.
template <int ST, bool BC, bool FX = false>
__device__ __forceinline__ void tmem_tile_step(const CUtensorMap* tm_tile, const CUtensorMap* tm_row,
                                               const StepParams& p, void* dst, int x0, int y0, int z0, int z1,
                                               unsigned char* smem_raw)
{
    using S = Storage<ST>;
    using T = typename S::T;
    using L = TmemLayout<ST>;
    const uint32_t raw_addr = smem_u32(smem_raw);
    const uint32_t sbase = (raw_addr + 127u) & ~127u;
    unsigned char* base = smem_raw + (sbase - raw_addr);
    const uint32_t bar0 = sbase + L::off_bar;
    auto full_t = [&](int b) { return bar0 + 8u * (L::bar_full_t + b); };
    auto empty_t = [&](int b) { return bar0 + 8u * (L::bar_empty_t + b); };
    auto full_r = [&](int r) { return bar0 + 8u * (L::bar_full_r + r); };
    auto empty_r = [&](int r) { return bar0 + 8u * (L::bar_empty_r + r); };
    auto qready = [&](int s) { return bar0 + 8u * (L::bar_qready + s); };
    volatile int* abort_flag = reinterpret_cast<volatile int*>(base + L::off_abort);

    const int K = (z1 - z0) + 2;  // planes z0-1 .. z1
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kLoader = kTmConsumers / 32;  // first warp of the loading warpgroup
    pdl_release();

    if (threadIdx.x == 0) {
        for (int b = 0; b < L::ntile; ++b) {
            mbar_init(full_t(b), 1);
            mbar_init(empty_t(b), kTmConsumers);
        }
        for (int r = 0; r < 2; ++r) {
            mbar_init(full_r(r), 1 + 32);  // loader lane 0 (expect_tx) + the cp.async arrivals of its 32 lanes
            mbar_init(empty_r(r), kTmConsumers + L::ring_threads);
        }
        for (int s = 0; s < kTmaQSlots; ++s) mbar_init(qready(s), kTmConsumers + L::ring_threads);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kLoader) {
        tmem_alloc(sbase + L::off_tmem, kTmTmemCols);
        tmem_relinquish();
    }
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    const uint32_t tmem_base = *reinterpret_cast<volatile uint32_t*>(base + L::off_tmem);
    pdl_wait();  // the previous step has written the source array

    // bounded in time (kTmaWaitNs), or as soon as another thread of the block gave up
    auto wait = [&](uint32_t bar, unsigned parity) { return bounded_wait(bar, parity, abort_flag, p.status, kTmaWaitNs); };
    auto drain = [&](uint32_t bar, unsigned parity) { bounded_drain(bar, parity, kTmaWaitNs); };
    auto plane_of = [&](int k) { return wrapi(z0 - 1 + k, p.nz); };

    if (warp >= kLoader) {
        if (warp == kLoader) {
            // ---------------------------------------------------- loader
            // ring column node kk: x0-1 for kk < 16, x0+32 for kk >= 16, row y0 + (kk & 15)
            const int ylo = wrapi(y0 - 1, p.ny), yhi = wrapi(y0 + kTmTileY, p.ny);
            const int cxl = wrapi(x0 - 1, p.nx), cxr = wrapi(x0 + kTileX, p.nx);
            int issued = 0;
            for (int k = 0; k < K; ++k) {
                const int b = k % L::ntile, r = k & 1;
                bool ok = true;
                if (k >= L::ntile) ok = wait(empty_t(b), ((k / L::ntile) - 1) & 1);
                if (ok && k >= 2) ok = wait(empty_r(r), ((k / 2) - 1) & 1);
                if (!__all_sync(0xffffffffu, ok)) break;
                const int zk = plane_of(k);
                if (lane == 0) {
                    mbar_arrive_expect_tx(full_t(b), L::tile_bytes);
                    tma_load_4d(sbase + L::off_tile + b * L::tile_bytes, tm_tile, x0, y0, zk, 0, full_t(b));
                    mbar_arrive_expect_tx(full_r(r), 2 * L::row_box_bytes);
                    tma_load_4d(sbase + L::off_rows + (2 * r) * L::row_stride, tm_row, x0, ylo, zk, 0, full_r(r));
                    tma_load_4d(sbase + L::off_rows + (2 * r + 1) * L::row_stride, tm_row, x0, yhi, zk, 0,
                                full_r(r));
                }
                unsigned* cols = reinterpret_cast<unsigned*>(base + L::off_cols + r * L::cols_bytes);
                for (int c = lane; c < 27 * L::ncol; c += 32) {
                    const int i = c / L::ncol, kk = c % L::ncol;
                    const int idx = i * p.N + zk * p.plane + (y0 + (kk & (kTmTileY - 1))) * p.nx +
                                    (kk < kTmTileY ? cxl : cxr);
                    cp_async4(cols + c, stage_src<ST>(p, idx));
                }
                cp_async_mbar_arrive(full_r(r));
                issued = k + 1;
            }
            cp_async_wait_all();
            // no copy may still be in flight when the block retires
            if (lane == 0) {
                for (int k = max(0, issued - L::ntile); k < issued; ++k) drain(full_t(k % L::ntile), (k / L::ntile) & 1);
                for (int k = max(0, issued - 2); k < issued; ++k) drain(full_r(k & 1), (k / 2) & 1);
            }
            __syncwarp();
        } else if (L::ring_threads > 0) {
            // ------------------------------------------------ ring anomaly
            // warp 1 of the group: the row below the tile, warp 2: the row
            // above, warp 3: the two columns (nodes x0-1 and x0+32 of the tile's rows)
            const int duty = warp - kLoader - 1;
            auto anomaly_of = [&](auto&& gval, float* q) {
                float drho, j[3];
                moments_of<3>(p, gval, drho, j);
                const float inv_rho = 1.0f / (p.rho_ref + drho);
#pragma unroll
                for (int a = 0; a < 3; ++a) q[a] = anomaly(p, a, j[a], j[a] * inv_rho);
            };
            float* qxs = reinterpret_cast<float*>(base + L::off_qx);
            float* qys = reinterpret_cast<float*>(base + L::off_qy);
            for (int k = 0; k < K; ++k) {
                const int r = k & 1, s = k % kTmaQSlots;
                if (!__all_sync(0xffffffffu, wait(full_r(r), (k / 2) & 1))) break;
                if (k > 0 && k < K - 1) {
                    float qh[3];
                    if (duty < 2) {
                        const T* row =
                            reinterpret_cast<const T*>(base + L::off_rows + (2 * r + duty) * L::row_stride) + lane;
                        anomaly_of([&](int i) { return raw_value<ST>(p, row[i * kTileX], i); }, qh);
                        qys[(s * (kTmTileY + 2) + (duty ? kTmTileY + 1 : 0)) * kTileX + lane] = qh[1];
                    } else {
                        const unsigned* cols =
                            reinterpret_cast<const unsigned*>(base + L::off_cols + r * L::cols_bytes) + lane;
                        const int cx = lane < kTmTileY ? wrapi(x0 - 1, p.nx) : wrapi(x0 + kTileX, p.nx);
                        const int idx0 = plane_of(k) * p.plane + (y0 + (lane & (kTmTileY - 1))) * p.nx + cx;
                        anomaly_of([&](int i) { return stage_value<ST>(p, cols[i * L::ncol], (i * p.N + idx0) & 1, i); },
                                   qh);
                        qxs[(s * kTmTileY + (lane & (kTmTileY - 1))) * (kTileX + 2) + (lane < kTmTileY ? 0 : kTileX + 1)] =
                            qh[0];
                    }
                }
                __syncwarp();
                mbar_arrive(empty_r(r));
                mbar_arrive(qready(s));
            }
        }
    } else {
        // ------------------------------------------------------ consumers
        const int tx = lane, ty = warp;
        const int gx = x0 + tx, gy = y0 + ty;
        const T* tile = reinterpret_cast<const T*>(base + L::off_tile);
        float* qxs = reinterpret_cast<float*>(base + L::off_qx);
        float* qys = reinterpret_cast<float*>(base + L::off_qy);
        auto QX = [&](int s, int y, int x) -> float& { return qxs[(s * kTmTileY + y) * (kTileX + 2) + x]; };
        auto QY = [&](int s, int y, int x) -> float& { return qys[(s * (kTmTileY + 2) + y) * kTileX + x]; };
        auto anomaly_m = [&](auto&& gval, float* q, float& drho, float* j, float& inv_rho) {
            moments_of<3>(p, gval, drho, j);
            inv_rho = 1.0f / (p.rho_ref + drho);
#pragma unroll
            for (int a = 0; a < 3; ++a) q[a] = anomaly(p, a, j[a], j[a] * inv_rho);
        };
        auto anomaly_of = [&](auto&& gval, float* q) {
            float drho, j[3], inv_rho;
            anomaly_m(gval, q, drho, j, inv_rho);
        };
        // TMEM columns of this thread: its warp's lane quarter; 32 columns per
        // warp of the quarter (warps w, w+4, w+8, w+12 share a quarter); 128 per plane slot
        const uint32_t t_own = tmem_base + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * 32);
        T* out = static_cast<T*>(dst);
        const int xo[3] = {gx == 0 ? p.nx - 1 : gx - 1, gx, gx == p.nx - 1 ? 0 : gx + 1};
        const int yo[3] = {(gy == 0 ? p.ny - 1 : gy - 1) * p.nx, gy * p.nx, (gy == p.ny - 1 ? 0 : gy + 1) * p.nx};
        constexpr int kPlaneElems = kTmTileY * kTileX;  // stride between populations in a tile buffer

        float qz_prev = 0.f, qz_cur = 0.f;
        // moments of the own node of the plane relaxed next (computed with its anomaly)
        float m_drho = 0.f, m_j[3] = {0.f, 0.f, 0.f}, m_inv_rho = 1.f;
        for (int k = 0; k < K; ++k) {
            const int b = k % L::ntile, r = k & 1, s = k % kTmaQSlots;
            const bool got = wait(full_t(b), (k / L::ntile) & 1) && wait(full_r(r), (k / 2) & 1);
            if (!__all_sync(0xffffffffu, got)) break;
            float q[3], k_drho, k_j[3], k_inv_rho;
            {
                const T* own = tile + b * 27 * kPlaneElems + ty * kTileX + tx;
                float g[27];
#pragma unroll
                for (int i = 0; i < 27; ++i) g[i] = raw_value<ST>(p, own[i * kPlaneElems], i);
                mbar_arrive(empty_t(b));
                if (k >= 1 && k < K - 1) tmem_store27(t_own + (uint32_t)((k & 1) * 128), g);
                anomaly_m([&](int i) { return g[i]; }, q, k_drho, k_j, k_inv_rho);
            }
            QX(s, ty, tx + 1) = q[0];
            QY(s, ty + 1, tx) = q[1];
            // ring share of this warp for plane k (duty rotates with k): 0 the
            // row below the tile, 1 the row above, 2 the two columns
            const int duty = (ty + k) & (kTmTileY - 1);
            if (L::ring_threads == 0 && k > 0 && k < K - 1) {
                if (duty < 2) {
                    const T* row = reinterpret_cast<const T*>(base + L::off_rows + (2 * r + duty) * L::row_stride) + tx;
                    float qh[3];
                    anomaly_of([&](int i) { return raw_value<ST>(p, row[i * kTileX], i); }, qh);
                    QY(s, duty ? kTmTileY + 1 : 0, tx) = qh[1];
                } else if (duty == 2) {
                    const unsigned* cols = reinterpret_cast<const unsigned*>(base + L::off_cols + r * L::cols_bytes) + tx;
                    const int cx = tx < kTmTileY ? wrapi(x0 - 1, p.nx) : wrapi(x0 + kTileX, p.nx);
                    const int idx0 = plane_of(k) * p.plane + (y0 + (tx & (kTmTileY - 1))) * p.nx + cx;
                    float qh[3];
                    anomaly_of([&](int i) { return stage_value<ST>(p, cols[i * L::ncol], (i * p.N + idx0) & 1, i); },
                               qh);
                    QX(s, tx & (kTmTileY - 1), tx < kTmTileY ? 0 : kTileX + 1) = qh[0];
                }
            }
            __syncwarp();
            mbar_arrive(empty_r(r));
            mbar_arrive(qready(s));
            if (k == 0) {
                qz_prev = q[2];
                continue;
            }
            if (k == 1) {
                qz_cur = q[2];
                m_drho = k_drho;
                m_inv_rho = k_inv_rho;
#pragma unroll
                for (int a = 0; a < 3; ++a) m_j[a] = k_j[a];
                continue;
            }
            // relax plane k-1 (z = z0 + k - 2) once every warp has published its anomaly
            const float qz_next = q[2];
            const int kc = k - 1, sc = kc % kTmaQSlots;
            if (!__all_sync(0xffffffffu, wait(qready(sc), (kc / kTmaQSlots) & 1))) break;
            float g[27];
            tmem_wait_st();
            tmem_load27(t_own + (uint32_t)((kc & 1) * 128), g);
            auto gval = [&](int i) { return g[i]; };
            const float drho = m_drho, j[3] = {m_j[0], m_j[1], m_j[2]};  // moments_of of the same values
            float d[3] = {0.f, 0.f, 0.f};
            if (p.eq_mode == 0) {
                d[0] = (QX(sc, ty, tx + 2) - QX(sc, ty, tx)) * p.inv_2lam[0];
                float qyp = QY(sc, ty + 2, tx), qym = QY(sc, ty, tx);
                if (BC && p.walls_y && gy == p.ny - 1) qyp = -QY(sc, ty + 1, tx);  // ghost beyond the wall
                if (BC && p.walls_y && gy == 0) qym = -QY(sc, ty + 1, tx);
                d[1] = (qyp - qym) * p.inv_2lam[1];
                d[2] = (qz_next - qz_prev) * p.inv_2lam[2];
            }
            const int z = z0 + k - 2;
            const int zo[3] = {wrapi(z - 1, p.nz) * p.plane, z * p.plane, wrapi(z + 1, p.nz) * p.plane};
            int yz[9];  // push target offset of the row (y + cy, z + cz)
#pragma unroll
            for (int c = 0; c < 9; ++c) yz[c] = yo[c % 3] + zo[c / 3];
            auto put = [&](int i, float gn) {
                const float v = S::shifted ? gn : fmaf(p.bw[i], p.rho_ref, gn);
                if (BC && p.walls_y && ((cy_of(i) == 1 && gy == p.ny - 1) || (cy_of(i) == -1 && gy == 0))) {
                    // half-way bounce-back: f'_i returns reversed to its own node, as
                    // population opp(i), stored against opp(i)'s baseline
                    const float vb = S::shifted ? v + bounce_rebase<3>(p, 26 - i) : v;
                    S::store(out + opaque((26 - i) * p.N) + gx + gy * p.nx + z * p.plane, vb);
                } else {
                    const int slot = opaque(i * p.N) + (xo[cx_of(i) + 1] + yz[(cy_of(i) + 1) + 3 * (cz_of<3>(i) + 1)]);
                    S::store(out + slot, v);
                }
            };
            // (the walls-and-force kernel recomputes it: one register fewer across the loop)
            relax_streamed<3, false, BC, FX>(p, gval, put, drho, j, d, BC ? 0.f : m_inv_rho);
            qz_prev = qz_cur;
            qz_cur = qz_next;
            m_drho = k_drho;
            m_inv_rho = k_inv_rho;
#pragma unroll
            for (int a = 0; a < 3; ++a) m_j[a] = k_j[a];
        }
        tmem_wait_st();
    }
    // every TMEM access of the block is complete before the loader frees it
    tmem_fence_before_sync();
    __syncthreads();
    if (warp == kLoader) {
        tmem_fence_after_sync();
        tmem_dealloc(tmem_base, kTmTmemCols);
    }
}

// The single-pass step of one grid: block (bx, by, bz) takes the tile column
// at (32 bx, 16 by), planes kSegPlanes bz onwards.  FX (with BC): the body
// force acts along x alone.
template <int ST, bool BC = false, bool FX = false>
__global__ void __launch_bounds__(kTmThreads, 1)
    k_single_pass_tmem(const __grid_constant__ CUtensorMap tm_tile, const __grid_constant__ CUtensorMap tm_row,
                       const __grid_constant__ StepParams p, void* dst)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int z0 = blockIdx.z * kSegPlanes;
    tmem_tile_step<ST, BC, FX>(&tm_tile, &tm_row, p, dst, blockIdx.x * kTileX, blockIdx.y * kTmTileY, z0,
                               min(p.nz, z0 + kSegPlanes), smem_raw);
}

template <int ST>
bool single_tmem_ok(const Solver& s, const void* src, const void* dst)
{
    using T = typename Storage<ST>::T;
    return s.nx % kTileX == 0 && s.ny % kTmTileY == 0 && (s.nx * (int)sizeof(T)) % 16 == 0 &&
           ((uintptr_t)src % 16 == 0) && ((uintptr_t)dst % 16 == 0);
}

template <int ST, bool BC = false, bool FX = false>
cudaError_t launch_single_tmem(const Solver& s, const StepParams& p, void* dst, bool* launched)
{
    *launched = false;
    if (!single_tmem_ok<ST>(s, p.f, dst)) return cudaSuccess;
    CUtensorMap tm_tile, tm_row;
    if (encode_population_maps(s, p.f, kTmTileY, &tm_tile, &tm_row) != cudaSuccess) return cudaSuccess;
    const int smem = TmemLayout<ST>::bytes;
    cudaError_t e = set_smem_limit_once<k_single_pass_tmem<ST, BC, FX>>(smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)(s.nx / kTileX), (unsigned)(s.ny / kTmTileY),
                    (unsigned)((s.nz + kSegPlanes - 1) / kSegPlanes));
    // programmatic dependent launch helps the 16-bit form (+0.5 %) and costs the
    // FP32 form 0.7 % (256^3, measured), so only 16-bit storage uses it
    if (sizeof(typename Storage<ST>::T) == 2) {
        e = launch_pdl(k_single_pass_tmem<ST, BC, FX>, grid, dim3(kTmThreads), smem, s.stream, tm_tile, tm_row, p, dst);
    } else {
        k_single_pass_tmem<ST, BC, FX><<<grid, kTmThreads, smem, s.stream>>>(tm_tile, tm_row, p, dst);
        e = cudaGetLastError();
    }
    *launched = e == cudaSuccess;
    return e;
}

// One single-pass step from s.f into dst (D3Q27 only; the caller swaps the arrays):
// the TMA-fed kernels where the geometry allows (32 x 16 tiles with TMEM,
// else 32 x 8 tiles), else the cp.async-staged ones.
template <int D>
cudaError_t step_single_impl(const Solver& s, void* dst, long long* launches)
{
    if constexpr (D != 3) {
        (void)s;
        (void)dst;
        (void)launches;
        return cudaErrorNotSupported;
    } else {
        StepParams p;
        fill_params(s, p);
        p.parity = 0;
        const dim3 grid((unsigned)((s.nx + kTileX - 1) / kTileX), (unsigned)((s.ny + kTileY - 1) / kTileY),
                        (unsigned)((s.nz + kSegPlanes - 1) / kSegPlanes));
        const size_t smem = sizeof(SingleSmem);
        cudaError_t e = cudaSuccess;
        ELBM_DISPATCH_STORAGE(s.storage, {
            bool done = false;
            if (p.walls_y || p.forced) {
                // walls and body force: the TMEM form only (the caller checks its geometry);
                // a force along x alone (or none) takes the lighter force increment
                const bool fx = p.g[1] == 0.f && p.g[2] == 0.f;
                e = fx ? launch_single_tmem<ST, true, true>(s, p, dst, &done)
                       : launch_single_tmem<ST, true, false>(s, p, dst, &done);
                if (e == cudaSuccess && !done) e = cudaErrorNotSupported;
                if (e == cudaSuccess) ++*launches;
                return e;
            }
            e = launch_single_tmem<ST>(s, p, dst, &done);
            if (e == cudaSuccess && !done) e = launch_single_tma<ST>(s, p, dst, &done);
            if (e != cudaSuccess || done) {
                if (e == cudaSuccess) ++*launches;
                return e;
            }
            if (single_fast_ok<ST>(s)) {
                const size_t fsmem = sizeof(FastSmem<ST>);
                e = set_smem_limit_once<k_single_pass_fast<ST>>((int)fsmem);
                if (e == cudaSuccess) k_single_pass_fast<ST><<<grid, kBlock, fsmem, s.stream>>>(p, dst);
            } else {
                e = set_smem_limit_once<k_single_pass<ST>>((int)smem);
                if (e == cudaSuccess) k_single_pass<ST><<<grid, kBlock, smem, s.stream>>>(p, dst);
            }
        });
        if (e != cudaSuccess) return e;
        ++*launches;
        return cudaGetLastError();
    }
}

}  // namespace elbm
