// Single-pass step with two population arrays, fed by the tensor memory
// accelerator (TMA) and split into a producer warp and eight consumer warps.
//
// What it computes is the single pass of single_pass.cuh (same tile, same
// per-node arithmetic, bit-identical results): a block owns a tile of
// 32 x 8 columns and marches through kSegPlanes z planes; for every plane it
// needs the populations of the tile and of the ring of nodes around it (for
// the anomaly Q~ of the face neighbours, Eq. Paastar1), and the anomaly of the
// planes above and below (own column only).
//
// How the work is arranged:
//   * the producer warp loads plane k of the tile with one 4-D TMA box
//     (x 32, y 8, z 1, population 27) and the two ring rows with two more,
//     into a ring of three tile buffers and two ring buffers; the two ring
//     columns (8 nodes each, not 16-byte aligned) come with cp.async, whose
//     completion the same mbarrier tracks.  Loads run two planes ahead.
//   * consumer warp w relaxes tile row w.  Per plane k it waits for the
//     tile/ring buffers of plane k (mbarrier "full"), computes the anomaly
//     of its node and of a share of the ring (the ring duty rotates over the
//     warps from plane to plane), publishes them (mbarrier "qready") and
//     relaxes plane k-1 once every warp has published the anomaly of plane
//     k-1.  Buffers go back to the producer through "empty" mbarriers.
//   * no block-wide barrier in the loop: a warp waits only for data it reads.
// Every wait is bounded; a wait that gives up sets ELBM_ERR_TIMEOUT in the
// status word and the block winds down (the producer first waits, again
// bounded, for the copies it has in flight).
#pragma once
#include <cuda.h>

#include <atomic>

#include "single_pass.cuh"

namespace elbm {

constexpr int kTmaThreads = kBlock + 32;  // 8 consumer warps + 1 producer warp
constexpr int kTmaQSlots = 4;             // anomaly planes kept (see the slot argument below)
constexpr unsigned long long kTmaWaitNs = 2000000000ull;  // a wait gives up after 2 s

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* ptr)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(ptr));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, unsigned bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Arrive on `bar` once every cp.async this thread has issued so far has landed
// (the arrival counts against the barrier's expected count).
__device__ __forceinline__ void cp_async_mbar_arrive(uint32_t bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
// Bounded wait for the completion of phase `parity` of an mbarrier: gives up
// after limit_ns (read from %globaltimer), or as soon as another thread of
// the block has given up (*abort_flag); the first thread to give up raises
// the flag and stores ELBM_ERR_TIMEOUT in the status word.  Returns true once
// the phase has completed.
__device__ __forceinline__ bool bounded_wait(uint32_t bar, unsigned parity, volatile int* abort_flag, int* status,
                                             unsigned long long limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (unsigned n = 1;; ++n) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((n & 63) == 0) {
            if (*abort_flag) return false;
            if (globaltimer_ns() - t0 > limit_ns) {
                if (!*abort_flag) {
                    *abort_flag = 1;
                    atomicExch(status, ELBM_ERR_TIMEOUT);
                }
                return false;
            }
        }
    }
}
// The same bound, for draining copies in flight (ignores the abort flag).
__device__ __forceinline__ void bounded_drain(uint32_t bar, unsigned parity, unsigned long long limit_ns)
{
    const unsigned long long t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity) && globaltimer_ns() - t0 < limit_ns) {}
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// ------------------------------------------------ tensor memory (TMEM)
// Tensor memory holds 128 lanes x 512 columns of 32 bits per SM; warp w of a
// CTA reaches lanes 32 (w % 4) .. 32 (w % 4) + 31 (its lane quarter), so CTAs
// that use it are whole warpgroups.
__device__ __forceinline__ void tmem_alloc(uint32_t smem_dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_dst), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 27 floats of this thread into columns t .. t+26 of its lane (x16 + x8 + x2 + x1).
__device__ __forceinline__ void tmem_store27(uint32_t t, const float* v)
{
#define ELBM_R(k) "r"(__float_as_uint(v[k]))
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(t),
        ELBM_R(0), ELBM_R(1), ELBM_R(2), ELBM_R(3), ELBM_R(4), ELBM_R(5), ELBM_R(6), ELBM_R(7), ELBM_R(8), ELBM_R(9),
        ELBM_R(10), ELBM_R(11), ELBM_R(12), ELBM_R(13), ELBM_R(14), ELBM_R(15)
        : "memory");
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(t + 16),
                 ELBM_R(16), ELBM_R(17), ELBM_R(18), ELBM_R(19), ELBM_R(20), ELBM_R(21), ELBM_R(22), ELBM_R(23)
                 : "memory");
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(t + 24), ELBM_R(24), ELBM_R(25)
                 : "memory");
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(t + 26), ELBM_R(26) : "memory");
#undef ELBM_R
}
// ... and back (waits for the loads before returning the values).
__device__ __forceinline__ void tmem_load27(uint32_t t, float* v)
{
    uint32_t r[27];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(t)
        : "memory");
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
                   "=r"(r[23])
                 : "r"(t + 16)
                 : "memory");
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(r[24]), "=r"(r[25]) : "r"(t + 24)
                 : "memory");
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r[26]) : "r"(t + 26) : "memory");
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 27; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory layout (byte offsets from a 128-byte aligned base).  TMA
// destinations start on 128-byte boundaries.
template <int ST>
struct TmaLayout {
    using T = typename Storage<ST>::T;
    static constexpr int es = (int)sizeof(T);
    static constexpr int tile_bytes = 27 * kTileY * kTileX * es;     // one plane of the tile
    static constexpr int row_box_bytes = 27 * kTileX * es;           // one ring row, all populations
    static constexpr int row_stride = (row_box_bytes + 127) / 128 * 128;
    static constexpr int cols_bytes = 27 * 2 * kTileY * 4;           // ring columns as 4-byte words
    static constexpr int qx_bytes = kTileY * (kTileX + 2) * 4;
    static constexpr int qy_bytes = (kTileY + 2) * kTileX * 4;
    static constexpr int off_tile = 0;                               // [3] planes
    static constexpr int off_rows = off_tile + 3 * tile_bytes;       // [2 slots][2 sides]
    static constexpr int off_cols = off_rows + 4 * row_stride;       // [2 slots]
    static constexpr int off_qx = off_cols + 2 * cols_bytes;         // [kTmaQSlots]
    static constexpr int off_qy = off_qx + kTmaQSlots * qx_bytes;
    static constexpr int off_bar = (off_qy + kTmaQSlots * qy_bytes + 7) / 8 * 8;
    // barriers: full_t[3], empty_t[3], full_r[2], empty_r[2], qready[kTmaQSlots], then the abort flag
    static constexpr int nbar = 10 + kTmaQSlots;
    static constexpr int off_abort = off_bar + 8 * nbar;
    static constexpr int bytes = off_abort + 16 + 128;               // + slack for aligning the base
    static_assert(tile_bytes % 128 == 0, "tile boxes must keep 128-byte alignment");
};

// One tile column of a single-pass step: the 32 x 8 columns at (x0, y0),
// planes z0 .. z1-1, from p.f into dst; every thread of the block takes part.
// tm_tile / tm_row are the tensor maps (8-row tile box) of p.f, kernel
// parameters or device memory made visible to the tensor-map proxy.
template <int ST>
__device__ __forceinline__ void tma_tile_step(const CUtensorMap* tm_tile, const CUtensorMap* tm_row,
                                              const StepParams& p, void* dst, int x0, int y0, int z0, int z1,
                                              unsigned char* smem_raw)
{
    using S = Storage<ST>;
    using T = typename S::T;
    using L = TmaLayout<ST>;
    const uint32_t raw_addr = smem_u32(smem_raw);
    const uint32_t sbase = (raw_addr + 127u) & ~127u;
    unsigned char* base = smem_raw + (sbase - raw_addr);
    const uint32_t bar0 = sbase + L::off_bar;
    auto full_t = [&](int b) { return bar0 + 8u * b; };
    auto empty_t = [&](int b) { return bar0 + 8u * (3 + b); };
    auto full_r = [&](int r) { return bar0 + 8u * (6 + r); };
    auto empty_r = [&](int r) { return bar0 + 8u * (8 + r); };
    auto qready = [&](int s) { return bar0 + 8u * (10 + s); };
    volatile int* abort_flag = reinterpret_cast<volatile int*>(base + L::off_abort);

    const int K = (z1 - z0) + 2;  // planes z0-1 .. z1
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int b = 0; b < 3; ++b) {
            mbar_init(full_t(b), 1);
            mbar_init(empty_t(b), kBlock);
        }
        for (int r = 0; r < 2; ++r) {
            mbar_init(full_r(r), 1 + 32);  // producer lane 0 (expect_tx) + 32 cp.async arrivals
            mbar_init(empty_r(r), kBlock);
        }
        for (int s = 0; s < kTmaQSlots; ++s) mbar_init(qready(s), kBlock);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // bounded in time (kTmaWaitNs), or as soon as another thread of the block gave up
    auto wait = [&](uint32_t bar, unsigned parity) { return bounded_wait(bar, parity, abort_flag, p.status, kTmaWaitNs); };
    auto drain = [&](uint32_t bar, unsigned parity) { bounded_drain(bar, parity, kTmaWaitNs); };
    auto plane_of = [&](int k) { return wrapi(z0 - 1 + k, p.nz); };

    if (warp == kBlock / 32) {
        // ------------------------------------------------------ producer
        // ring column node kk: x0-1 (kk < 8) or x0+32 (kk >= 8), row y0 + (kk & 7)
        const int ylo = wrapi(y0 - 1, p.ny), yhi = wrapi(y0 + kTileY, p.ny);
        int issued = 0;
        for (int k = 0; k < K; ++k) {
            const int b = k % 3, r = k & 1;
            if (k >= 3 && !wait(empty_t(b), ((k / 3) - 1) & 1)) break;
            if (k >= 2 && !wait(empty_r(r), ((k / 2) - 1) & 1)) break;
            const int zk = plane_of(k);
            if (lane == 0) {
                mbar_arrive_expect_tx(full_t(b), L::tile_bytes);
                tma_load_4d(sbase + L::off_tile + b * L::tile_bytes, tm_tile, x0, y0, zk, 0, full_t(b));
                mbar_arrive_expect_tx(full_r(r), 2 * L::row_box_bytes);
                tma_load_4d(sbase + L::off_rows + (2 * r) * L::row_stride, tm_row, x0, ylo, zk, 0, full_r(r));
                tma_load_4d(sbase + L::off_rows + (2 * r + 1) * L::row_stride, tm_row, x0, yhi, zk, 0, full_r(r));
            }
            unsigned* cols = reinterpret_cast<unsigned*>(base + L::off_cols + r * L::cols_bytes);
            for (int c = lane; c < 27 * 2 * kTileY; c += 32) {
                const int i = c / (2 * kTileY), kk = c % (2 * kTileY);
                const int cx = kk < kTileY ? wrapi(x0 - 1, p.nx) : wrapi(x0 + kTileX, p.nx);
                const int idx = i * p.N + zk * p.plane + (y0 + (kk & (kTileY - 1))) * p.nx + cx;
                cp_async4(cols + c, stage_src<ST>(p, idx));
            }
            cp_async_mbar_arrive(full_r(r));
            issued = k + 1;
        }
        cp_async_wait_all();
        // no bulk copy may still be in flight when the block retires
        for (int k = max(0, issued - 3); k < issued; ++k) drain(full_t(k % 3), (k / 3) & 1);
        for (int k = max(0, issued - 2); k < issued; ++k) drain(full_r(k & 1), (k / 2) & 1);
        return;
    }

    // ---------------------------------------------------------- consumers
    const int tx = lane, ty = warp;
    const int gx = x0 + tx, gy = y0 + ty;
    const T* tile = reinterpret_cast<const T*>(base + L::off_tile);
    float* qxs = reinterpret_cast<float*>(base + L::off_qx);
    float* qys = reinterpret_cast<float*>(base + L::off_qy);
    auto QX = [&](int s, int y, int x) -> float& { return qxs[(s * kTileY + y) * (kTileX + 2) + x]; };
    auto QY = [&](int s, int y, int x) -> float& { return qys[(s * (kTileY + 2) + y) * kTileX + x]; };
    auto anomaly_of = [&](auto&& gval, float* q) {
        float drho, j[3];
        moments_of<3>(p, gval, drho, j);
        const float inv_rho = 1.0f / (p.rho_ref + drho);
#pragma unroll
        for (int a = 0; a < 3; ++a) q[a] = anomaly(p, a, j[a], j[a] * inv_rho);
    };
    T* out = static_cast<T*>(dst);
    const int xo[3] = {gx == 0 ? p.nx - 1 : gx - 1, gx, gx == p.nx - 1 ? 0 : gx + 1};
    const int yo[3] = {(gy == 0 ? p.ny - 1 : gy - 1) * p.nx, gy * p.nx, (gy == p.ny - 1 ? 0 : gy + 1) * p.nx};
    constexpr int kPlaneElems = kTileY * kTileX;  // stride between populations in a tile buffer

    float qz_prev = 0.f, qz_cur = 0.f;
    for (int k = 0; k < K; ++k) {
        const int b = k % 3, r = k & 1, s = k % kTmaQSlots;
        if (!wait(full_t(b), (k / 3) & 1)) return;
        if (!wait(full_r(r), (k / 2) & 1)) return;
        // anomaly of the own node of plane k
        const T* own = tile + b * 27 * kPlaneElems + ty * kTileX + tx;
        float q[3];
        anomaly_of([&](int i) { return raw_value<ST>(p, own[i * kPlaneElems], i); }, q);
        QX(s, ty, tx + 1) = q[0];
        QY(s, ty + 1, tx) = q[1];
        // ring share of this warp for plane k (duty rotates with k): 0 the row
        // below the tile, 1 the row above, 2 the two columns (lanes 0..15)
        const int duty = (ty + k) & 7;
        if (k > 0 && k < K - 1) {
            if (duty < 2) {
                const T* row = reinterpret_cast<const T*>(base + L::off_rows + (2 * r + duty) * L::row_stride) + tx;
                float qh[3];
                anomaly_of([&](int i) { return raw_value<ST>(p, row[i * kTileX], i); }, qh);
                QY(s, duty ? kTileY + 1 : 0, tx) = qh[1];
            } else if (duty == 2 && tx < 2 * kTileY) {
                const unsigned* cols = reinterpret_cast<const unsigned*>(base + L::off_cols + r * L::cols_bytes) + tx;
                const int cx = tx < kTileY ? wrapi(x0 - 1, p.nx) : wrapi(x0 + kTileX, p.nx);
                const int idx0 = plane_of(k) * p.plane + (y0 + (tx & (kTileY - 1))) * p.nx + cx;
                float qh[3];
                anomaly_of([&](int i) { return stage_value<ST>(p, cols[i * 2 * kTileY], (i * p.N + idx0) & 1, i); },
                           qh);
                QX(s, tx & (kTileY - 1), tx < kTileY ? 0 : kTileX + 1) = qh[0];
            }
        }
        mbar_arrive(empty_r(r));
        mbar_arrive(qready(s));
        if (k == 0) {
            qz_prev = q[2];
            mbar_arrive(empty_t(b));
            continue;
        }
        if (k == 1) {
            qz_cur = q[2];
            continue;
        }
        // relax plane k-1 (z = z0 + k - 2) once every warp has published its anomaly
        const float qz_next = q[2];
        const int kc = k - 1, bc = kc % 3, sc = kc % kTmaQSlots;
        if (!wait(qready(sc), (kc / kTmaQSlots) & 1)) return;
        const T* cur = tile + bc * 27 * kPlaneElems + ty * kTileX + tx;
        float g[27];
#pragma unroll
        for (int i = 0; i < 27; ++i) g[i] = raw_value<ST>(p, cur[i * kPlaneElems], i);
        auto gval = [&](int i) { return g[i]; };
        float drho, j[3];
        moments_of<3>(p, gval, drho, j);
        float d[3] = {0.f, 0.f, 0.f};
        if (p.eq_mode == 0) {
            d[0] = (QX(sc, ty, tx + 2) - QX(sc, ty, tx)) * p.inv_2lam[0];
            d[1] = (QY(sc, ty + 2, tx) - QY(sc, ty, tx)) * p.inv_2lam[1];
            d[2] = (qz_next - qz_prev) * p.inv_2lam[2];
        }
        const int z = z0 + k - 2;
        const int zo[3] = {wrapi(z - 1, p.nz) * p.plane, z * p.plane, wrapi(z + 1, p.nz) * p.plane};
        auto put = [&](int i, float gn) {
            const int slot = opaque(i * p.N) + xo[cx_of(i) + 1] + yo[cy_of(i) + 1] + zo[cz_of<3>(i) + 1];
            S::store(out + slot, S::shifted ? gn : fmaf(p.bw[i], p.rho_ref, gn));
        };
        relax_streamed<3>(p, gval, put, drho, j, d);
        mbar_arrive(empty_t(bc));
        qz_prev = qz_cur;
        qz_cur = qz_next;
    }
}

// The single-pass step of one grid on 32 x 8 tiles: block (bx, by, bz) takes
// the tile column at (32 bx, 8 by), planes kSegPlanes bz onwards.
template <int ST>
__global__ void __launch_bounds__(kTmaThreads, 2)
    k_single_pass_tma(const __grid_constant__ CUtensorMap tm_tile, const __grid_constant__ CUtensorMap tm_row,
                      const __grid_constant__ StepParams p, void* dst)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int z0 = blockIdx.z * kSegPlanes;
    tma_tile_step<ST>(&tm_tile, &tm_row, p, dst, blockIdx.x * kTileX, blockIdx.y * kTileY, z0,
                      min(p.nz, z0 + kSegPlanes), smem_raw);
}

// TMA needs 16-byte aligned rows and whole tiles: nx a multiple of 32, ny a
// multiple of 8 (the fast path's condition) and 16-byte aligned arrays.
template <int ST>
bool single_tma_ok(const Solver& s, const void* src, const void* dst)
{
    return single_fast_ok<ST>(s) && ((uintptr_t)src % 16 == 0) && ((uintptr_t)dst % 16 == 0);
}

// Tensor maps of one population array: dims (x, y, z, population), boxes of
// the tile (32 x tile_y x 1 x 27) and of one ring row (32 x 1 x 1 x 27);
// cached in the solver per array and tile height.
cudaError_t encode_population_maps(const Solver& s, const void* f, int tile_y, CUtensorMap* tile, CUtensorMap* row);

// Raise kernel K's dynamic shared-memory limit to `bytes`, once per device
// and process.
template <auto K>
cudaError_t set_smem_limit_once(int bytes)
{
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

template <int ST>
cudaError_t launch_single_tma(const Solver& s, const StepParams& p, void* dst, bool* launched)
{
    *launched = false;
    if (!single_tma_ok<ST>(s, p.f, dst)) return cudaSuccess;
    CUtensorMap tm_tile, tm_row;
    cudaError_t e = encode_population_maps(s, p.f, kTileY, &tm_tile, &tm_row);
    if (e != cudaSuccess) return cudaSuccess;  // no TMA: the caller takes another single-pass kernel
    const int smem = TmaLayout<ST>::bytes;
    e = set_smem_limit_once<k_single_pass_tma<ST>>(smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)(s.nx / kTileX), (unsigned)(s.ny / kTileY),
                    (unsigned)((s.nz + kSegPlanes - 1) / kSegPlanes));
    k_single_pass_tma<ST><<<grid, kTmaThreads, smem, s.stream>>>(tm_tile, tm_row, p, dst);
    *launched = true;
    return cudaGetLastError();
}

}  // namespace elbm
