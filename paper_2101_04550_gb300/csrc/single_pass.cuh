// Single-pass form of the extended LBGK step with two population arrays.
//
// The correction term needs the anomaly Q~_aaa of the face neighbours at the
// same time level (Eq. Paastar1).  With a read-only source array and a
// separate destination, every block can recompute the anomaly of the nodes
// around its own tile, so one pass and one read of the populations suffice.
//
// State: `src` holds the post-streaming populations of every node at the
// node's own location (the layout of the in-place form's even parity).  A step
// reads src[i][x], relaxes, and pushes f'_i(x) to dst[i][x + c_i] (Eq. LBGK);
// then the arrays swap roles.
//
// Geometry (D3Q27): a block of kBlock = 256 threads owns a tile of 32 x 8
// columns and marches through a segment of kSegPlanes z planes.  Per plane k
// it (1) requests, with cp.async, the populations of plane k+2 of its tile and
// of the 80-node ring around it (2 columns x 8 and 2 rows x 32) into shared
// memory, (2) waits for the copies of plane k+1 (requested one plane earlier)
// and computes the anomaly of those nodes -- x and y components into a 3-deep
// ring of plane buffers with a one-node halo, the z component of its own node
// into a register, (3) after one barrier relaxes the nodes of plane k, whose
// populations were staged two planes earlier, using the anomaly of plane k
// (x, y differences) and of planes k-1, k+1 (z difference), while the copies
// of plane k+2 are in flight.  Threads whose column lies beyond a ragged grid
// edge take the periodic image of their position: they supply the anomaly of
// the wrapped node and relax nothing.
#pragma once
#include <utility>
#include "step_kernels.cuh"

namespace elbm {

constexpr int kTileX = 32, kTileY = 8;   // kTileX * kTileY == kBlock
constexpr int kHalo = 2 * kTileX + 2 * kTileY;
constexpr int kSegPlanes = 32;

#ifndef ELBM_SINGLE_MIN_BLOCKS
#define ELBM_SINGLE_MIN_BLOCKS 2
#endif

// Stages hold raw storage words: the tile as [i][ty][tx] elements (rows
// copied in 16-byte pieces when rows are 16-byte aligned), the ring as one
// 4-byte word per population and node.
struct SingleSmem {
    unsigned stage[3][27][kBlock];         // populations of the tile, planes k, k+1, k+2 (ring)
    unsigned halo_stage[2][27][kHalo];     // populations of the ring, planes k+1, k+2
    float qx[3][kTileY][kTileX + 2];       // Q~_xxx with an x halo, planes k, k+1, k+2 (ring)
    float qy[3][kTileY + 2][kTileX];       // Q~_yyy with a y halo
};

// Anomaly components of a node whose 27 populations were staged with stride
// `stride` (the sums of moments(), then Eq. Deviation).
template <int ST>
__device__ __forceinline__ void staged_anomaly(const StepParams& p, const unsigned* col, int stride,
                                               unsigned halves, float* q)
{
    auto gval = [&](int i) { return stage_value<ST>(p, ld_stage(col + i * stride), (int)((halves >> i) & 1u), i); };
    float drho, j[3];
    moments_of<3>(p, gval, drho, j);
    const float inv_rho = 1.0f / (p.rho_ref + drho);
#pragma unroll
    for (int a = 0; a < 3; ++a) q[a] = anomaly(p, a, j[a], j[a] * inv_rho);
}

// Issue the cp.async copies of the 27 own-location populations of node `cell`
// into a staged column; returns the half-word selector bits.
template <int ST>
__device__ __forceinline__ unsigned stage_node(const StepParams& p, int cell, unsigned* col, int stride)
{
    unsigned halves = 0;
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        const int idx = i * p.N + cell;
        halves |= (unsigned)(idx & 1) << i;
        cp_async4(col + i * stride, stage_src<ST>(p, idx));
    }
    return halves;
}

// Programmatic dependent launch.  A kernel launched after this one with the
// programmatic-serialization attribute may be scheduled once every block of
// this one has signalled (pdl_release, at the top of the kernel); its blocks
// run their prologue and then stop in pdl_wait until this kernel has finished
// and its memory operations are visible.  Without the attribute pdl_wait
// returns at once.
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch `kernel` with the programmatic-serialization attribute (outside a
// stream capture; inside one, as an ordinary launch).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = cap == cudaStreamCaptureStatusNone ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
__device__ __forceinline__ int modi(int v, int n) { return ((v % n) + n) % n; }

template <int ST>
__global__ void __launch_bounds__(kBlock, ELBM_SINGLE_MIN_BLOCKS) k_single_pass(StepParams p, void* dst)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SingleSmem& sm = *reinterpret_cast<SingleSmem*>(smem_raw);
    using S = Storage<ST>;
    const int tx = threadIdx.x & (kTileX - 1), ty = threadIdx.x / kTileX;
    const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * kTileY;
    const int z0 = blockIdx.z * kSegPlanes;
    const int z1 = min(p.nz, z0 + kSegPlanes);
    const bool active = (x0 + tx < p.nx) && (y0 + ty < p.ny);
    const int gx = modi(x0 + tx, p.nx), gy = modi(y0 + ty, p.ny);  // periodic image beyond a ragged edge
    const int col_off = gx + gy * p.nx;

    // ring node handled by this thread (threads 0 .. kHalo-1): rows y0-1 and
    // y0+kTileY for the y anomaly, columns x0-1 and x0+kTileX for the x anomaly
    int hx = 0, hy = 0, hslot = -1;
    if (threadIdx.x < 2 * kTileX) {
        hx = x0 + (threadIdx.x & (kTileX - 1));
        hy = (threadIdx.x < kTileX) ? y0 - 1 : y0 + kTileY;
        hslot = threadIdx.x;
    } else if (threadIdx.x < kHalo) {
        const int k = threadIdx.x - 2 * kTileX;
        hx = (k < kTileY) ? x0 - 1 : x0 + kTileX;
        hy = y0 + (k & (kTileY - 1));
        hslot = threadIdx.x;
    }
    const int h_off = modi(hx, p.nx) + modi(hy, p.ny) * p.nx;

    auto plane_of = [&](int z) { return wrapi(z, p.nz) * p.plane; };
    auto tile_halves = [&](int z) {
        const int idx0 = plane_of(z) + col_off;
        unsigned h = 0;
#pragma unroll
        for (int i = 0; i < 27; ++i) h |= (unsigned)((i * p.N + idx0) & 1) << i;
        return h;
    };
    auto ring_halves = [&](int z) {
        const int idx0 = plane_of(z) + h_off;
        unsigned h = 0;
#pragma unroll
        for (int i = 0; i < 27; ++i) h |= (unsigned)((i * p.N + idx0) & 1) << i;
        return h;
    };
    // request plane z of the tile (into stage[b]) and of the ring (halo_stage[hb])
    auto request_plane = [&](int z, int b, int hb) {
        const int base = plane_of(z);
        stage_node<ST>(p, base + col_off, &sm.stage[b][0][threadIdx.x], kBlock);
        if (hslot >= 0) stage_node<ST>(p, base + h_off, &sm.halo_stage[hb][0][hslot], kHalo);
        cp_async_commit();
    };
    // anomaly of the staged plane z into ring slot qs; returns this thread's Q~_zzz
    auto anomaly_plane = [&](int z, int b, int hb, int qs) -> float {
        float q[3];
        staged_anomaly<ST>(p, &sm.stage[b][0][threadIdx.x], kBlock, tile_halves(z), q);
        sm.qx[qs][ty][tx + 1] = q[0];
        sm.qy[qs][ty + 1][tx] = q[1];
        if (hslot >= 0) {
            float qh[3];
            staged_anomaly<ST>(p, &sm.halo_stage[hb][0][hslot], kHalo, ring_halves(z), qh);
            if (hslot < kTileX) sm.qy[qs][0][hslot] = qh[1];
            else if (hslot < 2 * kTileX) sm.qy[qs][kTileY + 1][hslot - kTileX] = qh[1];
            else {
                const int k = hslot - 2 * kTileX;
                if (k < kTileY) sm.qx[qs][k][0] = qh[0];
                else sm.qx[qs][k - kTileY][kTileX + 1] = qh[0];
            }
        }
        return q[2];
    };

    // prologue: Q~_zzz of plane z0-1 (own column only), everything of plane
    // z0, and the request of plane z0+1
    float qz_prev;
    {
        stage_node<ST>(p, plane_of(z0 - 1) + col_off, &sm.stage[2][0][threadIdx.x], kBlock);
        cp_async_wait_all();
        float q[3];
        staged_anomaly<ST>(p, &sm.stage[2][0][threadIdx.x], kBlock, tile_halves(z0 - 1), q);
        qz_prev = q[2];
    }
    request_plane(z0, 0, 0);
    request_plane(z0 + 1, 1, 1);
    cp_async_wait_prior();
    float qz_cur = anomaly_plane(z0, 0, 0, 0);

    typename S::T* out = static_cast<typename S::T*>(dst);
    for (int z = z0, m = 0; z < z1; ++z, ++m) {
        const int b = m % 3, qs = m % 3;
        // request plane z+2, then finish plane z+1 (requested one plane ago)
        request_plane(z + 2, (m + 2) % 3, m & 1);
        cp_async_wait_prior();
        const float qz_next = anomaly_plane(z + 1, (m + 1) % 3, (m + 1) & 1, (m + 1) % 3);
        const unsigned cur_halves = tile_halves(z);
        __syncthreads();
        if (active) {
            // relax node (gx, gy, z) from stage[b]
            const unsigned* col = &sm.stage[b][0][threadIdx.x];
            auto gval = [&](int i) {
                return stage_value<ST>(p, ld_stage(col + i * kBlock), (int)((cur_halves >> i) & 1u), i);
            };
            float drho, j[3];
            moments_of<3>(p, gval, drho, j);
            float d[3] = {0.f, 0.f, 0.f};
            if (p.eq_mode == 0) {
                d[0] = (sm.qx[qs][ty][tx + 2] - sm.qx[qs][ty][tx]) * p.inv_2lam[0];
                d[1] = (sm.qy[qs][ty + 2][tx] - sm.qy[qs][ty][tx]) * p.inv_2lam[1];
                d[2] = (qz_next - qz_prev) * p.inv_2lam[2];
            }
            // push targets: node (gx + cx, gy + cy, z + cz), periodic
            const int xo[3] = {gx == 0 ? p.nx - 1 : gx - 1, gx, gx == p.nx - 1 ? 0 : gx + 1};
            const int yo[3] = {(gy == 0 ? p.ny - 1 : gy - 1) * p.nx, gy * p.nx, (gy == p.ny - 1 ? 0 : gy + 1) * p.nx};
            const int zo[3] = {plane_of(z - 1), plane_of(z), plane_of(z + 1)};
            auto put = [&](int i, float gn) {
                const int slot = opaque(i * p.N) + xo[cx_of(i) + 1] + yo[cy_of(i) + 1] + zo[cz_of<3>(i) + 1];
                S::store(out + slot, S::shifted ? gn : fmaf(p.bw[i], p.rho_ref, gn));
            };
            relax_streamed<3>(p, gval, put, drho, j, d);
        }
        qz_prev = qz_cur;
        qz_cur = qz_next;
    }
    cp_async_wait_all();
}

// ---------------------------------------------------------------- fast path
// Grids with nx a multiple of 32, ny a multiple of 8 and 16-byte aligned rows
// (nx * sizeof(storage) a multiple of 16): the tile (32 x 8 nodes) and the two
// ring rows are copied in 16-byte pieces of raw storage elements, the two ring
// columns (8 nodes each) as the 4-byte words that contain them.  Each thread
// reads its node's 27 populations back once, into registers.
template <int ST>
struct FastSmem {
    using T = typename Storage<ST>::T;
    T tile[3][27][kTileY][kTileX];        // planes k, k+1, k+2 (ring of buffers)
    T rows[2][2][27][kTileX];             // ring rows y0-1, y0+8; planes k+1, k+2
    unsigned cols[2][27][2 * kTileY];     // ring columns x0-1, x0+32 (words); planes k+1, k+2
    float qx[3][kTileY][kTileX + 2];
    float qy[3][kTileY + 2][kTileX];
};

template <int ST>
__device__ __forceinline__ float raw_value(const StepParams& p, typename Storage<ST>::T v, int i)
{
    using S = Storage<ST>;
    const float f = S::load(&v);
    return S::shifted ? f : f - p.bw[i] * p.rho_ref;
}

template <int ST>
__global__ void __launch_bounds__(kBlock, ELBM_SINGLE_MIN_BLOCKS) k_single_pass_fast(StepParams p, void* dst)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using S = Storage<ST>;
    using T = typename S::T;
    FastSmem<ST>& sm = *reinterpret_cast<FastSmem<ST>*>(smem_raw);
    constexpr int EPC = 16 / (int)sizeof(T);   // elements per 16-byte piece
    constexpr int PPR = kTileX / EPC;          // pieces per tile row
    const int tx = threadIdx.x & (kTileX - 1), ty = threadIdx.x / kTileX;
    const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * kTileY;
    const int z0 = blockIdx.z * kSegPlanes;
    const int z1 = min(p.nz, z0 + kSegPlanes);
    const int gx = x0 + tx, gy = y0 + ty;
    const int row_lo = wrapi(y0 - 1, p.ny) * p.nx + x0, row_hi = wrapi(y0 + kTileY, p.ny) * p.nx + x0;
    const T* f = static_cast<const T*>(p.f);
    // ring column node of threads 0..15: x0-1 (k < 8) or x0+32 (k >= 8), row y0 + (k & 7)
    const int ck = threadIdx.x;
    const int c_off = (ck < 2 * kTileY)
                          ? wrapi(ck < kTileY ? x0 - 1 : x0 + kTileX, p.nx) + (y0 + (ck & (kTileY - 1))) * p.nx
                          : 0;
    auto plane_of = [&](int z) { return wrapi(z, p.nz) * p.plane; };

    auto request_plane = [&](int z, int b, int hb) {
        const int base = plane_of(z);
        for (int c = threadIdx.x; c < 27 * kTileY * PPR; c += kBlock) {
            const int i = c / (kTileY * PPR), r = (c / PPR) % kTileY, q = c % PPR;
            cp_async16(&sm.tile[b][i][r][q * EPC], f + i * p.N + base + (y0 + r) * p.nx + x0 + q * EPC);
        }
        for (int c = threadIdx.x; c < 2 * 27 * PPR; c += kBlock) {
            const int side = c / (27 * PPR), i = (c / PPR) % 27, q = c % PPR;
            cp_async16(&sm.rows[hb][side][i][q * EPC], f + i * p.N + base + (side ? row_hi : row_lo) + q * EPC);
        }
        if (ck < 2 * kTileY) {
#pragma unroll
            for (int i = 0; i < 27; ++i) cp_async4(&sm.cols[hb][i][ck], stage_src<ST>(p, i * p.N + base + c_off));
        }
        cp_async_commit();
    };
    auto anomaly_from = [&](auto&& gval, float* q) {
        float drho, j[3];
        moments_of<3>(p, gval, drho, j);
        const float inv_rho = 1.0f / (p.rho_ref + drho);
#pragma unroll
        for (int a = 0; a < 3; ++a) q[a] = anomaly(p, a, j[a], j[a] * inv_rho);
    };
    auto anomaly_plane = [&](int z, int b, int hb, int qs) -> float {
        float q[3];
        anomaly_from([&](int i) { return raw_value<ST>(p, sm.tile[b][i][ty][tx], i); }, q);
        sm.qx[qs][ty][tx + 1] = q[0];
        sm.qy[qs][ty + 1][tx] = q[1];
        if (threadIdx.x < 2 * kTileX) {  // ring rows: the y anomaly
            const int side = threadIdx.x / kTileX, x = threadIdx.x & (kTileX - 1);
            float qh[3];
            anomaly_from([&](int i) { return raw_value<ST>(p, sm.rows[hb][side][i][x], i); }, qh);
            sm.qy[qs][side ? kTileY + 1 : 0][x] = qh[1];
        } else if (threadIdx.x >= kBlock - 2 * kTileY) {  // ring columns: the x anomaly
            const int k = threadIdx.x - (kBlock - 2 * kTileY);
            const int idx = plane_of(z) + (k < kTileY ? wrapi(x0 - 1, p.nx) : wrapi(x0 + kTileX, p.nx)) +
                            (y0 + (k & (kTileY - 1))) * p.nx;
            float qh[3];
            anomaly_from([&](int i) { return stage_value<ST>(p, sm.cols[hb][i][k], (i * p.N + idx) & 1, i); }, qh);
            sm.qx[qs][k & (kTileY - 1)][k < kTileY ? 0 : kTileX + 1] = qh[0];
        }
        return q[2];
    };

    float qz_prev;
    request_plane(z0 - 1, 2, 0);
    cp_async_wait_all();
    __syncthreads();  // pieces staged by other threads are visible
    {
        float q[3];
        anomaly_from([&](int i) { return raw_value<ST>(p, sm.tile[2][i][ty][tx], i); }, q);
        qz_prev = q[2];
    }
    __syncthreads();  // ring buffers of plane z0-1 are reused below
    request_plane(z0, 0, 0);
    request_plane(z0 + 1, 1, 1);
    cp_async_wait_prior();
    __syncthreads();
    float qz_cur = anomaly_plane(z0, 0, 0, 0);

    T* out = static_cast<T*>(dst);
    for (int z = z0, m = 0; z < z1; ++z, ++m) {
        const int b = m % 3, qs = m % 3;
        __syncthreads();  // every thread is done with the buffers about to be refilled
        request_plane(z + 2, (m + 2) % 3, m & 1);
        cp_async_wait_prior();
        __syncthreads();  // plane z+1 staged by all threads
        const float qz_next = anomaly_plane(z + 1, (m + 1) % 3, (m + 1) & 1, (m + 1) % 3);
        __syncthreads();  // anomaly of plane z+1 complete
        float g[27];
#pragma unroll
        for (int i = 0; i < 27; ++i) g[i] = raw_value<ST>(p, sm.tile[b][i][ty][tx], i);
        auto gval = [&](int i) { return g[i]; };
        float drho, j[3];
        moments_of<3>(p, gval, drho, j);
        float d[3] = {0.f, 0.f, 0.f};
        if (p.eq_mode == 0) {
            d[0] = (sm.qx[qs][ty][tx + 2] - sm.qx[qs][ty][tx]) * p.inv_2lam[0];
            d[1] = (sm.qy[qs][ty + 2][tx] - sm.qy[qs][ty][tx]) * p.inv_2lam[1];
            d[2] = (qz_next - qz_prev) * p.inv_2lam[2];
        }
        const int xo[3] = {gx == 0 ? p.nx - 1 : gx - 1, gx, gx == p.nx - 1 ? 0 : gx + 1};
        const int yo[3] = {(gy == 0 ? p.ny - 1 : gy - 1) * p.nx, gy * p.nx, (gy == p.ny - 1 ? 0 : gy + 1) * p.nx};
        const int zo[3] = {plane_of(z - 1), plane_of(z), plane_of(z + 1)};
        auto put = [&](int i, float gn) {
            const int slot = opaque(i * p.N) + xo[cx_of(i) + 1] + yo[cy_of(i) + 1] + zo[cz_of<3>(i) + 1];
            S::store(out + slot, S::shifted ? gn : fmaf(p.bw[i], p.rho_ref, gn));
        };
        relax_streamed<3>(p, gval, put, drho, j, d);
        qz_prev = qz_cur;
        qz_cur = qz_next;
    }
    cp_async_wait_all();
}

template <int ST>
bool single_fast_ok(const Solver& s)
{
    using T = typename Storage<ST>::T;
    return s.nx % kTileX == 0 && s.ny % kTileY == 0 && (s.nx * (int)sizeof(T)) % 16 == 0;
}

inline size_t single_pass_smem() { return sizeof(SingleSmem); }

}  // namespace elbm
