// Kernels of the extended LBGK step and its utilities, templated on the
// lattice dimension D, the storage mode ST and (for the hot kernels) the AA
// streaming parity PAR.  Included by one translation unit per lattice.
#pragma once
#include <type_traits>
#include <cfloat>

#include "lbm_device.cuh"

namespace elbm {

constexpr int kBlock = 256;

// Resident blocks per SM the collide kernels are compiled for.
#ifndef ELBM_COLLIDE_MIN_BLOCKS
#define ELBM_COLLIDE_MIN_BLOCKS 4
#endif

#define ELBM_DISPATCH_STORAGE(storage, ...)                              \
    switch (storage) {                                                   \
        case ELBM_F32: { constexpr int ST = ELBM_F32; __VA_ARGS__; } break;             \
        case ELBM_F32_SHIFT: { constexpr int ST = ELBM_F32_SHIFT; __VA_ARGS__; } break; \
        case ELBM_F16_SHIFT: { constexpr int ST = ELBM_F16_SHIFT; __VA_ARGS__; } break; \
        case ELBM_BF16_SHIFT: { constexpr int ST = ELBM_BF16_SHIFT; __VA_ARGS__; } break; \
        default: return cudaErrorInvalidValue;                           \
    }

// ---------------------------------------------------------------- two-pass
// Pass 1: post-streaming moments of every node -> anomaly field q[a][cell]
// (Eqs. density, momentum, Deviation).  Reads the populations only.  BC: the
// variant that honours walls (p.walls_y) and the body force (p.forced).
template <int D, int ST, int PAR, bool BC = false>
__global__ void __launch_bounds__(kBlock) k_anomaly(StepParams p)
{
    const int cell = blockIdx.x * kBlock + threadIdx.x;
    if (cell >= p.N) return;
    const Node n = make_node<D>(p, cell);
    float g[Lat<D>::Q];
    gather<D, ST, PAR>(p, n, g, BC && p.walls_y);
    float drho, j[3];
    moments<D>(p, g, drho, j);
    const float inv_rho = 1.0f / (p.rho_ref + drho);
#pragma unroll
    for (int a = 0; a < D; ++a) p.q[a * p.N + cell] = anomaly(p, a, j[a], j[a] * inv_rho);
}

// Moments of a node from a population accessor gval(i) (the sums of moments()).
template <int D, typename G>
__device__ __forceinline__ void moments_of(const StepParams& p, G&& gval, float& drho, float* j)
{
    // lines of three along x (population index x fastest), then rows along y, then planes along z
    constexpr int NL = Lat<D>::Q / 3, NP = NL / 3 > 0 ? NL / 3 : 1;
    float t[NL], sx = 0.f, sy = 0.f;
#pragma unroll
    for (int L = 0; L < NL; ++L) {
        const float a = gval(3 * L), b = gval(3 * L + 1), c = gval(3 * L + 2);
        t[L] = (a + b) + c;
        sx += c - a;
    }
    float tp[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int P = 0; P < NP; ++P) {
        tp[P] = (t[3 * P] + t[3 * P + 1]) + t[3 * P + 2];
        sy += t[3 * P + 2] - t[3 * P];
    }
    drho = (D == 3) ? (tp[0] + tp[1]) + tp[2] : tp[0];
    const float sz = (D == 3) ? tp[2] - tp[0] : 0.f;
    j[0] = fmaf(p.lam[0], sx, p.j0[0]);
    j[1] = fmaf(p.lam[1], sy, p.j0[1]);
    j[2] = (D == 3) ? fmaf(p.lam[2], sz, p.j0[2]) : 0.f;
}

// Relaxation of one node toward the extended equilibrium with the
// conservation correction of relax(), for populations read through gval(i)
// (read twice, not kept in registers) and results handed to put(i, g'_i).
// POLY selects the conventional second-order equilibrium instead.  BC adds
// the body-force increment F_i (ForceIncrement) when p.forced is set; it is
// kept out of the conservation moments, so the node gains exactly the
// momentum rho g of the force.  FX: the force is known to act along x alone
// (ForceIncrementX, same bits, fewer registers).  inv_rho, if given (> 0),
// is the caller's 1 / (rho_ref + drho), the very value computed here otherwise.
template <int D, bool POLY = false, bool BC = false, bool FX = false, typename G, typename P>
__device__ __forceinline__ void relax_streamed(const StepParams& p, G&& gval, P&& put, float drho,
                                               const float* j, const float* d, float inv_rho_in = 0.f)
{
    constexpr int I0 = (Lat<D>::Q - 1) / 2;
    const float rho = p.rho_ref + drho;
    const float inv_rho = inv_rho_in > 0.f ? inv_rho_in : 1.0f / rho;
    float u[3], pcorr[3], du[3], dP[3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        u[a] = __fmul_rn(j[a], inv_rho);
        pcorr[a] = __fmul_rn(__fmul_rn(p.coef, inv_rho), d[a]);
    }
    baseline_args<D>(p, u, pcorr, du, dP);
    const float om = p.omega;
    const bool forced = BC && p.forced;
    typename std::conditional<FX, ForceIncrementX<D>, ForceIncrement<D>>::type frc;
    if (forced) frc.init(p, rho / om, u);
    float e0 = 0.f, ex = 0.f, ey = 0.f, ez = 0.f;
    float keep[2 * D + 1], kf[2 * D + 1];
    // the increments' moments, summed along the enumeration's lines: cz
    // innermost (D3Q27) or cx innermost (D2Q9), then cx, then cy
    float line[3], row[3];
    auto accumulate = [&](int i, float dl) {
        const int cx = cx_of(i), cy = cy_of(i);
        if (D == 3) {
            const int cz = cz_of<D>(i);
            line[cz + 1] = dl;
            if (cz != 1) return;
            row[cx + 1] = (line[0] + line[1]) + line[2];
            ez += line[2] - line[0];
        } else {
            row[cx + 1] = dl;
        }
        if (cx != 1) return;
        const float rs = (row[0] + row[1]) + row[2];
        ex += row[2] - row[0];
        e0 += rs;
        if (cy == 1) ey += rs;
        if (cy == -1) ey -= rs;
    };
    auto relax_one = [&](int i, float geq) {
        const float gi = gval(i);
        const float dl = __fsub_rn(geq, gi);
        accumulate(i, dl);
        const int k = corrected_slot<D>(i);
        if (k >= 0) {
            keep[k] = geq;
            if (forced) kf[k] = frc(i);
        } else {
            put(i, fmaf(om, forced ? dl + frc(i) : dl, gi));
        }
    };
    if (POLY) for_each_second_order<D>(p, drho, u, relax_one);
    else for_each_equilibrium<D>(p, drho, du, dP, relax_one);
    auto inc = [&](int k, float v) { return forced ? v + kf[k] : v; };
    const float hx = __fmul_rn(0.5f, ex), hy = __fmul_rn(0.5f, ey);
    // f*_k - f_k with the half-increment h of its axis: (keep - g) -+ h
    auto corr = [&](int k, int i, float h) { return inc(k, __fadd_rn(__fsub_rn(keep[k], gval(i)), h)); };
    put(I0, fmaf(om, inc(0, __fsub_rn(__fsub_rn(keep[0], gval(I0)), e0)), gval(I0)));
    put(I0 - 1, fmaf(om, corr(1, I0 - 1, hx), gval(I0 - 1)));
    put(I0 + 1, fmaf(om, corr(2, I0 + 1, -hx), gval(I0 + 1)));
    put(I0 - 3, fmaf(om, corr(3, I0 - 3, hy), gval(I0 - 3)));
    put(I0 + 3, fmaf(om, corr(4, I0 + 3, -hy), gval(I0 + 3)));
    if (D == 3) {
        const float hz = __fmul_rn(0.5f, ez);
        put(I0 - 9, fmaf(om, corr(5, I0 - 9, hz), gval(I0 - 9)));
        put(I0 + 9, fmaf(om, corr(6, I0 + 9, -hz), gval(I0 + 9)));
    }
}

// The per-node update once the anomaly field of this time level is complete:
// gather the post-streaming populations into the thread's shared-memory
// column `col` (stride STRIDE, the block size), central difference of q along each axis
// (Eq. Paastar1), extended equilibrium, relaxation, write-back in place.
// Populations are read back from the stage instead of being held in
// registers, which keeps the register count low enough for 32 resident
// warps per SM.  BC: walls (bounce-back slots, and the anomaly's ghost value
// beyond a wall is the negated value of the wall-adjacent node: Q~_yyy is odd
// in u_y and u_y = 0 on the wall) and the body force.
template <int D, int ST, int PAR, int STRIDE = kBlock, bool POLY = false, bool BC = false>
__device__ __forceinline__ void collide_staged(const StepParams& p, int cell, unsigned* col)
{
    constexpr int Q = Lat<D>::Q;
    using S = Storage<ST>;
    const Node n = make_node<D>(p, cell);
    const bool walls = BC && p.walls_y;
    unsigned halves = 0;  // bit i: population i sits in the upper half of its staged word
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int idx = read_slot<D>(n, p.N, i, PAR, walls);
        halves |= (unsigned)(idx & 1) << i;
        cp_async4(col + i * STRIDE, stage_src<ST>(p, idx));
    }
    float d[3] = {0.f, 0.f, 0.f};
    if (p.eq_mode == 0) {
        const float* q = p.q;
        d[0] = (q[n.at(1, 0, 0)] - q[n.at(-1, 0, 0)]) * p.inv_2lam[0];
        const float* qy = q + p.N;
        const float qyp = (walls && n.yhi) ? -qy[cell] : qy[n.at(0, 1, 0)];
        const float qym = (walls && n.ylo) ? -qy[cell] : qy[n.at(0, -1, 0)];
        d[1] = (qyp - qym) * p.inv_2lam[1];
        if (D == 3) d[2] = (q[2 * p.N + n.at(0, 0, 1)] - q[2 * p.N + n.at(0, 0, -1)]) * p.inv_2lam[2];
    }
    cp_async_wait_all();
    auto gval = [&](int i) {
        const float v = stage_value<ST>(p, ld_stage(col + i * STRIDE), (int)((halves >> i) & 1u), i);
        return (S::shifted && PAR == 1 && walls && read_bounced(n, i)) ? v + bounce_rebase<D>(p, i) : v;
    };
    float drho, j[3];
    moments_of<D>(p, gval, drho, j);
    typename S::T* f = static_cast<typename S::T*>(p.f);
    const int cell_o = opaque(cell);
    auto put = [&](int i, float gn) {
        const int slot = (PAR == 0) ? (Q - 1 - i) * p.N + cell_o : write_slot<D>(n, p.N, i, PAR, walls);
        if (S::shifted && PAR == 1 && walls && write_bounced(n, i)) gn += bounce_rebase<D>(p, Q - 1 - i);
        S::store(f + slot, S::shifted ? gn : fmaf(p.bw[i], p.rho_ref, gn));
    };
    relax_streamed<D, POLY, BC>(p, gval, put, drho, j, d);
}

// Pass 2 over every node: one node per thread, populations staged in shared
// memory.  POLY: the conventional second-order equilibrium (no anomaly pass).
// BC: walls and body force (compiled for one resident block fewer: the force
// terms need the registers).
template <int D, int ST, int PAR, bool POLY = false, bool BC = false>
__global__ void __launch_bounds__(kBlock, BC ? ELBM_COLLIDE_MIN_BLOCKS - 1 : ELBM_COLLIDE_MIN_BLOCKS) k_collide(StepParams p)
{
    __shared__ unsigned stage[Lat<D>::Q * kBlock];
    const int cell = blockIdx.x * kBlock + threadIdx.x;
    if (cell >= p.N) return;
    collide_staged<D, ST, PAR, kBlock, POLY, BC>(p, cell, stage + threadIdx.x);
}

template <int D>
cudaError_t step_two_pass_impl(const Solver& s, int parity, long long* launches)
{
    StepParams p;
    fill_params(s, p);
    p.parity = parity;
    // walls and body force: the kernels of bounded_step.cuh (own translation units)
    if (p.walls_y || p.forced) return step_bounded_impl<D>(s, parity, launches);
    const dim3 grid((unsigned)((s.N + kBlock - 1) / kBlock));
    const dim3 cgrid = grid;
    ELBM_DISPATCH_STORAGE(s.storage, {
        if (p.eq_mode == 2) {
            if (parity == 0) k_collide<D, ST, 0, true><<<cgrid, kBlock, 0, s.stream>>>(p);
            else k_collide<D, ST, 1, true><<<cgrid, kBlock, 0, s.stream>>>(p);
        } else if (parity == 0) {
            if (p.eq_mode == 0) { k_anomaly<D, ST, 0><<<grid, kBlock, 0, s.stream>>>(p); ++*launches; }
            k_collide<D, ST, 0><<<cgrid, kBlock, 0, s.stream>>>(p);
        } else {
            if (p.eq_mode == 0) { k_anomaly<D, ST, 1><<<grid, kBlock, 0, s.stream>>>(p); ++*launches; }
            k_collide<D, ST, 1><<<cgrid, kBlock, 0, s.stream>>>(p);
        }
        ++*launches;
    });
    return cudaGetLastError();
}

// -------------------------------------------------------------------- init
// f_i = rho Psi_i(u, T + u^2, lam) (Eq. 27eq) at every node, written to the
// even-parity slots.
template <int D, int ST, typename TIn>
__global__ void __launch_bounds__(kBlock) k_init(StepParams p, const TIn* rho, const TIn* u)
{
    using S = Storage<ST>;
    const int cell = blockIdx.x * kBlock + threadIdx.x;
    if (cell >= p.N) return;
    const float drho = (float)((double)rho[cell] - (double)p.rho_ref);
    float uu[3], zero[3] = {0.f, 0.f, 0.f}, du[3], dP[3];
#pragma unroll
    for (int a = 0; a < D; ++a) uu[a] = (float)u[(size_t)a * p.N + cell];
    baseline_args<D>(p, uu, zero, du, dP);
    typename S::T* f = static_cast<typename S::T*>(p.f);
    for_each_equilibrium<D>(p, drho, du, dP, [&](int i, float geq) {
        S::store(f + i * p.N + cell, S::shifted ? geq : geq + p.bw[i] * p.rho_ref);
    });
}

template <int D>
cudaError_t init_impl(const Solver& s, const void* rho, const void* u, int dtype, long long* launches)
{
    StepParams p;
    fill_params(s, p);
    const dim3 grid((unsigned)((s.N + kBlock - 1) / kBlock));
    ELBM_DISPATCH_STORAGE(s.storage, {
        if (dtype == ELBM_DTYPE_F64)
            k_init<D, ST, double><<<grid, kBlock, 0, s.stream>>>(p, (const double*)rho, (const double*)u);
        else
            k_init<D, ST, float><<<grid, kBlock, 0, s.stream>>>(p, (const float*)rho, (const float*)u);
        ++*launches;
    });
    return cudaGetLastError();
}

// ------------------------------------------------------------- read-outs
// Post-streaming populations of a node as deviations g_i, at the solver's
// current parity (not a hot path: parity is a run-time value here).
template <int D, int ST>
__device__ __forceinline__ void gather_any(const StepParams& p, const Node& n, float* g)
{
    if (p.parity == 0) gather<D, ST, 0>(p, n, g);
    else gather<D, ST, 1>(p, n, g, p.walls_y != 0);
}

// rho and u of every node (Eqs. density, momentum) with the step kernels'
// FP32 sums; with a body force u is reported at the half step, u + g/2.
template <int D, int ST, typename TOut>
__global__ void __launch_bounds__(kBlock) k_moments(StepParams p, TOut* rho, TOut* u)
{
    const int cell = blockIdx.x * kBlock + threadIdx.x;
    if (cell >= p.N) return;
    const Node n = make_node<D>(p, cell);
    float g[Lat<D>::Q];
    gather_any<D, ST>(p, n, g);
    float drho, j[3];
    moments<D>(p, g, drho, j);
    const float r = p.rho_ref + drho;
    const float inv_r = 1.0f / r;
    rho[cell] = (TOut)r;
#pragma unroll
    for (int a = 0; a < D; ++a) u[(size_t)a * p.N + cell] = (TOut)(j[a] * inv_r + 0.5f * p.g[a]);
}

template <int D>
cudaError_t moments_impl(const Solver& s, void* rho, void* u, int dtype, long long* launches)
{
    StepParams p;
    fill_params(s, p);
    const dim3 grid((unsigned)((s.N + kBlock - 1) / kBlock));
    ELBM_DISPATCH_STORAGE(s.storage, {
        if (dtype == ELBM_DTYPE_F64)
            k_moments<D, ST, double><<<grid, kBlock, 0, s.stream>>>(p, (double*)rho, (double*)u);
        else
            k_moments<D, ST, float><<<grid, kBlock, 0, s.stream>>>(p, (float*)rho, (float*)u);
        ++*launches;
    });
    return cudaGetLastError();
}

// Post-streaming population i of a node, unshifted, in FP64.
template <int D, int ST>
__device__ __forceinline__ double load_f64(const StepParams& p, const Node& n, int i)
{
    using S = Storage<ST>;
    const typename S::T* f = static_cast<const typename S::T*>(p.f);
    const bool walls = p.walls_y != 0;
    const float v = S::load(f + read_slot<D>(n, p.N, i, p.parity, walls));
    // a bounced slot holds population opp(i), stored against its own baseline
    const int b = (p.parity == 1 && walls && read_bounced(n, i)) ? Lat<D>::Q - 1 - i : i;
    return S::shifted ? (double)v + (double)p.bw[b] * (double)p.rho_ref : (double)v;
}

// Unshifted post-streaming populations f_i = g_i + w_i rho_ref, layout f[i][cell].
template <int D, int ST, typename TOut>
__global__ void __launch_bounds__(kBlock) k_get_f(StepParams p, TOut* out)
{
    const int cell = blockIdx.x * kBlock + threadIdx.x;
    if (cell >= p.N) return;
    const Node n = make_node<D>(p, cell);
#pragma unroll
    for (int i = 0; i < Lat<D>::Q; ++i)
        out[(size_t)i * p.N + cell] = (TOut)load_f64<D, ST>(p, n, i);
}

// Store caller populations at the even-parity slots.
template <int D, int ST, typename TIn>
__global__ void __launch_bounds__(kBlock) k_set_f(StepParams p, const TIn* in)
{
    using S = Storage<ST>;
    const int cell = blockIdx.x * kBlock + threadIdx.x;
    if (cell >= p.N) return;
    typename S::T* f = static_cast<typename S::T*>(p.f);
#pragma unroll
    for (int i = 0; i < Lat<D>::Q; ++i) {
        const double v = (double)in[(size_t)i * p.N + cell];
        const double stored = S::shifted ? v - (double)p.bw[i] * (double)p.rho_ref : v;
        S::store(f + i * p.N + cell, (float)stored);
    }
}

template <int D>
cudaError_t get_populations_impl(const Solver& s, void* f, int dtype, long long* launches)
{
    StepParams p;
    fill_params(s, p);
    const dim3 grid((unsigned)((s.N + kBlock - 1) / kBlock));
    ELBM_DISPATCH_STORAGE(s.storage, {
        if (dtype == ELBM_DTYPE_F64) k_get_f<D, ST, double><<<grid, kBlock, 0, s.stream>>>(p, (double*)f);
        else k_get_f<D, ST, float><<<grid, kBlock, 0, s.stream>>>(p, (float*)f);
        ++*launches;
    });
    return cudaGetLastError();
}

template <int D>
cudaError_t set_populations_impl(const Solver& s, const void* f, int dtype, long long* launches)
{
    StepParams p;
    fill_params(s, p);
    const dim3 grid((unsigned)((s.N + kBlock - 1) / kBlock));
    ELBM_DISPATCH_STORAGE(s.storage, {
        if (dtype == ELBM_DTYPE_F64) k_set_f<D, ST, double><<<grid, kBlock, 0, s.stream>>>(p, (const double*)f);
        else k_set_f<D, ST, float><<<grid, kBlock, 0, s.stream>>>(p, (const float*)f);
        ++*launches;
    });
    return cudaGetLastError();
}

// ------------------------------------------------------- FP64 diagnostics
// Stage 1: per node rho, u and min_i f_i (FP32, the step kernels' sums) into
// scratch mom[5][N].
template <int D, int ST>
__global__ void __launch_bounds__(kBlock) k_red_nodes(StepParams p, float* mom)
{
    const int cell = blockIdx.x * kBlock + threadIdx.x;
    if (cell >= p.N) return;
    const Node n = make_node<D>(p, cell);
    float g[Lat<D>::Q];
    gather_any<D, ST>(p, n, g);
    float drho, j[3];
    moments<D>(p, g, drho, j);
    float fmin = FLT_MAX;
#pragma unroll
    for (int i = 0; i < Lat<D>::Q; ++i) fmin = fminf(fmin, fmaf(p.bw[i], p.rho_ref, g[i]));
    const float r = p.rho_ref + drho;
    const float inv_r = 1.0f / r;
    mom[cell] = r;
    mom[(size_t)p.N + cell] = j[0] * inv_r + 0.5f * p.g[0];
    mom[(size_t)2 * p.N + cell] = j[1] * inv_r + 0.5f * p.g[1];
    mom[(size_t)3 * p.N + cell] = (D == 3) ? j[2] * inv_r + 0.5f * p.g[2] : 0.f;
    mom[(size_t)4 * p.N + cell] = fmin;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_min(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Reduce ELBM_NRED FP64 accumulators over a block: warp shuffles, then one
// shared-memory stage across the block's warps.  Result valid in thread 0.
__device__ __forceinline__ void block_reduce(double* acc, double* out)
{
    __shared__ double sh[kBlock / 32][ELBM_NRED];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < ELBM_NRED; ++k) {
        const double v = (k == 9) ? warp_min(acc[k]) : (k == 11) ? warp_max(acc[k]) : warp_sum(acc[k]);
        if (lane == 0) sh[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < ELBM_NRED) {
        const int k = threadIdx.x;
        double v = sh[0][k];
        for (int w = 1; w < kBlock / 32; ++w)
            v = (k == 9) ? fmin(v, sh[w][k]) : (k == 11) ? fmax(v, sh[w][k]) : v + sh[w][k];
        out[k] = v;
    }
}

// Compensated FP32 sum: hi + lo carries the running sum to about twice FP32's
// precision -- each addition is split exactly into its rounded sum and the
// rounding error (Knuth's TwoSum error-free transformation), and the errors
// accumulate in lo.  For the few dozen terms a thread adds, hi + lo is within
// about n 2^-48 of the exact sum, so per-thread partial sums keep FP64-grade
// accuracy while the arithmetic stays on the FP32 pipes (FP64 issue is far
// slower on this GPU); the sums across threads and blocks are FP64.
struct Sum2f {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float s = hi + x;
        const float bp = s - hi;
        const float err = (hi - (s - bp)) + (x - bp);
        hi = s;
        lo += err;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Stage 2: per-block FP64 partial sums (grid-stride over nodes, compensated
// FP32 within a thread); vorticity and d_x u_x by central differences with
// node spacing lam.  With walls the
// velocity beyond a wall is the negated value of the wall-adjacent node
// (no slip half-way between the nodes), and the wall-normal gradient of u_x
// at each wall node comes from the quadratic through the wall (u = 0, a
// distance lam_y/2 away) and the first two nodes: (9 u_x(1st) - u_x(2nd)) / (3 lam_y).
template <int D>
__global__ void __launch_bounds__(kBlock) k_red_sum(StepParams p, const float* mom, double* partials)
{
    Sum2f sum[ELBM_NRED];  // entries 9 (min) and 11 (max) unused
    float fmin_ = FLT_MAX, umax = 0.f;
    int nonfinite = 0;
    const float* ux = mom + p.N;
    const float* uy = mom + 2 * (size_t)p.N;
    const float* uz = mom + 3 * (size_t)p.N;
    const float ix = 0.5f / p.lam[0], iy = 0.5f / p.lam[1], iz = 0.5f / p.lam[2];
    for (int cell = blockIdx.x * kBlock + threadIdx.x; cell < p.N; cell += gridDim.x * kBlock) {
        const Node n = make_node<D>(p, cell);
        const float r = mom[cell];
        const float u0 = ux[cell], u1 = uy[cell], u2 = uz[cell];
        const float uu = u0 * u0 + u1 * u1 + u2 * u2;
        const bool finite = isfinite(r) && isfinite(uu);
        const bool walls = p.walls_y != 0;
        auto dy = [&](const float* v) {
            const float up = (walls && n.yhi) ? -v[cell] : v[n.at(0, 1, 0)];
            const float dn = (walls && n.ylo) ? -v[cell] : v[n.at(0, -1, 0)];
            return (up - dn) * iy;
        };
        const float dxuy = (uy[n.at(1, 0, 0)] - uy[n.at(-1, 0, 0)]) * ix;
        const float dyux = dy(ux);
        float w2 = (dxuy - dyux) * (dxuy - dyux);
        if (walls && (n.ylo || n.yhi)) {
            const float second = n.ylo ? ux[n.at(0, 1, 0)] : ux[n.at(0, -1, 0)];
            sum[12].add((9.0f * u0 - second) * (1.0f / (3.0f * p.lam[1])));
        }
        if (D == 3) {
            const float dyuz = dy(uz);
            const float dzuy = (uy[n.at(0, 0, 1)] - uy[n.at(0, 0, -1)]) * iz;
            const float dzux = (ux[n.at(0, 0, 1)] - ux[n.at(0, 0, -1)]) * iz;
            const float dxuz = (uz[n.at(1, 0, 0)] - uz[n.at(-1, 0, 0)]) * ix;
            w2 += (dyuz - dzuy) * (dyuz - dzuy) + (dzux - dxuz) * (dzux - dxuz);
        }
        const float dxux = (ux[n.at(1, 0, 0)] - ux[n.at(-1, 0, 0)]) * ix;
        sum[0].add(r);
        sum[1].add(r * u0);
        sum[2].add(r * u1);
        sum[3].add(r * u2);
        sum[4].add(r * uu);
        sum[5].add(uu);
        sum[6].add(w2);
        sum[7].add(dxux * dxux);
        sum[8].add(u0 * u0);
        fmin_ = fminf(fmin_, mom[4 * (size_t)p.N + cell]);
        nonfinite += finite ? 0 : 1;
        umax = fmaxf(umax, finite ? sqrtf(uu) : 0.f);
    }
    double acc[ELBM_NRED];
#pragma unroll
    for (int k = 0; k < ELBM_NRED; ++k) acc[k] = sum[k].value();
    acc[9] = fmin_ == FLT_MAX ? DBL_MAX : (double)fmin_;
    acc[10] = (double)nonfinite;
    acc[11] = (double)umax;
    block_reduce(acc, partials + (size_t)blockIdx.x * ELBM_NRED);
}

// Stage 3: one block folds the partials in a fixed order (deterministic).
template <int D>
__global__ void __launch_bounds__(kBlock) k_red_final(const double* partials, int nblocks, double* out)
{
    double acc[ELBM_NRED];
#pragma unroll
    for (int k = 0; k < ELBM_NRED; ++k) acc[k] = 0.0;
    acc[9] = DBL_MAX;
    for (int b = threadIdx.x; b < nblocks; b += kBlock) {
        const double* q = partials + (size_t)b * ELBM_NRED;
#pragma unroll
        for (int k = 0; k < ELBM_NRED; ++k)
            acc[k] = (k == 9) ? fmin(acc[k], q[k]) : (k == 11) ? fmax(acc[k], q[k]) : acc[k] + q[k];
    }
    block_reduce(acc, out);
}

// Sums of rho and rho u_a of a caller field (FP64), for the automatic storage
// baseline velocity: out[0] = sum rho, out[1 + a] = sum rho u_a.
template <int D, typename TIn>
__global__ void __launch_bounds__(kBlock) k_field_sums(int N, const TIn* rho, const TIn* u, double* partials)
{
    double acc[ELBM_NRED];
#pragma unroll
    for (int k = 0; k < ELBM_NRED; ++k) acc[k] = 0.0;
    acc[9] = DBL_MAX;
    for (int cell = blockIdx.x * kBlock + threadIdx.x; cell < N; cell += gridDim.x * kBlock) {
        const double r = (double)rho[cell];
        acc[0] += r;
#pragma unroll
        for (int a = 0; a < D; ++a) acc[1 + a] += r * (double)u[(size_t)a * N + cell];
    }
    block_reduce(acc, partials + (size_t)blockIdx.x * ELBM_NRED);
}

template <int D>
cudaError_t field_sums_impl(const Solver& s, const void* rho, const void* u, int dtype, long long* launches)
{
    if (dtype == ELBM_DTYPE_F64)
        k_field_sums<D, double><<<s.red_blocks, kBlock, 0, s.stream>>>((int)s.N, (const double*)rho,
                                                                      (const double*)u, s.partials);
    else
        k_field_sums<D, float><<<s.red_blocks, kBlock, 0, s.stream>>>((int)s.N, (const float*)rho,
                                                                     (const float*)u, s.partials);
    k_red_final<D><<<1, kBlock, 0, s.stream>>>(s.partials, s.red_blocks, s.red_out);
    *launches += 2;
    return cudaGetLastError();
}

// Shear-mode projection (the amplitude of the shear wave, Sec. III.A):
// out[0] = sum_x (u . dir) cos(k . x), out[1] = sum_x (u . dir) sin(k . x), in
// FP64, with x = (i lam_x, j lam_y, k lam_z) the node's physical position and
// u the reported velocity.  The phase is reduced modulo 2 pi in FP64.
struct ModeArgs {
    double k[3], dir[3];
};

template <int D, int ST>
__global__ void __launch_bounds__(kBlock) k_mode_sums(StepParams p, ModeArgs m, double* partials)
{
    double acc[ELBM_NRED];
#pragma unroll
    for (int q = 0; q < ELBM_NRED; ++q) acc[q] = 0.0;
    acc[9] = DBL_MAX;
    for (int cell = blockIdx.x * kBlock + threadIdx.x; cell < p.N; cell += gridDim.x * kBlock) {
        const Node n = make_node<D>(p, cell);
        float g[Lat<D>::Q];
        gather_any<D, ST>(p, n, g);
        float drho, j[3];
        moments<D>(p, g, drho, j);
        const float inv_r = 1.0f / (p.rho_ref + drho);
        double us = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) us += (double)(j[a] * inv_r + 0.5f * p.g[a]) * m.dir[a];
        const int z = (D == 3) ? cell / p.plane : 0;
        const int r = cell - z * p.plane;
        const int y = r / p.nx, x = r - y * p.nx;
        const double phase = m.k[0] * x * (double)p.lam[0] + m.k[1] * y * (double)p.lam[1] +
                             (D == 3 ? m.k[2] * z * (double)p.lam[2] : 0.0);
        double sn, cs;
        sincos(phase, &sn, &cs);
        acc[0] += us * cs;
        acc[1] += us * sn;
    }
    block_reduce(acc, partials + (size_t)blockIdx.x * ELBM_NRED);
}

template <int D>
cudaError_t mode_sums_impl(const Solver& s, const double* k, const double* dir, long long* launches)
{
    StepParams p;
    fill_params(s, p);
    ModeArgs m;
    for (int a = 0; a < 3; ++a) {
        m.k[a] = k[a];
        m.dir[a] = dir[a];
    }
    ELBM_DISPATCH_STORAGE(s.storage, {
        k_mode_sums<D, ST><<<s.red_blocks, kBlock, 0, s.stream>>>(p, m, s.partials);
    });
    k_red_final<D><<<1, kBlock, 0, s.stream>>>(s.partials, s.red_blocks, s.red_out);
    *launches += 2;
    return cudaGetLastError();
}

template <int D>
cudaError_t reduce_impl(const Solver& s, long long* launches)
{
    StepParams p;
    fill_params(s, p);
    const dim3 grid((unsigned)((s.N + kBlock - 1) / kBlock));
    ELBM_DISPATCH_STORAGE(s.storage, {
        k_red_nodes<D, ST><<<grid, kBlock, 0, s.stream>>>(p, s.mom);
    });
    k_red_sum<D><<<s.red_blocks, kBlock, 0, s.stream>>>(p, s.mom, s.partials);
    k_red_final<D><<<1, kBlock, 0, s.stream>>>(s.partials, s.red_blocks, s.red_out);
    *launches += 3;
    return cudaGetLastError();
}

}  // namespace elbm
