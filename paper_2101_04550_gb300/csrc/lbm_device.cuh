// Device-side building blocks of the extended LBGK step: lattice constants,
// storage conversion, AA-pattern gather/scatter, moments, the diagonal anomaly
// and the product-form extended equilibrium with BGK relaxation.
//
// Arithmetic is FP32.  Populations are handled as deviations from a baseline
// equilibrium, g_i = f_i - rho_ref b_i with b_i = Psi_i(U0, T + U0^2, lam) (the
// rest weights w_i for U0 = 0), so that the large constant part never enters
// a rounding step; the equilibrium deviation rho Psi_i - rho_ref b_i is formed
// from per-axis differences (see for_each_equilibrium()).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "elbm_internal.h"

namespace elbm {

// ------------------------------------------------------------------ lattice
// Population i <-> c_i: i = (cx+1) + 3 (cy+1) + 9 (cz+1) (Eq. d3q27vel);
// D2Q9 is the same ordering without z.  opposite(i) = Q-1-i.
template <int D>
struct Lat {
    static constexpr int Q = (D == 2) ? 9 : 27;
};
__host__ __device__ constexpr int cx_of(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int cy_of(int i) { return (i / 3) % 3 - 1; }
template <int D>
__host__ __device__ constexpr int cz_of(int i) { return D == 3 ? i / 9 - 1 : 0; }

// ------------------------------------------------------------------ storage
template <int ST>
struct Storage;
template <>
struct Storage<ELBM_F32> {
    using T = float;
    static constexpr bool shifted = false;
    __device__ static float load(const T* p) { return *p; }
    __device__ static void store(T* p, float v) { *p = v; }
    __device__ static T cvt(float v) { return v; }
};
template <>
struct Storage<ELBM_F32_SHIFT> {
    using T = float;
    static constexpr bool shifted = true;
    __device__ static float load(const T* p) { return *p; }
    __device__ static void store(T* p, float v) { *p = v; }
    __device__ static T cvt(float v) { return v; }
};
template <>
struct Storage<ELBM_F16_SHIFT> {
    using T = __half;
    static constexpr bool shifted = true;
    __device__ static float load(const T* p) { return __half2float(*p); }
    __device__ static void store(T* p, float v) { *p = __float2half_rn(v); }
    __device__ static T cvt(float v) { return __float2half_rn(v); }
};
template <>
struct Storage<ELBM_BF16_SHIFT> {
    using T = __nv_bfloat16;
    static constexpr bool shifted = true;
    __device__ static float load(const T* p) { return __bfloat162float(*p); }
    __device__ static void store(T* p, float v) { *p = __float2bfloat16_rn(v); }
    __device__ static T cvt(float v) { return __float2bfloat16_rn(v); }
};

// --------------------------------------------------------------- node index
// Periodic neighbour offsets of one node: ox[c+1] = x+c (wrapped),
// oy[c+1] = (y+c wrapped)*nx, oz[c+1] = (z+c wrapped)*nx*ny.
struct Node {
    int cell;
    int ox[3], oy[3], oz[3];
    bool ylo, yhi;  // first / last node along y (next to a wall when walls are on)
    __device__ int at(int cx, int cy, int cz) const { return ox[cx + 1] + oy[cy + 1] + oz[cz + 1]; }
};

// floor(n / d) for 0 <= n < 2^31 with the round-up multiplier of d
// (m, s from host_divider; Granlund and Montgomery, PLDI 1994, Sec. 4):
// t = umulhi(n, m), q = (t + n) >> s.
__device__ __forceinline__ int fast_div(int n, unsigned m, int s)
{
    return (int)((__umulhi((unsigned)n, m) + (unsigned)n) >> s);
}

template <int D>
__device__ __forceinline__ Node make_node(const StepParams& p, int cell)
{
    Node n;
    n.cell = cell;
    const int z = (D == 3) ? fast_div(cell, p.div_plane_m, p.div_plane_s) : 0;
    const int r = cell - z * p.plane;
    const int y = fast_div(r, p.div_nx_m, p.div_nx_s);
    const int x = r - y * p.nx;
    n.ox[1] = x;
    n.ox[0] = (x == 0) ? p.nx - 1 : x - 1;
    n.ox[2] = (x == p.nx - 1) ? 0 : x + 1;
    n.oy[1] = y * p.nx;
    n.oy[0] = ((y == 0) ? p.ny - 1 : y - 1) * p.nx;
    n.oy[2] = ((y == p.ny - 1) ? 0 : y + 1) * p.nx;
    n.ylo = (y == 0);
    n.yhi = (y == p.ny - 1);
    if (D == 3) {
        n.oz[1] = z * p.plane;
        n.oz[0] = ((z == 0) ? p.nz - 1 : z - 1) * p.plane;
        n.oz[2] = ((z == p.nz - 1) ? 0 : z + 1) * p.plane;
    } else {
        n.oz[0] = n.oz[1] = n.oz[2] = 0;
    }
    return n;
}

// ------------------------------------------------------- AA-pattern streaming
// The populations live in one array (in place).  Before an even step the
// post-streaming f_i(x) sits in slot (i, x); the step writes its post-collision
// value to slot (opp(i), x).  Before an odd step f_i(x) sits in slot
// (opp(i), x - c_i) and the step writes to slot (i, x + c_i).  Either way a node
// reads and writes the same slot set, and the slot sets of distinct nodes are
// disjoint (Eq. LBGK: f_i moves one node along c_i per step).
//
// With walls below y = 0 and above y = ny-1 (half-way bounce-back) a
// population that would cross a wall comes back reversed to the node it left:
// f_i(x, t+1) = f'_opp(i)(x, t).  The even step needs no change (it touches
// only the node's own slots).  In the odd step, f_i(x) with x - c_i beyond a
// wall is f'_opp(i)(x), which the even step left in slot (i, x); and f'_i(x)
// with x + c_i beyond a wall becomes f_opp(i)(x) of the next step, slot
// (opp(i), x).  Reads and writes of a node still cover one and the same slot
// set: population i is bounced on reading exactly when opp(i) is bounced on
// writing.
//
// A stored deviation is taken against the baseline of the population it
// holds, so a bounced population, which changes from opp(i) to i, is rebased
// by rho_ref (b_opp(i) - b_i) on reading and by rho_ref (b_i - b_opp(i)) on
// writing (zero for the rest baseline, which is symmetric).
__device__ __forceinline__ bool read_bounced(const Node& n, int i)
{
    return (cy_of(i) == 1 && n.ylo) || (cy_of(i) == -1 && n.yhi);
}
__device__ __forceinline__ bool write_bounced(const Node& n, int i)
{
    return (cy_of(i) == 1 && n.yhi) || (cy_of(i) == -1 && n.ylo);
}
template <int D>
__device__ __forceinline__ int read_slot(const Node& n, int N, int i, int parity, bool walls = false)
{
    constexpr int Q = Lat<D>::Q;
    if (parity == 0) return i * N + n.cell;
    if (walls && read_bounced(n, i)) return i * N + n.cell;
    return (Q - 1 - i) * N + n.at(-cx_of(i), -cy_of(i), -cz_of<D>(i));
}
template <int D>
__device__ __forceinline__ int write_slot(const Node& n, int N, int i, int parity, bool walls = false)
{
    constexpr int Q = Lat<D>::Q;
    if (parity == 0) return (Q - 1 - i) * N + n.cell;
    if (walls && write_bounced(n, i)) return (Q - 1 - i) * N + n.cell;
    return i * N + n.at(cx_of(i), cy_of(i), cz_of<D>(i));
}
// Rebase of a bounced read of population i: rho_ref (b_opp(i) - b_i).
template <int D>
__device__ __forceinline__ float bounce_rebase(const StepParams& p, int i)
{
    return p.rho_ref * (p.bw[Lat<D>::Q - 1 - i] - p.bw[i]);
}

template <int D, int ST, int PAR>
__device__ __forceinline__ void gather(const StepParams& p, const Node& n, float* g, bool walls = false)
{
    using S = Storage<ST>;
    const typename S::T* f = static_cast<const typename S::T*>(p.f);
#pragma unroll
    for (int i = 0; i < Lat<D>::Q; ++i) {
        const float v = S::load(f + read_slot<D>(n, p.N, i, PAR, walls));
        g[i] = S::shifted ? v : v - p.bw[i] * p.rho_ref;
        if (S::shifted && PAR == 1 && walls && read_bounced(n, i)) g[i] += bounce_rebase<D>(p, i);
    }
}

template <int D, int ST, int PAR>
__device__ __forceinline__ void scatter(const StepParams& p, const Node& n, const float* g, bool walls = false)
{
    using S = Storage<ST>;
    typename S::T* f = static_cast<typename S::T*>(p.f);
#pragma unroll
    for (int i = 0; i < Lat<D>::Q; ++i) {
        float v = S::shifted ? g[i] : g[i] + p.bw[i] * p.rho_ref;
        if (S::shifted && PAR == 1 && walls && write_bounced(n, i)) v += bounce_rebase<D>(p, Lat<D>::Q - 1 - i);
        S::store(f + write_slot<D>(n, p.N, i, PAR, walls), v);
    }
}

// ---------------------------------------------- shared-memory staged gather
// The populations of a node are copied asynchronously (cp.async, no register
// cost) into the calling thread's column of a [Q][kStageStride] shared-memory
// stage, then read back twice (moments, relaxation).  Copies move 4-byte
// words; a 16-bit population is taken from the word that contains it, so the
// population array carries 16 bytes of tail padding.
__device__ __forceinline__ void cp_async4(unsigned* smem_dst, const void* gmem_src)
{
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(gmem_src) : "memory");
}
// An integer the compiler must treat as unknown: recomputing an address from
// it is cheaper than keeping 27 addresses alive across the collision.
__device__ __forceinline__ int opaque(int x)
{
    asm volatile("" : "+r"(x));
    return x;
}

// 16-byte asynchronous copy (global -> shared, both 16-byte aligned).
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src)
{
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(gmem_src) : "memory");
}

// Fresh read of a staged word (volatile, so that the two read-backs of a
// population are not merged into one long-lived register).
__device__ __forceinline__ unsigned ld_stage(const unsigned* smem)
{
    unsigned v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"((unsigned)__cvta_generic_to_shared(smem)));
    return v;
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Wait until at most one committed group (the newest) is still in flight.
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

template <int ST>
__device__ __forceinline__ const void* stage_src(const StepParams& p, int idx)
{
    using S = Storage<ST>;
    if (sizeof(typename S::T) == 4) return static_cast<const float*>(p.f) + idx;
    return static_cast<const unsigned*>(p.f) + (idx >> 1);
}

// Value of the population staged from element idx (deviation g_i).
template <int ST>
__device__ __forceinline__ float stage_value(const StepParams& p, unsigned word, int idx, int i)
{
    using S = Storage<ST>;
    float v;
    if (ST == ELBM_F16_SHIFT) v = __half2float(__ushort_as_half((unsigned short)(word >> ((idx & 1) * 16))));
    else if (ST == ELBM_BF16_SHIFT) v = __bfloat162float(__ushort_as_bfloat16((unsigned short)(word >> ((idx & 1) * 16))));
    else v = __uint_as_float(word);
    return S::shifted ? v : v - p.bw[i] * p.rho_ref;
}

// ------------------------------------------------------------------ moments
// drho = sum_i g_i (so rho = rho_ref + drho, Eq. density, since sum_i b_i = 1);
// j_a = rho_ref U0_a + lam_a sum_i c_ia g_i = rho u_a (Eq. momentum, since the
// baseline b_i carries the momentum rho_ref U0).
template <int D>
__device__ __forceinline__ void moments(const StepParams& p, const float* g, float& drho, float* j)
{
    // lines of three along x (population index x fastest), then rows along y, then planes along z
    constexpr int NL = Lat<D>::Q / 3, NP = NL / 3 > 0 ? NL / 3 : 1;
    float t[NL], sx = 0.f, sy = 0.f;
#pragma unroll
    for (int L = 0; L < NL; ++L) {
        const float a = g[3 * L], b = g[3 * L + 1], c = g[3 * L + 2];
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

// Diagonal anomaly Q~_aaa = rho u_a (lam_a^2 - 3T) - rho u_a^3 = j_a (lam_a^2 - 3T - u_a^2)
// (Eq. Deviation, R = 1).
//
// Rounding steps here and in the equilibrium below are spelled out (fmaf
// where a product and a sum are fused, __fmul_rn / __fadd_rn / __fsub_rn
// where they are not), so that the compiler has no contraction left to
// choose: every kernel form computes the same roundings, whatever the code
// around the helpers, and the forms agree bit for bit by construction.
__device__ __forceinline__ float anomaly(const StepParams& p, int a, float ja, float ua)
{
    return __fmul_rn(ja, fmaf(-ua, ua, p.lam2m3T[a]));
}

// ------------------------------------------------- extended equilibrium + BGK
// Equilibrium deviation geq_i = rho Psi_i(u, P, lam) - rho_ref b_i from the
// storage baseline b_i = Psi_i(U0, T + U0^2, lam) (U0 = 0 gives the rest
// equilibrium w_i).  Per axis the triplet (Eqs. phi0S, phiPlusS, phiMinusS) is
// Psi_c = base_c + delta_c with, for du = u - U0 and dP = P - (T + U0^2),
// delta_0 = -dP/lam^2 and delta_{+-1} = (+-du/lam + dP/lam^2)/2, so
//   Psi_i - b_i = sum_a (prod_{b<a} base_b) delta_a (prod_{b>a} Psi_b)
// is formed without cancellation, and rho Psi_i - rho_ref b_i =
// (rho - rho_ref) Psi_i + rho_ref (Psi_i - b_i).  fn sees the populations
// with cz innermost, then cx, then cy (relax() and relax_streamed() sum the
// increments along these lines).
template <int D, typename F>
__device__ __forceinline__ void for_each_equilibrium(const StepParams& p, float drho, const float* du,
                                                     const float* dP, F&& fn)
{
    float A[3][3], dl[3][3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const float s = __fmul_rn(dP[a], p.inv_lam2[a]);
        const float t = __fmul_rn(du[a], p.inv_lam[a]);
        dl[a][0] = __fmul_rn(0.5f, __fsub_rn(s, t));
        dl[a][1] = -s;
        dl[a][2] = __fmul_rn(0.5f, __fadd_rn(s, t));
#pragma unroll
        for (int c = 0; c < 3; ++c) A[a][c] = __fadd_rn(p.base[a][c], dl[a][c]);
    }
    // rho_ref is folded into the x factors: dlx_r = rho_ref delta_x, base_xr = rho_ref base_x
    float dlx_r[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) dlx_r[c] = __fmul_rn(p.rho_ref, dl[0][c]);
#pragma unroll
    for (int cy = 0; cy < 3; ++cy) {
#pragma unroll
        for (int cx = 0; cx < 3; ++cx) {
            const float pxy = __fmul_rn(A[0][cx], A[1][cy]);
            // rho_ref (prod_{x,y} Psi - prod_{x,y} base)
            const float dxy_r = fmaf(dlx_r[cx], A[1][cy], __fmul_rn(p.base_xr[cx], dl[1][cy]));
            if (D == 2) {
                fn(cx + 3 * cy, fmaf(drho, pxy, dxy_r));
            } else {
#pragma unroll
                for (int cz = 0; cz < 3; ++cz) {
                    const float psi = __fmul_rn(pxy, A[2][cz]);
                    const float dpsi_r = fmaf(dxy_r, A[2][cz], __fmul_rn(p.bxy_r[cx + 3 * cy], dl[2][cz]));
                    fn(cx + 3 * cy + 9 * cz, fmaf(drho, psi, dpsi_r));
                }
            }
        }
    }
}

// The conventional second-order equilibrium (Sec. III preamble): the product
// form of Eq. 27eq with every term of total degree above two in u dropped.
// Per axis Psi_c(u, T + u^2, lam) = A_c + B_c u + C_c u^2 with A_c the rest
// triplet, B_{+-1} = +-1/(2 lam), B_0 = 0, C_{+-1} = 1/(2 lam^2), C_0 = -1/lam^2,
// so with l_a = B u_a and s_a = (B + C u_a) u_a the truncated product is
//   S_i = w_i + sum_a s_a prod_{b != a} A_b + sum_{a<b} l_a l_b prod_{c != a,b} A_c,
// and fn(i, rho S_i - rho_ref w_i) = fn(i, drho w_i + rho (S_i - w_i)).
// Defined for the rest baseline (U0 = 0), where base = rest triplet.
template <int D, typename F>
__device__ __forceinline__ void for_each_second_order(const StepParams& p, float drho, const float* u, F&& fn)
{
    const float rho = p.rho_ref + drho;
    float A[3][3], l[3][3], sq[3][3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const float hb = 0.5f * p.inv_lam[a] * u[a];
        const float q2 = u[a] * u[a] * p.inv_lam2[a];
        l[a][0] = -hb;
        l[a][1] = 0.f;
        l[a][2] = hb;
        sq[a][0] = fmaf(0.5f, q2, -hb);
        sq[a][1] = -q2;
        sq[a][2] = fmaf(0.5f, q2, hb);
#pragma unroll
        for (int c = 0; c < 3; ++c) A[a][c] = p.base[a][c];
    }
#pragma unroll
    for (int cy = 0; cy < 3; ++cy) {
#pragma unroll
        for (int cx = 0; cx < 3; ++cx) {
            if (D == 2) {
                const float dev = sq[0][cx] * A[1][cy] + sq[1][cy] * A[0][cx] + l[0][cx] * l[1][cy];
                const int i = cx + 3 * cy;
                fn(i, fmaf(drho, p.bw[i], rho * dev));
            } else {
#pragma unroll
                for (int cz = 0; cz < 3; ++cz) {
                    const float dev = sq[0][cx] * A[1][cy] * A[2][cz] + sq[1][cy] * A[0][cx] * A[2][cz] +
                                      sq[2][cz] * A[0][cx] * A[1][cy] + l[0][cx] * l[1][cy] * A[2][cz] +
                                      l[0][cx] * l[2][cz] * A[1][cy] + l[1][cy] * l[2][cz] * A[0][cx];
                    const int i = cx + 3 * cy + 9 * cz;
                    fn(i, fmaf(drho, p.bw[i], rho * dev));
                }
            }
        }
    }
}

// Per-axis arguments of for_each_equilibrium for velocity u and pressure
// excess over T, pex = P - T: du = u - U0, dP = pex - U0^2 = du (u + U0) + (pex - u^2).
template <int D>
__device__ __forceinline__ void baseline_args(const StepParams& p, const float* u, const float* corr,
                                              float* du, float* dP)
{
#pragma unroll
    for (int a = 0; a < D; ++a) {
        du[a] = __fsub_rn(u[a], p.u0[a]);
        dP[a] = fmaf(du[a], __fadd_rn(u[a], p.u0[a]), corr[a]);
    }
}

// Body-force increment of the exact-difference reading of the forcing,
// F_i = rho [Psi_i(u + g, T + (u + g)^2, lam) - Psi_i(u, T + u^2, lam)] (the
// product-form equilibrium of Eqs. prod, 27eq at the shifted and the unshifted
// velocity), handed out divided by omega so that it joins the increment
// omega (f*_i - f_i) before the one rounding of the relaxation.  The
// difference of the products is telescoped over the axes,
//   prod_a A_a - prod_a B_a = sum_a (prod_{b<a} A_b) (A_a - B_a) (prod_{b>a} B_b),
// with A the triplet at u + g, B at u, and per axis, for dP = g (2u + g),
//   A_0 - B_0 = -dP / lam^2,  A_{+-1} - B_{+-1} = (+-g / lam + dP / lam^2) / 2,
// so the small increment carries no cancellation.
template <int D>
struct ForceIncrement {
    float A[3][3], B[3][3], dl[3][3];

    __device__ __forceinline__ void init(const StepParams& p, float rho_over_omega, const float* u)
    {
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const float ua = u[a], ga = p.g[a], ug = ua + ga;
            const float il = p.inv_lam[a], il2 = p.inv_lam2[a];
            const float sb = fmaf(ua, ua, p.T) * il2, sa = fmaf(ug, ug, p.T) * il2;
            B[a][0] = 0.5f * (sb - ua * il);
            B[a][1] = 1.0f - sb;
            B[a][2] = 0.5f * (sb + ua * il);
            A[a][0] = 0.5f * (sa - ug * il);
            A[a][1] = 1.0f - sa;
            A[a][2] = 0.5f * (sa + ug * il);
            const float s = ga * (ua + ug) * il2, t = ga * il;
            dl[a][0] = rho_over_omega * (0.5f * (s - t));
            dl[a][1] = rho_over_omega * (-s);
            dl[a][2] = rho_over_omega * (0.5f * (s + t));
        }
    }
    // F_i / omega for population i
    __device__ __forceinline__ float operator()(int i) const
    {
        const int x = cx_of(i) + 1, y = cy_of(i) + 1;
        if (D == 2) return fmaf(dl[0][x], B[1][y], A[0][x] * dl[1][y]);
        const int z = cz_of<D>(i) + 1;
        return fmaf(dl[0][x] * B[1][y], B[2][z], fmaf(A[0][x] * dl[1][y], B[2][z], A[0][x] * A[1][y] * dl[2][z]));
    }
};

// The body-force increment of ForceIncrement for a force along x alone
// (g_y = g_z = 0, the channel of Sec. III.E).  The telescoped sum then keeps
// only its x term, F_i / omega = (rho / omega) (A_x - B_x)_{c_ix} B_{y,c_iy}
// B_{z,c_iz}; the other two terms are exact zeros, so this gives the same
// bits as the general form with a third of its registers.
template <int D>
struct ForceIncrementX {
    float dl[3], By[3], Bz[3];

    __device__ __forceinline__ void init(const StepParams& p, float rho_over_omega, const float* u)
    {
        {
            const float ua = u[0], ga = p.g[0], ug = ua + ga;
            const float il = p.inv_lam[0], il2 = p.inv_lam2[0];
            const float s = ga * (ua + ug) * il2, t = ga * il;
            dl[0] = rho_over_omega * (0.5f * (s - t));
            dl[1] = rho_over_omega * (-s);
            dl[2] = rho_over_omega * (0.5f * (s + t));
        }
#pragma unroll
        for (int a = 1; a < D; ++a) {
            const float ua = u[a], il = p.inv_lam[a];
            const float sb = fmaf(ua, ua, p.T) * p.inv_lam2[a];
            float* B = a == 1 ? By : Bz;
            B[0] = 0.5f * (sb - ua * il);
            B[1] = 1.0f - sb;
            B[2] = 0.5f * (sb + ua * il);
        }
    }
    __device__ __forceinline__ float operator()(int i) const
    {
        const int x = cx_of(i) + 1, y = cy_of(i) + 1;
        if (D == 2) return fmaf(dl[x], By[y], 0.f);
        return fmaf(dl[x] * By[y], Bz[cz_of<D>(i) + 1], 0.f);
    }
};

// Slot of population i among the ones that carry the conservation
// correction (rest, then -x, +x, -y, +y, -z, +z), or -1.
template <int D>
__host__ __device__ constexpr int corrected_slot(int i)
{
    constexpr int I0 = (Lat<D>::Q - 1) / 2;
    return i == I0 ? 0 : i == I0 - 1 ? 1 : i == I0 + 1 ? 2 : i == I0 - 3 ? 3 : i == I0 + 3 ? 4
         : (D == 3 && i == I0 - 9) ? 5 : (D == 3 && i == I0 + 9) ? 6 : -1;
}

// Relax g toward the extended equilibrium (Eq. LBGK with f* of Eq. 27eqext).
// d[a] is the central difference of the anomaly along axis a; the pressure
// diagonal is P*_aa = T + u_a^2 + (2-omega)/(2 rho omega) d_a (Eq. Paastar1).
//
// In exact arithmetic f* carries the node's rho and rho u (Eqs. density,
// momentum), so relaxation conserves them.  In FP32 the rounding of rho, of
// u = j/rho and of the triplet terms leaves the computed equilibrium with a
// mass and momentum off by a fraction of an ulp, and in near-uniform flow
// that error has the same sign at every node and every step.  So the moments
// e0 = sum_i dlt_i and e_a = sum_i c_ia dlt_i of the increments
// dlt_i = geq_i - g_i (small numbers, summed accurately) are removed before
// the single rounding of g + omega dlt: e0 from the rest population and
// +-e_a/2 from the two populations along axis a.
template <int D>
__device__ __forceinline__ void relax(const StepParams& p, float* g, float drho, const float* j,
                                      const float* d)
{
    constexpr int I0 = (Lat<D>::Q - 1) / 2;
    const float rho = p.rho_ref + drho;
    const float inv_rho = 1.0f / rho;
    float u[3], pcorr[3], du[3], dP[3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        u[a] = j[a] * inv_rho;
        pcorr[a] = p.coef * inv_rho * d[a];
    }
    baseline_args<D>(p, u, pcorr, du, dP);
    const float om = p.omega;
    float e0 = 0.f, ex = 0.f, ey = 0.f, ez = 0.f;
    float keep[2 * D + 1];
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
    for_each_equilibrium<D>(p, drho, du, dP, [&](int i, float geq) {
        const float dl = geq - g[i];
        accumulate(i, dl);
        const int k = corrected_slot<D>(i);
        if (k >= 0) keep[k] = geq;
        else g[i] = fmaf(om, dl, g[i]);
    });
    const float hx = 0.5f * ex, hy = 0.5f * ey;
    g[I0] = fmaf(om, (keep[0] - g[I0]) - e0, g[I0]);
    g[I0 - 1] = fmaf(om, (keep[1] - g[I0 - 1]) + hx, g[I0 - 1]);
    g[I0 + 1] = fmaf(om, (keep[2] - g[I0 + 1]) - hx, g[I0 + 1]);
    g[I0 - 3] = fmaf(om, (keep[3] - g[I0 - 3]) + hy, g[I0 - 3]);
    g[I0 + 3] = fmaf(om, (keep[4] - g[I0 + 3]) - hy, g[I0 + 3]);
    if (D == 3) {
        const float hz = 0.5f * ez;
        g[I0 - 9] = fmaf(om, (keep[5] - g[I0 - 9]) + hz, g[I0 - 9]);
        g[I0 + 9] = fmaf(om, (keep[6] - g[I0 + 9]) - hz, g[I0 + 9]);
    }
}

}  // namespace elbm
