// Single-pass step of the D2Q9 lattice with two population arrays.
//
// The per-node arithmetic is that of the two-pass form (moments_of,
// anomaly, relax_streamed), so the results agree bit for bit.  A block of
// kD2Threads threads owns a strip of columns and marches along y through a
// segment of rows: thread t holds column x0 - 1 + t, so the first and last
// thread only supply the anomaly of the two columns beside the strip (the x
// central difference of Eq. Paastar1) and the kD2Cols threads between them
// relax their nodes.  Per row k of the march (rows y0-1 .. y1):
//   * every thread loads the 9 populations of its node (coalesced: x is the
//     fastest index), forms the moments (Eqs. density, momentum) and the
//     diagonal anomaly Q~_xxx, Q~_yyy (Eq. Deviation), and writes Q~_xxx to a
//     ring of three shared-memory rows; Q~_yyy stays in registers;
//   * one block barrier, then row k-1 is relaxed (Eqs. Paastar1, 27eqext,
//     LBGK) from the populations kept in registers since the previous row,
//     with the x difference from the shared row and the y difference from
//     Q~_yyy of rows k and k-2, and pushed to (x + cx, y + cy) of the
//     destination array (periodic).
// A segment of S rows reads S + 2 rows; each destination slot is written by
// exactly one thread of one block.
#pragma once
#include "single_pass.cuh"

namespace elbm {

constexpr int kD2Threads = 128;
constexpr int kD2Cols = kD2Threads - 2;  // relaxed columns per block

template <int ST>
__global__ void __launch_bounds__(kD2Threads) k_single_pass_d2q9(const __grid_constant__ StepParams p, void* dst,
                                                                 int seg)
{
    using S = Storage<ST>;
    using T = typename S::T;
    __shared__ float qxs[3][kD2Threads];
    pdl_release();
    const int t = threadIdx.x;
    const int xr = blockIdx.x * kD2Cols - 1 + t;  // column before the periodic wrap
    const bool inner = t >= 1 && t <= kD2Cols && xr < p.nx;
    const int gx = modi(xr, p.nx);
    const int y0 = blockIdx.y * seg, y1 = min(p.ny, y0 + seg);
    const int K = (y1 - y0) + 2;  // rows y0-1 .. y1
    const T* src = static_cast<const T*>(p.f);
    T* out = static_cast<T*>(dst);
    const int xo[3] = {gx == 0 ? p.nx - 1 : gx - 1, gx, gx == p.nx - 1 ? 0 : gx + 1};

    float gp[9];                                  // populations of the row relaxed next
    float m_drho = 0.f, m_j[3] = {0.f, 0.f, 0.f}, m_inv = 1.f;
    float qy_m1 = 0.f, qy_m2 = 0.f;               // Q~_yyy of rows k-1 and k-2
#pragma unroll
    for (int i = 0; i < 9; ++i) gp[i] = 0.f;
    // raw populations of row k, loaded one row ahead so that the loads of row
    // k + 1 are in flight while row k - 1 is relaxed
    T raw[9];
    pdl_wait();  // the previous step has written the source array
    {
        const int node = wrapi(y0 - 1, p.ny) * p.nx + gx;
#pragma unroll
        for (int i = 0; i < 9; ++i) raw[i] = src[i * p.N + node];
    }
    for (int k = 0; k < K; ++k) {
        float g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = raw_value<ST>(p, raw[i], i);
        if (k + 1 < K) {
            const int node = wrapi(y0 + k, p.ny) * p.nx + gx;
#pragma unroll
            for (int i = 0; i < 9; ++i) raw[i] = src[i * p.N + node];
        }
        float drho, j[3];
        moments_of<2>(p, [&](int i) { return g[i]; }, drho, j);
        const float inv = 1.0f / (p.rho_ref + drho);
        const float qx = anomaly(p, 0, j[0], j[0] * inv);
        const float qy = anomaly(p, 1, j[1], j[1] * inv);
        qxs[k % 3][t] = qx;
        __syncthreads();
        if (k >= 2 && inner) {
            // relax row k-1 (y = y0 + k - 2)
            const int r = (k - 1) % 3;
            float d[3] = {0.f, 0.f, 0.f};
            if (p.eq_mode == 0) {
                d[0] = (qxs[r][t + 1] - qxs[r][t - 1]) * p.inv_2lam[0];
                d[1] = (qy - qy_m2) * p.inv_2lam[1];
            }
            const int yc = y0 + k - 2;
            const int yo[3] = {(yc == 0 ? p.ny - 1 : yc - 1) * p.nx, yc * p.nx, (yc == p.ny - 1 ? 0 : yc + 1) * p.nx};
            auto put = [&](int i, float gn) {
                const int slot = opaque(i * p.N) + xo[cx_of(i) + 1] + yo[cy_of(i) + 1];
                S::store(out + slot, S::shifted ? gn : fmaf(p.bw[i], p.rho_ref, gn));
            };
            relax_streamed<2>(p, [&](int i) { return gp[i]; }, put, m_drho, m_j, d, m_inv);
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) gp[i] = g[i];
        m_drho = drho;
        m_j[0] = j[0];
        m_j[1] = j[1];
        m_inv = inv;
        qy_m2 = qy_m1;
        qy_m1 = qy;
    }
}

// Rows per segment: short enough that the grid has several blocks per
// resident slot of the GPU, between 8 and 64 rows; on a grid that 8-row
// segments would leave with less than one wave of blocks (8 resident blocks
// of 128 threads per SM), as few as 4 rows, enough for about one wave (at
// 1024 x 512: 4 rows run 1.47x faster than 8, measured).
inline int d2q9_segment_rows(const Solver& s)
{
    const long long gx = (s.nx + kD2Cols - 1) / kD2Cols;
    const long long sms = s.num_sms > 0 ? s.num_sms : 152;
    const long long slots = 8 * sms;
    if (gx * ((s.ny + 7) / 8) < slots) {
        long long seg = (gx * s.ny + slots - 1) / slots;
        return (int)(seg < 4 ? 4 : seg > 8 ? 8 : seg);
    }
    const long long want = 4ll * 16 * sms;
    long long seg = (gx * s.ny + want - 1) / want;
    if (seg < 8) seg = 8;
    if (seg > 64) seg = 64;
    return (int)seg;
}

inline cudaError_t step_single_d2q9(const Solver& s, void* dst, long long* launches)
{
    StepParams p;
    fill_params(s, p);
    p.parity = 0;
    const int seg = d2q9_segment_rows(s);
    const dim3 grid((unsigned)((s.nx + kD2Cols - 1) / kD2Cols), (unsigned)((s.ny + seg - 1) / seg));
    cudaError_t e = cudaSuccess;
    ELBM_DISPATCH_STORAGE(s.storage, { e = launch_pdl(k_single_pass_d2q9<ST>, grid, dim3(kD2Threads), 0, s.stream, p, dst, seg); });
    if (e == cudaSuccess) ++*launches;
    return e;
}

}  // namespace elbm
