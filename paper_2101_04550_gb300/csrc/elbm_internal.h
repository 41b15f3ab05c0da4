// Internal declarations of the elbm CUDA library: the solver handle, the
// by-value parameter block every kernel receives, and the launchers that the
// per-lattice translation units export to the C-ABI layer.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "elbm.h"

namespace elbm {

constexpr int kMaxQ = 27;

// Everything a step kernel needs, passed by value (lives in the constant
// parameter bank).  Derived constants are precomputed on the host in double
// and rounded once to float.
struct StepParams {
    void* f;              // populations, storage type per `storage`, layout f[i][cell]
    float* q;             // diagonal anomaly field q[a][cell] (Eq. Deviation)
    int* status;          // device status word
    int nx, ny, nz;       // nodes per axis (nz = 1 for D2Q9)
    int N;                // nx*ny*nz
    int plane;            // nx*ny
    unsigned div_nx_m, div_plane_m;  // round-up multipliers for division by nx and by nx*ny
    int div_nx_s, div_plane_s;       // and their shifts
    float lam[3];         // stretching factors lam_a
    float inv_lam[3];     // 1/lam_a
    float inv_lam2[3];    // 1/lam_a^2
    float inv_2lam[3];    // 1/(2 lam_a): central-difference weight (node spacing lam_a)
    float lam2m3T[3];     // lam_a^2 - 3T
    float base[3][3];     // storage baseline triplet per axis: Psi_c(U0_a, T + U0_a^2, lam_a)
    float base_xr[3];     // rho_ref base[0][c]
    float bxy_r[9];       // rho_ref base[0][cx] base[1][cy], index cx + 3 cy
    float bw[kMaxQ];      // storage baseline b_i = prod_a base[a][c_ia+1]; stored g_i = f_i - rho_ref b_i
    float u0[3];          // baseline velocity U0 (zero unless set)
    float j0[3];          // rho_ref U0: baseline momentum
    float T;              // temperature (R = 1)
    float omega;          // relaxation frequency
    float coef;           // (2 - omega) / (2 omega)
    float rho_ref;        // reference density of the shifted storage
    float g[3];           // body-force acceleration
    int forced;           // g != 0
    int walls_y;          // half-way bounce-back walls below y = 0 and above y = ny-1
    int eq_mode;          // 0 extended, 1 product form, 2 second order
    int parity;           // AA streaming parity of the step about to run (0 even, 1 odd)
};

struct Solver {
    int lattice = 0, D = 0, Q = 0;
    int nx = 0, ny = 0, nz = 0;
    long long N = 0;
    int storage = 0;
    double lam[3] = {1, 1, 1};
    double T = 0, nu = 0, omega = 0, rho_ref = 1.0;
    double g[3] = {0, 0, 0};
    double u_ref[3] = {0, 0, 0};   // storage baseline velocity U0 (shifted storage modes)
    int u_ref_auto = 0;            // 1: U0 = mean velocity of the field given to elbm_init
    int eq_mode = 0;
    int kernel = 0;       // 0 auto, 1 two-pass, 2 graph-pipelined, 3 single pass (two arrays), 4 fused in place
    int fused_ok = 0;     // the fused in-place form fits this grid (every tile column co-resident)
    unsigned long long* progress = nullptr;  // fused form: per-block progress counters
    unsigned long long epoch = 0;            // fused form: launches so far
    int walls_y = 0;
    int parity = 0;
    int initialised = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    void* f = nullptr;                // populations (current)
    void* f2 = nullptr;               // second population array of the single-pass form
    float* q = nullptr;               // anomaly field
    cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};  // graph-pipelined step per parity
    int graph_nodes = 0;
    int* status = nullptr;            // device status word
    float* mom = nullptr;             // reduction scratch: rho, u[3], fmin per node
    double* partials = nullptr;       // reduction scratch: per-block FP64 partial sums
    double* red_out = nullptr;        // device copy of the ELBM_NRED results
    double host_red[ELBM_NRED] = {};  // host copy of the results
    int red_blocks = 0;
    long long steps_done = 0;
    long long launches = 0;
    size_t bytes = 0;
    long long uid = 0;                // unique per solver of the process (never reused)
    // tensor maps of the TMA-fed single-pass kernels, cached per population
    // array and tile height (tma_maps.cu); a map depends only on the array's
    // address and the grid, so a cached one stays valid for that address
    alignas(64) mutable unsigned char tmap[2][2][128] = {};
    mutable const void* tmap_f[2] = {nullptr, nullptr};
    mutable int tmap_tile_y[2] = {0, 0};
    mutable int tmap_next = 0;
};

// One member of a batch (see batch.cuh).
struct BatchMember {
    StepParams p;         // the member's parameter block (its parity field is ignored)
    int block_begin[2];   // first block of the member in launches of 128 and of 256 threads
    int parity;           // streaming parity before the first step of a launch sequence
};

// Members of one batch at most.
constexpr int kBatchMax = 40;

size_t storage_bytes(int storage);
// Record the message elbm_last_error() returns on the calling thread; returns code.
int set_error(int code, const char* msg);
void fill_params(const Solver& s, StepParams& p);

// Launchers, explicitly instantiated per lattice (kernels_d2q9.cu,
// kernels_d3q27.cu).  Each returns the CUDA error of its launches and adds the
// number of kernel launches it issued to *launches.
template <int D> cudaError_t step_two_pass_impl(const Solver&, int, long long*);
template <int D> cudaError_t step_bounded_impl(const Solver&, int, long long*);
template <int D> cudaError_t step_single_impl(const Solver&, void*, long long*);
template <> cudaError_t step_single_impl<2>(const Solver&, void*, long long*);  // kernels_d2q9.cu
bool single_tmem_geometry(const Solver& s);
bool fused_available(const Solver& s);
cudaError_t step_fused_impl(const Solver& s, int parity, unsigned long long* progress, unsigned long long epoch,
                            long long* launches);
int single_pass_variant(const Solver& s);
// Kernel form a step of s uses (1 two-pass, 2 graph-pipelined, 3 single pass, 4 fused in place):
// the requested form where it applies, else the two-pass form.
int effective_kernel(const Solver* s);
// Whether the automatic form steps s in the single pass (given its second array).
bool auto_single(const Solver* s);
template <int D> cudaError_t build_step_graph_impl(const Solver&, int, cudaGraphExec_t*, int*);
template <int D> cudaError_t init_impl(const Solver&, const void*, const void*, int, long long*);
template <int D> cudaError_t moments_impl(const Solver&, void*, void*, int, long long*);
template <int D> cudaError_t get_populations_impl(const Solver&, void*, int, long long*);
template <int D> cudaError_t set_populations_impl(const Solver&, const void*, int, long long*);
template <int D> cudaError_t reduce_impl(const Solver&, long long*);
template <int D> cudaError_t mode_sums_impl(const Solver&, const double*, const double*, long long*);
template <int D> cudaError_t field_sums_impl(const Solver&, const void*, const void*, int, long long*);
template <int D>
cudaError_t batch_enqueue_impl(int, int, int, int, const void*, int, cudaStream_t, long long*);
// Flattened single-pass batch (batch_single.cuh): size of one member record,
// filling the record of solver s (s.f as array 0, s.f2 as array 1; tensor
// maps re-encoded when encode_maps), and enqueueing nsteps launches of a
// batch kernel (TMEM kernel on 32 x 16 tile columns or TMA kernel on 32 x 8)
// over a work list of nwork items (x member, y x0, z y0, w z0 | z1 << 16) in
// device memory; sp_tma_member: whether the 32 x 8 form takes a solver.
size_t sp_member_bytes();
cudaError_t sp_member_fill(const Solver& s, void* record, bool encode_maps);
void sp_member_set_phase(void* record, int phase);
cudaError_t sp_batch_enqueue(int storage, int tile_y, bool bc, bool fx, const void* members, const void* work,
                             int nwork, int nsteps, cudaStream_t st, long long* launches);
bool sp_tma_member(const Solver& s);

}  // namespace elbm

// The opaque handle of the C ABI is the solver itself.
struct elbm_solver : public elbm::Solver {};
