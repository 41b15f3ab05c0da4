// C ABI of the elbm library (declared in include/elbm.h): argument checks,
// ownership of device memory, choice of kernel form, host<->device staging.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "elbm_internal.h"

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(e == cudaErrorMemoryAllocation ? ELBM_ERR_OOM : ELBM_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

}  // namespace

namespace elbm {

int set_error(int code, const char* msg)
{
    std::snprintf(g_err, sizeof g_err, "%s", msg);
    return code;
}

bool base_triplet(double T, double lam, double U0, float out[3], double* u0_eff);

size_t storage_bytes(int storage)
{
    return (storage == ELBM_F16_SHIFT || storage == ELBM_BF16_SHIFT) ? 2 : 4;
}

// Storage-baseline triplet per axis, Psi_c(U0, T + U0^2, lam), rounded so that
// the three floats sum to exactly one (centre a multiple of 2^-24, sides
// multiples of 2^-25).  Returns false if a value is not positive.  *u0_eff
// receives the velocity the rounded triplet carries, lam (b_+ - b_-).
bool base_triplet(double T, double lam, double U0, float out[3], double* u0_eff)
{
    const double P0 = T + U0 * U0;
    const double centre = std::nearbyint((1.0 - P0 / (lam * lam)) * 16777216.0) / 16777216.0;
    const double sides = 1.0 - centre;
    const double plus = std::nearbyint((0.5 * sides + 0.5 * U0 / lam) * 33554432.0) / 33554432.0;
    const double minus = sides - plus;
    out[0] = (float)minus;
    out[1] = (float)centre;
    out[2] = (float)plus;
    *u0_eff = lam * (plus - minus);
    return minus > 0.0 && centre > 0.0 && plus > 0.0;
}

static bool shifted_storage(int storage) { return storage != ELBM_F32; }

// Round-up multiplier and shift for floor(n / d), 0 <= n < 2^31, d >= 1:
// t = umulhi(n, m), q = (t + n) >> s with s = ceil(log2 d) and
// m = floor(2^32 (2^s - d) / d) + 1.  This is the unsigned division by an
// invariant integer of Granlund and Montgomery ("Division by invariant
// integers using multiplication", PLDI 1994, Sec. 4): the 33-bit multiplier
// 2^32 + m; for n < 2^31 the sum t + n cannot overflow 32 bits, so the
// shift needs no halving step.
static void host_divider(unsigned d, unsigned* m, int* s)
{
    int k = 0;
    while ((1ull << k) < d) ++k;
    *s = k;
    *m = (unsigned)(((1ull << 32) * ((1ull << k) - d)) / d + 1);
}

void fill_params(const Solver& s, StepParams& p)
{
    std::memset(&p, 0, sizeof p);
    p.f = s.f;
    p.q = s.q;
    p.status = s.status;
    p.nx = s.nx;
    p.ny = s.ny;
    p.nz = s.nz;
    p.N = (int)s.N;
    p.plane = s.nx * s.ny;
    host_divider((unsigned)s.nx, &p.div_nx_m, &p.div_nx_s);
    host_divider((unsigned)p.plane, &p.div_plane_m, &p.div_plane_s);
    for (int a = 0; a < 3; ++a) {
        const double l = s.lam[a];
        p.lam[a] = (float)l;
        p.inv_lam[a] = (float)(1.0 / l);
        p.inv_lam2[a] = (float)(1.0 / (l * l));
        p.inv_2lam[a] = (float)(0.5 / l);
        p.lam2m3T[a] = (float)(l * l - 3.0 * s.T);
    }
    for (int a = 0; a < 3; ++a) {
        const double U0 = (a < s.D && shifted_storage(s.storage)) ? s.u_ref[a] : 0.0;
        double u0_eff = 0.0;
        base_triplet(s.T, s.lam[a], U0, p.base[a], &u0_eff);
        p.u0[a] = (float)u0_eff;
        p.j0[a] = (float)(s.rho_ref * u0_eff);
    }
    for (int i = 0; i < s.Q; ++i) {
        const int c[3] = {i % 3, (i / 3) % 3, i / 9};
        double b = 1.0;
        for (int a = 0; a < s.D; ++a) b *= (double)p.base[a][c[a]];
        p.bw[i] = (float)b;
    }
    for (int cx = 0; cx < 3; ++cx) {
        p.base_xr[cx] = (float)(s.rho_ref * (double)p.base[0][cx]);
        for (int cy = 0; cy < 3; ++cy)
            p.bxy_r[cx + 3 * cy] = (float)(s.rho_ref * (double)p.base[0][cx] * (double)p.base[1][cy]);
    }
    p.T = (float)s.T;
    p.omega = (float)s.omega;
    p.coef = (float)((2.0 - s.omega) / (2.0 * s.omega));
    p.rho_ref = (float)s.rho_ref;
    for (int a = 0; a < 3; ++a) p.g[a] = (float)s.g[a];
    p.forced = (s.g[0] != 0.0 || s.g[1] != 0.0 || s.g[2] != 0.0);
    p.walls_y = s.walls_y;
    p.eq_mode = s.eq_mode;
    p.parity = s.parity;
}

// Kernel form a step uses.  Automatic (0): once the second population array
// has been allocated, the single pass on the D3Q27 grids its TMEM kernel takes
// (x a multiple of 32 nodes, y of 16) and on periodic, unforced D2Q9 grids;
// the two-pass form otherwise (the fused in-place form, 4, reads less but
// runs slower, so only a request for it selects it).  The second-order equilibrium runs in the
// two-pass form; walls and the body force in the two-pass form or, on the
// TMEM geometry of D3Q27, the TMEM single pass (the D2Q9 single pass has
// neither).
static bool bounded_solver(const Solver* s)
{
    return s->walls_y || s->g[0] != 0.0 || s->g[1] != 0.0 || s->g[2] != 0.0;
}

bool auto_single(const Solver* s)
{
    if (s->eq_mode == 2) return false;
    return s->D == 3 ? elbm::single_tmem_geometry(*s) : !bounded_solver(s);
}

// The fused in-place form takes D3Q27 grids whose tile columns all fit the
// GPU at once, periodic and unforced, with the extended or product-form equilibrium.
static bool fused_applies(const Solver* s) { return s->fused_ok && !bounded_solver(s) && s->eq_mode != 2; }

int effective_kernel(const Solver* s)
{
    if (s->eq_mode == 2) return 1;
    if (s->kernel == 0) return (s->f2 && auto_single(s)) ? 3 : 1;
    if (s->kernel == 4) return fused_applies(s) ? 4 : 1;
    if (!bounded_solver(s)) return s->kernel;
    return (s->kernel == 3 && elbm::single_tmem_geometry(*s)) ? 3 : 1;
}

}  // namespace elbm

using elbm::Solver;

namespace {

int check_status(elbm_solver* s)
{
    int st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, s->status, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (st != 0) {
        cudaMemsetAsync(s->status, 0, sizeof(int), s->stream);
        cudaStreamSynchronize(s->stream);
        return fail(st, "a bounded device-side wait gave up (code %d); the state is undefined", st);
    }
    return ELBM_OK;
}

bool shifted_storage_mode(int storage) { return storage != ELBM_F32; }

// The graph-pipelined step bakes the parameter block into its kernel nodes;
// any change of parameters drops the graphs (they are rebuilt on demand).
void drop_graphs(elbm_solver* s)
{
    for (auto& g : s->graph_exec) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

size_t population_bytes(const elbm_solver* s)
{
    // 16 bytes of tail padding: 16-bit populations are staged as the 4-byte
    // word that contains them, which for the last one reaches past the array
    return (size_t)s->Q * s->N * elbm::storage_bytes(s->storage) + 16;
}

// The single-pass form needs a second population array.  Requested
// explicitly (kernel 3), a failed allocation is an error; for the automatic
// form (kernel 0) on a grid the TMEM single pass takes it is an attempt, and
// without the array the solver steps in the two-pass form.  The in-place forms
// (1, 2, 4) release it: the current state always sits in s->f.
int ensure_second_array(elbm_solver* s, int kernel)
{
    if (kernel == 1 || kernel == 2 || kernel == 4) {
        if (s->f2) {
            cudaFreeAsync(s->f2, s->stream);  // stream-ordered: after the queued steps that use it
            s->f2 = nullptr;
            s->bytes -= population_bytes(s);
        }
        return ELBM_OK;
    }
    if (s->f2) return ELBM_OK;
    if (kernel == 0 && !(s->D == 2 || elbm::single_tmem_geometry(*s))) return ELBM_OK;
    cudaError_t e = cudaMallocAsync(&s->f2, population_bytes(s), s->stream);
    if (e != cudaSuccess) {
        s->f2 = nullptr;
        if (kernel == 0) {
            (void)cudaGetLastError();  // the automatic form falls back to the two-pass form
            return ELBM_OK;
        }
        return cuda_fail(e, "second population array");
    }
    s->bytes += population_bytes(s);
    return ELBM_OK;
}

}  // namespace

extern "C" {

const char* elbm_last_error(void) { return g_err; }

int elbm_create(int lattice, int nx, int ny, int nz, const double* stretch, double T, double nu,
                int storage, void* stream, elbm_solver** out)
{
    g_err[0] = 0;
    if (!out) return fail(ELBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (lattice != ELBM_D2Q9 && lattice != ELBM_D3Q27) return fail(ELBM_ERR_ARG, "lattice must be 9 or 27");
    const int D = lattice == ELBM_D2Q9 ? 2 : 3;
    if (nx < 3 || ny < 3) return fail(ELBM_ERR_ARG, "nx and ny must be >= 3");
    if (D == 2 && nz != 1) return fail(ELBM_ERR_ARG, "D2Q9 needs nz == 1");
    if (D == 3 && nz < 3) return fail(ELBM_ERR_ARG, "D3Q27 needs nz >= 3");
    const long long N = (long long)nx * ny * nz;
    if (N * lattice >= (1ll << 31)) return fail(ELBM_ERR_ARG, "grid too large: nx*ny*nz*Q must be < 2^31");
    double lam[3] = {1.0, 1.0, 1.0};
    if (stretch)
        for (int a = 0; a < D; ++a) lam[a] = stretch[a];
    for (int a = 0; a < D; ++a)
        if (!(lam[a] > 0.0) || !std::isfinite(lam[a])) return fail(ELBM_ERR_ARG, "stretch must be finite and > 0");
    if (!(T > 0.0) || !std::isfinite(T)) return fail(ELBM_ERR_ARG, "T must be finite and > 0");
    double lmin2 = lam[0] * lam[0];
    for (int a = 1; a < D; ++a) lmin2 = std::min(lmin2, lam[a] * lam[a]);
    if (T >= lmin2) return fail(ELBM_ERR_UNREALIZABLE, "T = %g >= min lam^2 = %g: rest population not positive", T, lmin2);
    if (!(nu > 0.0) || !std::isfinite(nu)) return fail(ELBM_ERR_ARG, "nu must be finite and > 0");
    if (storage != ELBM_F32 && storage != ELBM_F16_SHIFT && storage != ELBM_BF16_SHIFT && storage != ELBM_F32_SHIFT)
        return fail(ELBM_ERR_ARG, "unknown storage mode %d", storage);

    static std::atomic<long long> next_uid{0};
    elbm_solver* s = new elbm_solver();
    s->uid = ++next_uid;
    s->lattice = lattice;
    s->D = D;
    s->Q = lattice;
    s->nx = nx;
    s->ny = ny;
    s->nz = nz;
    s->N = N;
    s->storage = storage;
    for (int a = 0; a < 3; ++a) s->lam[a] = lam[a];
    s->T = T;
    s->nu = nu;
    s->omega = 1.0 / (nu / T + 0.5);  // Eq. nu with R = 1, delta t = 1
    s->stream = (cudaStream_t)stream;

    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
    const size_t qbytes = (size_t)D * N * sizeof(float);
    // stream-ordered allocations: freeing them later does not synchronise the device
    if (e == cudaSuccess) e = cudaMallocAsync(&s->f, population_bytes(s), s->stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&s->q, qbytes, s->stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&s->status, sizeof(int), s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->status, 0, sizeof(int), s->stream);
    if (e != cudaSuccess) {
        int rc = cuda_fail(e, "elbm_create");
        elbm_destroy(s);
        return rc;
    }
    s->bytes = population_bytes(s) + qbytes;
    s->fused_ok = elbm::fused_available(*s) ? 1 : 0;
    (void)cudaGetLastError();  // an occupancy query that failed only means "no fused form"
    const int rc = ensure_second_array(s, s->kernel);
    if (rc != ELBM_OK) {
        elbm_destroy(s);
        return rc;
    }
    *out = s;
    return ELBM_OK;
}

void elbm_destroy(elbm_solver* s)
{
    if (!s) return;
    drop_graphs(s);
    // stream-ordered frees: they wait for the solver's queued work, not the device
    for (void* ptr : {s->f, s->f2, (void*)s->q, (void*)s->status, (void*)s->mom, (void*)s->partials,
                      (void*)s->red_out, (void*)s->progress})
        if (ptr) cudaFreeAsync(ptr, s->stream);
    delete s;
}

int elbm_set_option(elbm_solver* s, int key, double value)
{
    if (!s) return fail(ELBM_ERR_ARG, "solver is NULL");
    drop_graphs(s);
    switch (key) {
        case ELBM_OPT_EQUILIBRIUM:
            if (value != 0.0 && value != 1.0 && value != 2.0) return fail(ELBM_ERR_ARG, "equilibrium must be 0, 1 or 2");
            if (value == 2.0 && (s->u_ref_auto || s->u_ref[0] != 0.0 || s->u_ref[1] != 0.0 || s->u_ref[2] != 0.0))
                return fail(ELBM_ERR_ARG, "the second-order equilibrium needs the rest storage baseline (U0 = 0)");
            s->eq_mode = (int)value;
            return ELBM_OK;
        case ELBM_OPT_KERNEL: {
            if (value != 0.0 && value != 1.0 && value != 2.0 && value != 3.0 && value != 4.0)
                return fail(ELBM_ERR_ARG, "kernel must be 0, 1, 2, 3 or 4");
            const int rc = ensure_second_array(s, (int)value);
            if (rc != ELBM_OK) return rc;
            s->kernel = (int)value;
            return ELBM_OK;
        }
        case ELBM_OPT_RHO_REF:
            if (!(value > 0.0) || !std::isfinite(value)) return fail(ELBM_ERR_ARG, "rho_ref must be > 0");
            if (s->initialised) return fail(ELBM_ERR_STATE, "rho_ref must be set before init");
            s->rho_ref = value;
            return ELBM_OK;
        case ELBM_OPT_U_REF_X:
        case ELBM_OPT_U_REF_Y:
        case ELBM_OPT_U_REF_Z: {
            const int a = key - ELBM_OPT_U_REF_X;
            if (!std::isfinite(value)) return fail(ELBM_ERR_ARG, "baseline velocity must be finite");
            if (s->initialised) return fail(ELBM_ERR_STATE, "the baseline velocity must be set before init");
            if (a >= s->D) return value == 0.0 ? ELBM_OK : fail(ELBM_ERR_ARG, "no such axis for this lattice");
            if (s->eq_mode == 2 && value != 0.0)
                return fail(ELBM_ERR_ARG, "the second-order equilibrium needs the rest storage baseline (U0 = 0)");
            float tri[3];
            double ueff;
            if (!elbm::base_triplet(s->T, s->lam[a], value, tri, &ueff))
                return fail(ELBM_ERR_UNREALIZABLE, "baseline velocity %g gives a non-positive baseline population", value);
            s->u_ref[a] = value;
            s->u_ref_auto = 0;
            return ELBM_OK;
        }
        case ELBM_OPT_U_REF_AUTO:
            if (value != 0.0 && value != 1.0) return fail(ELBM_ERR_ARG, "u_ref_auto must be 0 or 1");
            if (s->initialised) return fail(ELBM_ERR_STATE, "the baseline velocity must be set before init");
            s->u_ref_auto = (int)value;
            return ELBM_OK;
        case ELBM_OPT_FORCE_X:
        case ELBM_OPT_FORCE_Y:
        case ELBM_OPT_FORCE_Z: {
            const int a = key - ELBM_OPT_FORCE_X;
            if (!std::isfinite(value)) return fail(ELBM_ERR_ARG, "body force must be finite");
            if (a >= s->D) return value == 0.0 ? ELBM_OK : fail(ELBM_ERR_ARG, "no such axis for this lattice");
            s->g[a] = value;
            return ELBM_OK;
        }
        case ELBM_OPT_WALLS_Y:
            if (value != 0.0 && value != 1.0) return fail(ELBM_ERR_ARG, "walls_y must be 0 or 1");
            s->walls_y = (int)value;
            return ELBM_OK;
        default:
            return fail(ELBM_ERR_ARG, "unknown option %d", key);
    }
}

static cudaError_t ensure_reduce_scratch(elbm_solver* s);

static cudaError_t stage_to_device(const void* host, size_t bytes, void** dev, cudaStream_t st)
{
    cudaError_t e = cudaMallocAsync(dev, bytes, st);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(*dev, host, bytes, cudaMemcpyHostToDevice, st);
}

// The device address of page-locked host memory mapped into the device's
// address space (cudaHostAlloc, cudaHostRegister), else nullptr (pageable
// memory).  Kernels then read or write such a buffer in place: the transfer
// runs at the link's rate inside the kernel, with no staging copy.
static void* mapped_host(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int elbm_init(elbm_solver* s, const void* rho, const void* u, int dtype, int on_device)
{
    (void)cudaGetLastError();  // a stale error of an earlier call is not this call's
    if (!s || !rho || !u) return fail(ELBM_ERR_ARG, "NULL argument");
    if (dtype != ELBM_DTYPE_F32 && dtype != ELBM_DTYPE_F64) return fail(ELBM_ERR_ARG, "dtype must be F32 or F64");
    const size_t es = dtype == ELBM_DTYPE_F64 ? 8 : 4;
    const void* drho = rho;
    const void* du = u;
    void *t1 = nullptr, *t2 = nullptr;
    cudaError_t e = cudaSuccess;
    void* mr = on_device ? nullptr : mapped_host(rho);
    void* mu = on_device ? nullptr : mapped_host(u);
    const bool in_place = mr && mu;  // page-locked host fields: read where they are
    if (in_place) {
        drho = mr;
        du = mu;
    } else if (!on_device) {
        e = stage_to_device(rho, es * s->N, &t1, s->stream);
        if (e == cudaSuccess) e = stage_to_device(u, es * s->D * s->N, &t2, s->stream);
        drho = t1;
        du = t2;
    }
    if (e == cudaSuccess && s->u_ref_auto && shifted_storage_mode(s->storage)) {
        // baseline velocity = mean velocity sum(rho u)/sum(rho) of the given field
        e = ensure_reduce_scratch(s);
        if (e == cudaSuccess)
            e = (s->D == 2) ? elbm::field_sums_impl<2>(*s, drho, du, dtype, &s->launches)
                            : elbm::field_sums_impl<3>(*s, drho, du, dtype, &s->launches);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->host_red, s->red_out, sizeof(double) * ELBM_NRED, cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e == cudaSuccess) {
            for (int a = 0; a < s->D; ++a) {
                const double U0 = s->host_red[1 + a] / s->host_red[0];
                float tri[3];
                double ueff;
                s->u_ref[a] = (std::isfinite(U0) && elbm::base_triplet(s->T, s->lam[a], U0, tri, &ueff)) ? U0 : 0.0;
            }
        }
    }
    if (e == cudaSuccess)
        e = (s->D == 2) ? elbm::init_impl<2>(*s, drho, du, dtype, &s->launches)
                        : elbm::init_impl<3>(*s, drho, du, dtype, &s->launches);
    if (!on_device) {
        if (t1) cudaFreeAsync(t1, s->stream);
        if (t2) cudaFreeAsync(t2, s->stream);
    }
    if (e == cudaSuccess && in_place) e = cudaStreamSynchronize(s->stream);  // the caller's buffers are read
    if (e != cudaSuccess) return cuda_fail(e, "elbm_init");
    s->parity = 0;
    s->steps_done = 0;
    s->initialised = 1;
    drop_graphs(s);
    return ELBM_OK;
}

int elbm_step(elbm_solver* s, int n)
{
    (void)cudaGetLastError();  // a stale error of an earlier call is not this call's
    if (!s) return fail(ELBM_ERR_ARG, "solver is NULL");
    if (n < 0) return fail(ELBM_ERR_ARG, "n must be >= 0");
    if (!s->initialised) return fail(ELBM_ERR_STATE, "elbm_step before elbm_init");
    const int kernel = elbm::effective_kernel(s);
    cudaError_t e = cudaSuccess;
    int left = n;
    while (left > 0 && e == cudaSuccess) {
        if (kernel == 3 && s->parity == 0 && s->f2) {
            // single pass: own-location state in f, result in f2, then swap
            e = (s->D == 2) ? elbm::step_single_impl<2>(*s, s->f2, &s->launches)
                            : elbm::step_single_impl<3>(*s, s->f2, &s->launches);
            std::swap(s->f, s->f2);
            --left;
        } else if (kernel == 4) {
            // fused in place: one cooperative launch per step, progress counters on first use
            if (!s->progress) {
                const int nblocks = ((s->nx + 31) / 32) * ((s->ny + 7) / 8);
                e = cudaMallocAsync((void**)&s->progress, sizeof(unsigned long long) * nblocks, s->stream);
                if (e == cudaSuccess)
                    e = cudaMemsetAsync(s->progress, 0, sizeof(unsigned long long) * nblocks, s->stream);
                if (e != cudaSuccess) {
                    s->progress = nullptr;
                    break;
                }
                s->bytes += sizeof(unsigned long long) * nblocks;
            }
            e = elbm::step_fused_impl(*s, s->parity, s->progress, ++s->epoch, &s->launches);
            s->parity ^= 1;
            --left;
        } else if (kernel == 2) {
            if (!s->graph_exec[s->parity]) {
                e = (s->D == 2) ? elbm::build_step_graph_impl<2>(*s, s->parity, &s->graph_exec[s->parity], &s->graph_nodes)
                                : elbm::build_step_graph_impl<3>(*s, s->parity, &s->graph_exec[s->parity], &s->graph_nodes);
                if (e != cudaSuccess) break;
            }
            e = cudaGraphLaunch(s->graph_exec[s->parity], s->stream);
            s->launches += s->graph_nodes;
            s->parity ^= 1;
            --left;
        } else {
            // two-pass (also brings an odd-parity state back to the own-location layout)
            e = (s->D == 2) ? elbm::step_two_pass_impl<2>(*s, s->parity, &s->launches)
                            : elbm::step_two_pass_impl<3>(*s, s->parity, &s->launches);
            s->parity ^= 1;
            --left;
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "elbm_step");
    s->steps_done += n;
    return ELBM_OK;
}

int elbm_sync(elbm_solver* s)
{
    if (!s) return fail(ELBM_ERR_ARG, "solver is NULL");
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "elbm_sync");
    return check_status(s);
}

int elbm_moments(elbm_solver* s, void* rho, void* u, int dtype, int on_device)
{
    (void)cudaGetLastError();  // a stale error of an earlier call is not this call's
    if (!s || !rho || !u) return fail(ELBM_ERR_ARG, "NULL argument");
    if (dtype != ELBM_DTYPE_F32 && dtype != ELBM_DTYPE_F64) return fail(ELBM_ERR_ARG, "dtype must be F32 or F64");
    if (!s->initialised) return fail(ELBM_ERR_STATE, "elbm_moments before elbm_init");
    const size_t es = dtype == ELBM_DTYPE_F64 ? 8 : 4;
    void *drho = rho, *du = u;
    cudaError_t e = cudaSuccess;
    void* mr = on_device ? nullptr : mapped_host(rho);
    void* mu = on_device ? nullptr : mapped_host(u);
    const bool staged = !on_device && !(mr && mu);  // page-locked host fields are written in place
    if (!on_device && !staged) {
        drho = mr;
        du = mu;
    }
    if (staged) {
        e = cudaMallocAsync(&drho, es * s->N, s->stream);
        if (e == cudaSuccess) e = cudaMallocAsync(&du, es * s->D * s->N, s->stream);
    }
    if (e == cudaSuccess)
        e = (s->D == 2) ? elbm::moments_impl<2>(*s, drho, du, dtype, &s->launches)
                        : elbm::moments_impl<3>(*s, drho, du, dtype, &s->launches);
    if (staged) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(rho, drho, es * s->N, cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(u, du, es * s->D * s->N, cudaMemcpyDeviceToHost, s->stream);
        cudaFreeAsync(drho, s->stream);
        cudaFreeAsync(du, s->stream);
    }
    cudaError_t e2 = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return cuda_fail(e, "elbm_moments");
    return check_status(s);
}

int elbm_get_populations(elbm_solver* s, void* f, int dtype, int on_device)
{
    (void)cudaGetLastError();  // a stale error of an earlier call is not this call's
    if (!s || !f) return fail(ELBM_ERR_ARG, "NULL argument");
    if (dtype != ELBM_DTYPE_F32 && dtype != ELBM_DTYPE_F64) return fail(ELBM_ERR_ARG, "dtype must be F32 or F64");
    if (!s->initialised) return fail(ELBM_ERR_STATE, "elbm_get_populations before init");
    const size_t bytes = (dtype == ELBM_DTYPE_F64 ? 8 : 4) * (size_t)s->Q * s->N;
    void* df = f;
    cudaError_t e = cudaSuccess;
    if (!on_device) e = cudaMallocAsync(&df, bytes, s->stream);
    if (e == cudaSuccess)
        e = (s->D == 2) ? elbm::get_populations_impl<2>(*s, df, dtype, &s->launches)
                        : elbm::get_populations_impl<3>(*s, df, dtype, &s->launches);
    if (!on_device && e == cudaSuccess) e = cudaMemcpyAsync(f, df, bytes, cudaMemcpyDeviceToHost, s->stream);
    if (!on_device) cudaFreeAsync(df, s->stream);
    cudaError_t e2 = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return cuda_fail(e, "elbm_get_populations");
    return check_status(s);
}

int elbm_set_populations(elbm_solver* s, const void* f, int dtype, int on_device)
{
    (void)cudaGetLastError();  // a stale error of an earlier call is not this call's
    if (!s || !f) return fail(ELBM_ERR_ARG, "NULL argument");
    if (dtype != ELBM_DTYPE_F32 && dtype != ELBM_DTYPE_F64) return fail(ELBM_ERR_ARG, "dtype must be F32 or F64");
    const size_t bytes = (dtype == ELBM_DTYPE_F64 ? 8 : 4) * (size_t)s->Q * s->N;
    const void* df = f;
    void* tmp = nullptr;
    cudaError_t e = cudaSuccess;
    if (!on_device) {
        e = stage_to_device(f, bytes, &tmp, s->stream);
        df = tmp;
    }
    if (e == cudaSuccess)
        e = (s->D == 2) ? elbm::set_populations_impl<2>(*s, df, dtype, &s->launches)
                        : elbm::set_populations_impl<3>(*s, df, dtype, &s->launches);
    if (tmp) cudaFreeAsync(tmp, s->stream);
    cudaError_t e2 = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return cuda_fail(e, "elbm_set_populations");
    s->parity = 0;
    s->initialised = 1;
    return ELBM_OK;
}

static cudaError_t ensure_reduce_scratch(elbm_solver* s)
{
    cudaError_t e = cudaSuccess;
    if (!s->mom) {
        s->red_blocks = std::max(1, std::min(8 * s->num_sms, (int)((s->N + 255) / 256)));
        e = cudaMallocAsync((void**)&s->mom, 5 * sizeof(float) * (size_t)s->N, s->stream);
        if (e == cudaSuccess) e = cudaMallocAsync((void**)&s->partials, sizeof(double) * ELBM_NRED * s->red_blocks, s->stream);
        if (e == cudaSuccess) e = cudaMallocAsync((void**)&s->red_out, sizeof(double) * ELBM_NRED, s->stream);
        if (e != cudaSuccess) {
            if (s->mom) cudaFreeAsync(s->mom, s->stream);
            if (s->partials) cudaFreeAsync(s->partials, s->stream);
            if (s->red_out) cudaFreeAsync(s->red_out, s->stream);
            s->mom = nullptr;
            s->partials = s->red_out = nullptr;
            return e;
        }
        s->bytes += 5 * sizeof(float) * (size_t)s->N + sizeof(double) * ELBM_NRED * (s->red_blocks + 1);
    }
    return e;
}

int elbm_reduce(elbm_solver* s, double* out)
{
    (void)cudaGetLastError();  // a stale error of an earlier call is not this call's
    if (!s || !out) return fail(ELBM_ERR_ARG, "NULL argument");
    if (!s->initialised) return fail(ELBM_ERR_STATE, "elbm_reduce before init");
    cudaError_t e = ensure_reduce_scratch(s);
    if (e != cudaSuccess) return cuda_fail(e, "elbm_reduce scratch");
    e = (s->D == 2) ? elbm::reduce_impl<2>(*s, &s->launches) : elbm::reduce_impl<3>(*s, &s->launches);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->host_red, s->red_out, sizeof(double) * ELBM_NRED, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "elbm_reduce");
    std::memcpy(out, s->host_red, sizeof(double) * ELBM_NRED);
    int rc = check_status(s);
    if (rc != ELBM_OK) return rc;
    if (out[10] > 0.0) return fail(ELBM_ERR_NONFINITE, "%.0f nodes hold non-finite values", out[10]);
    return ELBM_OK;
}

int elbm_mode_sums(elbm_solver* s, const double* k, const double* dir, double* out)
{
    (void)cudaGetLastError();  // a stale error of an earlier call is not this call's
    if (!s || !k || !dir || !out) return fail(ELBM_ERR_ARG, "NULL argument");
    if (!s->initialised) return fail(ELBM_ERR_STATE, "elbm_mode_sums before init");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(k[a]) || !std::isfinite(dir[a])) return fail(ELBM_ERR_ARG, "k and dir must be finite");
    cudaError_t e = ensure_reduce_scratch(s);
    if (e != cudaSuccess) return cuda_fail(e, "elbm_mode_sums scratch");
    e = (s->D == 2) ? elbm::mode_sums_impl<2>(*s, k, dir, &s->launches)
                    : elbm::mode_sums_impl<3>(*s, k, dir, &s->launches);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->host_red, s->red_out, sizeof(double) * ELBM_NRED, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "elbm_mode_sums");
    out[0] = s->host_red[0];
    out[1] = s->host_red[1];
    return check_status(s);
}

int elbm_kernel_form(const elbm_solver* s, int* variant)
{
    if (variant) *variant = 0;
    if (!s) return fail(ELBM_ERR_ARG, "solver is NULL");
    const int form = elbm::effective_kernel(s);
    if (form == 3 && variant) *variant = elbm::single_pass_variant(*s);
    return form;
}

long long elbm_cells(const elbm_solver* s) { return s ? s->N : 0; }
long long elbm_steps_done(const elbm_solver* s) { return s ? s->steps_done : 0; }
double elbm_omega(const elbm_solver* s) { return s ? s->omega : 0.0; }
long long elbm_device_bytes(const elbm_solver* s) { return s ? (long long)s->bytes : 0; }
long long elbm_launch_count(const elbm_solver* s) { return s ? s->launches : 0; }

int elbm_get_u_ref(const elbm_solver* s, double* out)
{
    if (!s || !out) return fail(ELBM_ERR_ARG, "NULL argument");
    for (int a = 0; a < 3; ++a) out[a] = (a < s->D && shifted_storage_mode(s->storage)) ? s->u_ref[a] : 0.0;
    return ELBM_OK;
}

}  // extern "C"
