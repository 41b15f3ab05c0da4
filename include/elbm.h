/*
 * elbm.h — C ABI of the GB300 (sm_103a) extended lattice Boltzmann library.
 *
 * The library advances the LBGK equation (Eq. LBGK) with the extended
 * product-form equilibrium f*_i = rho Psi_i(u, P*, lam) (Eqs. prod, 27eqext)
 * whose diagonal pressure P*_aa = T + u_a^2 + (2 - omega)/(2 rho omega) d_a Q~_aaa
 * carries the central difference of the diagonal anomaly
 * Q~_aaa = rho u_a (lam_a^2 - 3 T) - rho u_a^3 (Eqs. Deviation, Paastar1), on the
 * D2Q9 and D3Q27 lattices with velocities v_i = (lam_x c_ix, lam_y c_iy, lam_z c_iz)
 * (Eqs. d3q27vel, d3q27velSTRETCHED).  Units: R = 1, delta t = 1; the node
 * spacing along axis a is lam_a; omega follows from nu = (1/omega - 1/2) T (Eq. nu).
 *
 * Conventions shared by every entry point
 *   - Population index i = (cx+1) + 3 (cy+1) + 9 (cz+1)  (Q = 27),
 *                      i = (cx+1) + 3 (cy+1)             (Q = 9);
 *     the opposite direction of i is Q-1-i.
 *   - Caller-side fields are structure-of-arrays with x fastest:
 *       rho[nz][ny][nx], u[D][nz][ny][nx], f[Q][nz][ny][nx].
 *     For D2Q9, nz must be 1 and u has two components.
 *   - Pointers flagged "on_device" are CUDA device pointers that must be valid
 *     on the solver's stream; otherwise they are host pointers.
 *   - Every int-returning call returns ELBM_OK (0) or a negative ELBM_ERR_*
 *     code and never throws; elbm_last_error() gives the message of the
 *     calling thread's last failure.
 *   - All device work is enqueued on the stream given to elbm_create.  Calls
 *     that return data to the host synchronise that stream.
 *
 * The library owns the device memory it allocates (populations, the anomaly
 * field and reduction partials); elbm_destroy frees it.  The caller owns every
 * buffer it passes in.
 */
#ifndef ELBM_H
#define ELBM_H

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ codes */
#define ELBM_OK                0
#define ELBM_ERR_ARG          -1  /* invalid argument or size                         */
#define ELBM_ERR_UNREALIZABLE -2  /* T >= min lam_a^2: rest population not positive   */
#define ELBM_ERR_OOM          -3  /* device allocation failed                         */
#define ELBM_ERR_CUDA         -4  /* a CUDA runtime call or a launch failed           */
#define ELBM_ERR_NONFINITE    -5  /* a diagnostic found NaN/Inf in the state          */
#define ELBM_ERR_TIMEOUT      -6  /* a bounded device-side wait gave up               */
#define ELBM_ERR_STATE        -7  /* call out of order (e.g. step before init)        */

/* ---------------------------------------------------------------- lattices */
#define ELBM_D2Q9   9
#define ELBM_D3Q27 27

/* --------------------------------------------------------- storage of f_i */
/* Collision arithmetic is FP32 in every mode.  "SHIFT" modes store
 * g_i = f_i - w_i rho_ref with w_i = Psi_i(0, T, lam) the rest equilibrium at the
 * run's T and stretch (rho_ref = 1 unless set by ELBM_OPT_RHO_REF before init;
 * see ELBM_OPT_U_REF_* for a moving baseline); half-precision stores round to
 * nearest even. */
#define ELBM_F32         0  /* f_i as float                       (4 B/population) */
#define ELBM_F16_SHIFT   1  /* g_i as IEEE half                   (2 B/population) */
#define ELBM_BF16_SHIFT  2  /* g_i as bfloat16                    (2 B/population) */
#define ELBM_F32_SHIFT   3  /* g_i as float                       (4 B/population) */

/* ------------------------------------------------------- caller dtypes */
#define ELBM_DTYPE_F32 0
#define ELBM_DTYPE_F64 1

/* ----------------------------------------------------------- options */
/* ELBM_OPT_EQUILIBRIUM: 0 = extended equilibrium (Eq. 27eqext, default);
 *   1 = product-form equilibrium without the correction (Eq. 27eq);
 *   2 = product form truncated to second order in u (the conventional
 *       equilibrium of Sec. III preamble; two-pass form, rest storage baseline). */
#define ELBM_OPT_EQUILIBRIUM 1
/* ELBM_OPT_KERNEL: the form of the step; every form evaluates the same per-node
 *   arithmetic and gives bit-identical results.
 *   0 = automatic (the default): the single pass (form 3) on D3Q27 grids
 *       with nx a multiple of 32 and ny of 16 (TMEM kernel) and on periodic,
 *       unforced D2Q9 grids, for which elbm_create (or setting this option)
 *       allocates the second population array -- twice the population
 *       memory; if that allocation fails the solver keeps one array and steps
 *       in the two-pass form.  Other D3Q27 grids, D2Q9 with walls or a force,
 *       and the second-order equilibrium: the two-pass form.
 *       elbm_kernel_form() reports the choice;
 *   1 = two-pass, in place: an anomaly pass over the grid, then the collide pass;
 *   2 = graph-pipelined, in place: a CUDA graph of per-chunk anomaly and collide
 *       kernels, so that the collide kernels re-read populations from L2;
 *       forms 1 and 2 release a second population array if one is held;
 *   4 = fused in place (D3Q27; periodic, unforced, extended or product-form
 *       equilibrium): one array in the AA layout, one cooperative launch per
 *       step in which a block owns a 32 x 8 tile column, keeps each node's
 *       populations in registers from its anomaly to its collision one plane
 *       later, and exchanges the anomaly with the neighbouring tile columns
 *       through the anomaly field and progress counters (bounded waits), so
 *       every population is read once.  Needs every tile column resident at
 *       once (at most two per SM); other grids, walls, force and the
 *       second-order equilibrium take the two-pass form.  Releases a second
 *       array if one is held;
 *   3 = single pass with a second population array: every block recomputes
 *       the anomaly around its tile and reads the populations once.  D3Q27:
 *       TMA-fed with the populations parked in tensor memory when nx is a
 *       multiple of 32 and ny of 16; 32 x 8 TMA tiles when ny is a multiple
 *       of 8; cp.async-staged otherwise.  D2Q9: strips of 126 columns
 *       marching along y, any grid.  Setting it allocates the second array.
 *   The second-order equilibrium always runs in the two-pass form; walls and
 *   the body force run in form 3 only on the D3Q27 TMEM geometry (nx a
 *   multiple of 32, ny of 16) and in the two-pass form otherwise. */
#define ELBM_OPT_KERNEL      2
/* ELBM_OPT_RHO_REF: reference density of the shifted storage (before init). */
#define ELBM_OPT_RHO_REF     3
/* ELBM_OPT_FORCE_X/Y/Z: constant body-force acceleration g (channel flow,
 *   Sec. III.E); applied as f_i += f^eq_i(rho, u + g) - f^eq_i(rho, u). */
#define ELBM_OPT_FORCE_X     4
#define ELBM_OPT_FORCE_Y     5
#define ELBM_OPT_FORCE_Z     6
/* ELBM_OPT_WALLS_Y: 1 = half-way bounce-back walls below y = 0 and above
 *   y = ny-1 (periodic otherwise); the anomaly's ghost value beyond a wall is
 *   the negated value of the wall-adjacent node. */
#define ELBM_OPT_WALLS_Y     7
/* ELBM_OPT_U_REF_X/Y/Z: velocity U0 of the storage baseline of the SHIFT modes
 *   (before init).  Stored values are g_i = f_i - rho_ref b_i with
 *   b_i = Psi_i(U0, T + U0^2, lam), the product-form equilibrium of (rho_ref, U0)
 *   (Eqs. prod, 27eq); U0 = 0 (the default) gives the rest weights w_i.  A U0
 *   near the flow's mean velocity shrinks the stored values and so the
 *   rounding error of half-precision storage.  Ignored by ELBM_F32. */
#define ELBM_OPT_U_REF_X     8
#define ELBM_OPT_U_REF_Y     9
#define ELBM_OPT_U_REF_Z    10
/* ELBM_OPT_U_REF_AUTO: 1 = at elbm_init set U0 to the mean velocity
 *   sum(rho u) / sum(rho) of the given field (conserved on periodic grids). */
#define ELBM_OPT_U_REF_AUTO 11

/* ------------------------------------------------------- diagnostics */
/* elbm_reduce output, all accumulated in FP64 over every node (sums, not means):
 *  [0] sum rho          [1..3] sum rho u_a        [4] sum rho |u|^2
 *  [5] sum |u|^2        [6] sum |curl u|^2 (central differences, spacing lam)
 *  [7] sum (d_x u_x)^2  [8] sum u_x^2             [9] min_i,x f_i (realizability)
 *  [10] number of nodes with a non-finite rho or u  [11] max |u|
 *  [12] with walls: sum over the nodes next to either wall of the wall-normal
 *       gradient of u_x, (9 u_x(first node) - u_x(second node)) / (3 lam_y)
 *       (quadratic through the no-slip wall half a spacing away); the mean
 *       wall shear stress is rho nu [12] / (2 nx nz).  0 without walls.
 *  With walls, y-differences take the velocity beyond a wall as the negated
 *  value of the wall-adjacent node.                                            */
#define ELBM_NRED 13

typedef struct elbm_solver elbm_solver;

/*
 * Create a solver for one periodic grid.
 *   lattice  ELBM_D2Q9 or ELBM_D3Q27.
 *   nx,ny,nz nodes per axis, each >= 3 (nz = 1 for D2Q9); nx*ny*nz*Q < 2^31.
 *   stretch  lam_x, lam_y, lam_z > 0 (Eq. d3q27velSTRETCHED); stretch[2] is
 *            ignored for D2Q9.  NULL means all ones.
 *   T        temperature, 0 < T < min_a lam_a^2 (so that Psi_0 > 0 at rest).
 *   nu       kinematic viscosity > 0; omega = 1/(nu/T + 1/2) (Eq. nu).
 *   storage  ELBM_F32, ELBM_F16_SHIFT, ELBM_BF16_SHIFT or ELBM_F32_SHIFT.
 *   stream   cudaStream_t to enqueue on (NULL: the legacy default stream).
 * On success *out owns the populations; the state is undefined until elbm_init
 * or elbm_set_populations.
 */
int elbm_create(int lattice, int nx, int ny, int nz, const double* stretch, double T,
                double nu, int storage, void* stream, elbm_solver** out);

/* Free everything the solver owns.  NULL is a no-op. */
void elbm_destroy(elbm_solver* s);

/* Set an ELBM_OPT_* option.  Returns ELBM_ERR_ARG for an unknown key or value. */
int elbm_set_option(elbm_solver* s, int key, double value);

/*
 * Initialise the populations to the product-form equilibrium of the given
 * fields, f_i = rho Psi_i(u, T + u^2, lam) (Eq. 27eq), and reset the step count.
 *   rho  nx*ny*nz values; u  D*nx*ny*nz values; dtype ELBM_DTYPE_F32/F64.
 *   on_device  nonzero: rho and u are device pointers, read by work enqueued on
 *        the solver's stream (keep them valid until it has run).  Zero: host
 *        pointers.  Page-locked host buffers (cudaHostAlloc, cudaHostRegister)
 *        are read in place by the initialisation kernel, and the call returns
 *        once they have been read; pageable ones are copied to a device buffer
 *        first.
 */
int elbm_init(elbm_solver* s, const void* rho, const void* u, int dtype, int on_device);

/*
 * Advance n >= 0 time steps (Eq. LBGK with f* of Eq. 27eqext).  Asynchronous:
 * returns once the work is enqueued.  Each step: streaming, moments
 * (Eqs. density, momentum), the anomaly and its central difference, the
 * extended equilibrium, relaxation.
 */
int elbm_step(elbm_solver* s, int n);

/*
 * Density and velocity of the current (post-streaming) state, Eqs. density and
 * momentum.  With a body force the velocity is the half-step value u + g/2.
 * Synchronises the solver's stream.  on_device as for elbm_init: page-locked
 * host buffers are written in place by the moments kernel, pageable ones
 * through a device buffer.
 */
int elbm_moments(elbm_solver* s, void* rho, void* u, int dtype, int on_device);

/* Read / write the post-streaming populations f_i (unshifted) in the layout
 * f[Q][nz][ny][nx].  Writing resets the internal streaming parity. */
int elbm_get_populations(elbm_solver* s, void* f, int dtype, int on_device);
int elbm_set_populations(elbm_solver* s, const void* f, int dtype, int on_device);

/* FP64 diagnostics of the current state into out[ELBM_NRED] (host).  Synchronises.
 * Returns ELBM_ERR_NONFINITE (after filling out) if a node is non-finite. */
int elbm_reduce(elbm_solver* s, double* out);

/*
 * FP64 projection of the velocity on one Fourier mode, the amplitude
 * measurement of the shear-wave viscosity test (Sec. III.A):
 *   out[0] = sum_x (u(x) . dir) cos(k . x),  out[1] = sum_x (u(x) . dir) sin(k . x)
 * over every node, with x = (i lam_x, j lam_y, k lam_z) the node's physical
 * position, u the reported velocity (as elbm_moments gives it), k[3] the
 * wavevector in physical units and dir[3] the projection direction (the
 * z components are ignored for D2Q9).  The mode's amplitude is
 * 2 sqrt(out[0]^2 + out[1]^2) / N.  Synchronises the solver's stream.
 * Errors: ELBM_ERR_ARG (NULL or non-finite arguments), ELBM_ERR_STATE
 * (before init), ELBM_ERR_CUDA.
 */
int elbm_mode_sums(elbm_solver* s, const double* k, const double* dir, double* out);

/* Block the host until the solver's stream is idle. */
int elbm_sync(elbm_solver* s);

/* Kernel form the next elbm_step of s uses: 1 two-pass, 2 graph-pipelined,
 * 3 single pass, 4 fused in place (ELBM_OPT_KERNEL and the grid decide it;
 * see there), or
 * ELBM_ERR_ARG for NULL.  For form 3, *variant (if not NULL) receives the
 * single-pass kernel: 1 TMEM (32 x 16 tiles), 2 TMA (32 x 8 tiles),
 * 3 cp.async-staged (D3Q27), 4 the D2Q9 row march; 0 for the other forms.
 * Host-side query, no CUDA call. */
int elbm_kernel_form(const elbm_solver* s, int* variant);

/* Informational queries. */
long long elbm_cells(const elbm_solver* s);
long long elbm_steps_done(const elbm_solver* s);
double elbm_omega(const elbm_solver* s);
/* Device bytes of populations + anomaly field (+ reduction scratch once used). */
long long elbm_device_bytes(const elbm_solver* s);
/* Number of kernel launches this solver has issued since creation. */
long long elbm_launch_count(const elbm_solver* s);

/* ------------------------------------------------------------- batches */
/*
 * A batch advances many grids together: members share lattice, storage mode,
 * stream and kernel form, and may differ in size, stretch, T and nu; every
 * member's result is bit-identical to stepping it alone.  The batch holds the
 * solvers (it does not own them); destroy the batch before any of its solvers.
 * A batch holds at most 40 solvers.  Its form follows its members' kernel
 * form (ELBM_OPT_KERNEL and the grid decide it, as for elbm_step):
 *  - two-pass members (periodic, unforced, extended or product-form
 *    equilibrium): one batched step is two launches (anomaly pass and collide
 *    pass of the two-pass form, Eqs. LBGK, Deviation, Paastar1, 27eqext) over
 *    all members, from a table of their parameters in device memory of the
 *    batch, refreshed at every elbm_batch_step;
 *  - single-pass members (kernel form 3, D3Q27, two population arrays;
 *    walls and body force allowed where the single pass takes them): the
 *    members on the TMEM geometry (nx a multiple of 32, ny of 16) advance in
 *    one launch per step of a flattened kernel over a work list of (member,
 *    32 x 16 tile column, z segment) items, with every member's parameter block
 *    and tensor maps in device memory of the batch; the nsteps launches are
 *    captured as a CUDA graph and replayed.  The tile shape (32 x 16 columns
 *    with the TMEM kernel, 32 x 8 with the TMA kernel for periodic, unforced
 *    members with ny a multiple of 8), the segment depth (32, 16 or 8
 *    planes) and the order of the work list come from an autotuner (see
 *    elbm_batch_tuning), which may also choose per-member graphs: each
 *    member's sequence of solo single-pass launches captured once and replayed
 *    on private streams of the batch, side by side -- the form other
 *    single-pass members (32 x 8 TMA or cp.async kernels) always take.  If any
 *    member has walls or a body force, the flattened launch uses the kernel
 *    that honours them for every member (same bits for the others).
 * Any number of batches, of either form, may be live at once.
 * Mixing the forms in one batch returns ELBM_ERR_ARG.
 */
typedef struct elbm_batch elbm_batch;

int elbm_batch_create(elbm_solver* const* solvers, int n, elbm_batch** out);

/* Membership: a solver joins (same lattice, storage mode and stream as the
 * batch, initialised, not yet a member) or leaves between elbm_batch_step
 * calls; joining and leaving need no new CUDA graph unless the batch grows
 * beyond twice its earlier block count.  elbm_batch_size gives the member count. */
int elbm_batch_add(elbm_batch* b, elbm_solver* s);
int elbm_batch_remove(elbm_batch* b, elbm_solver* s);
int elbm_batch_size(const elbm_batch* b);

/* Advance every member by nsteps >= 0 steps, asynchronously with respect to
 * the device, ordered after earlier work on the members' stream.  Two-pass
 * form: the first batch of a (lattice, storage) kind in the process times one
 * real step with 128- and one with 256-thread blocks and keeps the faster for
 * every later batch of that kind (the autotuner); the launch sequence of
 * nsteps steps is captured once as a CUDA graph, on a stream of the batch's
 * own, and replayed.  Single-pass form: see above; a member's graphs are
 * released when it leaves (once their launches are complete). */
int elbm_batch_step(elbm_batch* b, int nsteps);

/* Chosen block size (0 before tuning, and for the single-pass form), the two
 * tuning step times in ms (128, 256) and the number of kernel launches issued
 * so far. */
int elbm_batch_info(const elbm_batch* b, int* block_size, double* tuned_ms, long long* launches);

/* Single-pass form: the configuration the last elbm_batch_step used and the
 * autotuner's timings of two steps of the whole batch in each candidate, for
 * the batch's tuning key (shared by every batch of the process with the same
 * storage mode, walls/force setting and floor(log2(nodes)) of its members).
 * Configurations 0..11 are the flattened launch -- one kernel per step over a
 * work list of tile columns of every member that kernel takes, the others as
 * per-member graphs; 12 is per-member graphs for every member:
 *   *config       0..12;
 *   *tile_rows    16 (TMEM kernel, configs 0..5), 8 (TMA kernel, configs
 *                 6..11; periodic, unforced members), 0 for config 12;
 *   *seg_planes   z planes per work item (32, 16 or 8; 0 for config 12);
 *   *interleaved  1 if the work list interleaves the members item by item,
 *                 0 if it takes them one after another;
 *   ms[ELBM_BATCH_CONFIGS]  tuning times in ms (-1 for one not yet timed).
 * Config c has tile_rows 16 for c < 6, 8 for c < 12; seg_planes 32, 16, 8
 * for c % 3 = 0, 1, 2; interleaved for c % 6 >= 3.  Any output pointer may be
 * NULL.  Returns ELBM_OK once the tuning of the key is complete (or when no
 * member takes a flattened kernel, or a configuration is pinned), 1 while it
 * is still in progress (the tuning spreads over calls with fewer than 26
 * steps; until it completes config 0 runs), ELBM_ERR_STATE for a two-pass
 * batch or before the first single-pass step. */
#define ELBM_BATCH_CONFIGS 13
int elbm_batch_tuning(const elbm_batch* b, int* config, int* tile_rows, int* seg_planes, int* interleaved,
                      double* ms);

/* Single-pass form: run configuration `config` (0..12, as elbm_batch_tuning
 * numbers them) from the next elbm_batch_step on instead of the autotuner's
 * choice; -1 returns to the autotuner.  Every configuration computes the same
 * bits.  ELBM_ERR_ARG for a value out of range, ELBM_ERR_STATE for a
 * two-pass batch. */
int elbm_batch_set_config(elbm_batch* b, int config);

void elbm_batch_destroy(elbm_batch* b);

/* Baseline velocity U0 of the shifted storage in use, out[3] (zeros for ELBM_F32). */
int elbm_get_u_ref(const elbm_solver* s, double* out);

/*
 * Allocation-free step.  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory themselves -- applications
 * that route every device allocation through their own pool, plugins whose
 * host framework forbids allocations on its threads, or code running where
 * cudaMalloc, which may synchronise the device, is not allowed.  It creates
 * no solver and calls no allocating routine; the caller passes the
 * populations and gets them back advanced.
 *   f        device pointer to float populations f[Q][nz][ny][nx] (unshifted,
 *            layout of elbm_get_populations), advanced in place by nsteps
 *            two-pass steps and left in that same layout.
 *   lattice, nx, ny, nz, stretch, T, nu: as for elbm_create;
 *            nx*ny*nz must not exceed 262144 (ELBM_ERR_ARG otherwise).
 *   stream   cudaStream_t to enqueue on; the call returns once the work is
 *            enqueued (synchronise the stream before reading f).
 * The anomaly field lives in a fixed 3 MiB device array that this library
 * holds on every GPU where it is used, until the process exits.  All calls
 * on a device share that array, so calls whose work overlaps on the GPU (for
 * example on two streams) race and give wrong results; serialise them.  The
 * first call on a device looks up the array's device address (set-up that
 * must not happen inside a stream capture), so make one call, for example
 * with nsteps = 0, before capturing.  That address is valid for the life of
 * the device's context: after a cudaDeviceReset do not call this entry point
 * on that device again in the same process.  A CUDA error still pending from
 * the caller's earlier work is reported as ELBM_ERR_CUDA and left in place;
 * nothing is launched then.  Errors: ELBM_ERR_ARG, ELBM_ERR_UNREALIZABLE,
 * ELBM_ERR_CUDA; elbm_last_error() has the message.
 */
int elbm_step_noalloc(int lattice, int nx, int ny, int nz, const double* stretch, double T,
                      double nu, float* f, int nsteps, void* stream);

/*
 * Self-test of the device-side failure detection (not part of the paper's
 * method).  The TMA-fed single-pass kernels wait on mbarriers; each wait is
 * bounded in time and, when it gives up, sets ELBM_ERR_TIMEOUT in the solver's
 * status word (read by elbm_sync, elbm_moments, elbm_get_populations and
 * elbm_reduce) instead of hanging.  This call runs that same bounded wait on
 * a barrier phase that never completes, with a bound of limit_ms (1..2000)
 * milliseconds, on `stream` (NULL: the legacy default stream), and waits for
 * it.  Returns ELBM_ERR_TIMEOUT when the wait gave up as designed (the
 * expected result); ELBM_ERR_ARG for a bound out of range; ELBM_ERR_CUDA on a
 * CUDA error; ELBM_ERR_STATE if no timeout was reported.  The device stays
 * usable afterwards.
 */
int elbm_selftest_wait_timeout(int limit_ms, void* stream);

/*
 * The same self-test for the other bounded wait of the library: the fused
 * in-place form (ELBM_OPT_KERNEL 4) waits for progress counters of the
 * neighbouring tile columns.  This call runs that wait on a counter that
 * nothing advances, with a bound of limit_ms (1..2000) milliseconds, and
 * returns as elbm_selftest_wait_timeout does (ELBM_ERR_TIMEOUT expected).
 */
int elbm_selftest_counter_timeout(int limit_ms, void* stream);

/* Message of the calling thread's last failure ("" if none). */
const char* elbm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ELBM_H */
