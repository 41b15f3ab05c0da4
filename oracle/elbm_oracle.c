/*
 * FP64 CPU oracle of the extended lattice Boltzmann (LBGK) time step of
 * Saadat, Dorschner & Karlin, "Extended Lattice Boltzmann Model" (arXiv 2101.04550).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * restatement of the method that the CUDA path is checked against.  Only the
 * test-suite, the smoke check and the CPU-baseline leg of the benchmark load
 * it.  It shares no code, header, table or constant with the CUDA library.
 *
 * Conventions (Sec. III preamble: R = 1; delta t = 1):
 *   - velocities c_i in {-1,0,1}^D (Eq. d3q27vel) with the population index
 *       i = (c_x+1) + 3 (c_y+1) + 9 (c_z+1)      (D = 3, Q = 27)
 *       i = (c_x+1) + 3 (c_y+1)                  (D = 2, Q = 9),
 *     so the opposite direction of i is Q-1-i;
 *   - particle velocities v_i = (lam_x c_ix, lam_y c_iy, lam_z c_iz)
 *     (Eq. d3q27velSTRETCHED): a population moves one node per step, so the
 *     node spacing along alpha is lam_alpha;
 *   - fields are stored structure-of-arrays, x fastest:
 *       f[i][z][y][x], rho[z][y][x], u[alpha][z][y][x].
 *
 * Every step is computed whole-grid by whole-grid in the order the paper
 * states the model: moments (Eqs. density, momentum), the diagonal anomaly
 * (Eq. Deviation), its central difference (Eq. Paastar1), the extended
 * pressure diagonal, the product-form extended equilibrium (Eqs. prod,
 * 27eqext), BGK relaxation and streaming (Eq. LBGK).  Populations are kept in
 * two arrays (read one, write the other).
 *
 * The paper gives neither a wall scheme nor a forcing scheme for its channel
 * (Sec. III.E); the wall and body-force options follow stated readings
 * (half-way bounce-back with a negated ghost anomaly; exact-difference
 * forcing) and are pinned by a closed form (uniform acceleration), exact
 * conservation, mirror symmetry and the steady Poiseuille parabola.
 *
 * Test infrastructure: the GPU library never calls this code.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Equilibrium used in the relaxation step. */
enum {
    ORA_EXTENDED = 0,     /* f* = rho Psi(u, P*, lam), Eq. 27eqext                  */
    ORA_PRODUCT = 1,      /* f^eq = rho Psi(u, P^eq, lam), Eq. 27eq (no correction) */
    ORA_SECOND_ORDER = 2  /* Eq. 27eq truncated to second order in u (Sec. III)     */
};

typedef struct {
    int D;              /* 2 or 3                                                    */
    int n[3];           /* nodes along x, y, z (n[2] = 1 when D = 2)                 */
    double lam[3];      /* stretching factors lam_alpha                              */
    double T;           /* temperature (R = 1)                                       */
    double omega;       /* relaxation frequency, Eq. nu                              */
    int mode;           /* ORA_EXTENDED / ORA_PRODUCT / ORA_SECOND_ORDER             */
    int walls_y;        /* 1: half-way bounce-back walls below y = 0 and above ny-1  */
    double g[3];        /* constant body-force acceleration (0 for none)             */
} ora_lattice;

/* ---------------------------------------------------------------- lattice */

int ora_Q(int D) { return D == 2 ? 9 : 27; }

/* Velocity c_i of population i (Eq. d3q27vel), in the ordering above. */
void ora_velocity(int D, int i, int c[3])
{
    c[0] = i % 3 - 1;
    c[1] = (i / 3) % 3 - 1;
    c[2] = (D == 3) ? i / 9 - 1 : 0;
}

static long ora_cells(const ora_lattice *L) { return (long)L->n[0] * L->n[1] * L->n[2]; }

static long ora_index(const ora_lattice *L, int x, int y, int z)
{
    return (long)x + (long)L->n[0] * ((long)y + (long)L->n[1] * (long)z);
}

static int wrap(int a, int n) { return ((a % n) + n) % n; }

/* --------------------------------------------------- product-form populations */

/*
 * The one-dimensional triplet Psi_{-1}, Psi_0, Psi_{+1} of (u, P, lam)
 * (Eqs. phi0S, phiPlusS, phiMinusS): out[0] = Psi_{-1}, out[1] = Psi_0,
 * out[2] = Psi_{+1}.
 */
void ora_triplet(double u, double P, double lam, double out[3])
{
    out[1] = 1.0 - P / (lam * lam);
    out[2] = 0.5 * (u / lam + P / (lam * lam));
    out[0] = 0.5 * (-u / lam + P / (lam * lam));
}

/*
 * Product form Psi_i(u, P, lam) = prod_alpha Psi_{c_i alpha}(u_alpha, P_alpha, lam_alpha)
 * (Eq. prod).  For D = 2 only alpha = x, y enter.
 */
void ora_product(int D, const double u[3], const double P[3], const double lam[3],
                 double *Psi)
{
    double t[3][3];
    for (int a = 0; a < D; ++a) ora_triplet(u[a], P[a], lam[a], t[a]);
    int Q = ora_Q(D);
    for (int i = 0; i < Q; ++i) {
        int c[3];
        ora_velocity(D, i, c);
        double p = 1.0;
        for (int a = 0; a < D; ++a) p *= t[a][c[a] + 1];
        Psi[i] = p;
    }
}

/* Equilibrium f^eq_i = rho Psi_i(u, P^eq, lam) with P^eq_aa = R T + u_a^2 (Eqs. Peqa, 27eq). */
void ora_equilibrium(int D, double rho, const double u[3], double T, const double lam[3],
                     double *feq)
{
    double P[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) P[a] = T + u[a] * u[a];
    ora_product(D, u, P, lam, feq);
    for (int i = 0; i < ora_Q(D); ++i) feq[i] *= rho;
}

/*
 * The "conventional" equilibrium of Sec. III: the product form (Eq. 27eq)
 * with every term of total degree higher than two in the velocity dropped.
 * Each factor is Psi_c(u_a, T + u_a^2, lam_a) = A_c + B_c u_a + C_c u_a^2, so the
 * product keeps the constant, the linear terms, the squares u_a^2 and the
 * cross products u_a u_b.
 */
void ora_second_order_equilibrium(int D, double rho, const double u[3], double T,
                                  const double lam[3], double *feq)
{
    int Q = ora_Q(D);
    for (int i = 0; i < Q; ++i) {
        int c[3];
        ora_velocity(D, i, c);
        double A[3], B[3], C[3];
        for (int a = 0; a < D; ++a) {
            double l2 = lam[a] * lam[a];
            if (c[a] == 0) { A[a] = 1.0 - T / l2; B[a] = 0.0; C[a] = -1.0 / l2; }
            else { A[a] = 0.5 * T / l2; B[a] = 0.5 * c[a] / lam[a]; C[a] = 0.5 / l2; }
        }
        double s = 0.0, prodA = 1.0;
        for (int a = 0; a < D; ++a) prodA *= A[a];
        s += prodA;
        for (int a = 0; a < D; ++a) {
            double others = 1.0;
            for (int b = 0; b < D; ++b) if (b != a) others *= A[b];
            s += (B[a] * u[a] + C[a] * u[a] * u[a]) * others;
        }
        for (int a = 0; a < D; ++a)
            for (int b = a + 1; b < D; ++b) {
                double others = 1.0;
                for (int g = 0; g < D; ++g) if (g != a && g != b) others *= A[g];
                s += B[a] * B[b] * u[a] * u[b] * others;
            }
        feq[i] = rho * s;
    }
}

/* ------------------------------------------------------------------ moments */

/* rho = sum_i f_i (Eq. density); rho u = sum_i v_i f_i (Eq. momentum) of one cell. */
void ora_cell_moments(int D, const double *fc, const double lam[3], double *rho, double u[3])
{
    int Q = ora_Q(D);
    double r = 0.0, j[3] = {0, 0, 0};
    for (int i = 0; i < Q; ++i) {
        int c[3];
        ora_velocity(D, i, c);
        r += fc[i];
        for (int a = 0; a < D; ++a) j[a] += lam[a] * c[a] * fc[i];
    }
    *rho = r;
    for (int a = 0; a < 3; ++a) u[a] = (a < D) ? j[a] / r : 0.0;
}

/* Diagonal anomaly Q~_aaa = rho u_a (lam_a^2 - 3 R T) - rho u_a^3 (Eq. Deviation). */
double ora_anomaly(double rho, double u, double lam, double T)
{
    return rho * u * (lam * lam - 3.0 * T) - rho * u * u * u;
}

/* Equilibrium-based moment tensors of one cell (for the tests of Eqs. Peq, Qeq):
 * P[a][b] = sum_i v_ia v_ib f_i and Qt[a][b][c] = sum_i v_ia v_ib v_ic f_i. */
void ora_cell_tensors(int D, const double *fc, const double lam[3], double P[9], double Qt[27])
{
    int Q = ora_Q(D);
    memset(P, 0, 9 * sizeof(double));
    memset(Qt, 0, 27 * sizeof(double));
    for (int i = 0; i < Q; ++i) {
        int c[3];
        ora_velocity(D, i, c);
        double v[3];
        for (int a = 0; a < 3; ++a) v[a] = lam[a] * c[a];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                P[3 * a + b] += v[a] * v[b] * fc[i];
                for (int g = 0; g < 3; ++g) Qt[9 * a + 3 * b + g] += v[a] * v[b] * v[g] * fc[i];
            }
    }
}

/* ------------------------------------------------------------ field helpers */

/* f = f^eq(rho0(x), u0(x)) on every node: the initial populations. */
void ora_init(const ora_lattice *L, const double *rho, const double *u, double *f)
{
    int Q = ora_Q(L->D);
    long N = ora_cells(L);
    double feq[27];
    for (long x = 0; x < N; ++x) {
        double uc[3] = {0, 0, 0};
        for (int a = 0; a < L->D; ++a) uc[a] = u[a * N + x];
        ora_equilibrium(L->D, rho[x], uc, L->T, L->lam, feq);
        for (int i = 0; i < Q; ++i) f[i * N + x] = feq[i];
    }
}

/*
 * Density and velocity of every node.  With a body force the reported velocity
 * is the half-step average u + g/2 (the reading used for forced flows).
 */
void ora_macros(const ora_lattice *L, const double *f, double *rho, double *u)
{
    int Q = ora_Q(L->D);
    long N = ora_cells(L);
    double fc[27];
    for (long x = 0; x < N; ++x) {
        for (int i = 0; i < Q; ++i) fc[i] = f[i * N + x];
        double r, uc[3];
        ora_cell_moments(L->D, fc, L->lam, &r, uc);
        rho[x] = r;
        for (int a = 0; a < L->D; ++a) u[a * N + x] = uc[a] + 0.5 * L->g[a];
    }
}

/*
 * Second-order central difference along alpha of a nodal field q (Eq. Paastar1):
 * dq(x) = [q(x + e_alpha) - q(x - e_alpha)] / (2 lam_alpha), node spacing lam_alpha.
 * Periodic wrap; with walls in y, the ghost value beyond a wall is the negated
 * value of the first fluid node (the anomaly is odd in u_y and u_y vanishes on
 * a wall).
 */
void ora_central_difference(const ora_lattice *L, const double *q, int alpha, double *dq)
{
    int nx = L->n[0], ny = L->n[1], nz = L->n[2];
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int p[3] = {x, y, z}, m[3] = {x, y, z};
                p[alpha] += 1;
                m[alpha] -= 1;
                double qp, qm;
                long here = ora_index(L, x, y, z);
                if (alpha == 1 && L->walls_y && p[1] == ny) qp = -q[here];
                else qp = q[ora_index(L, wrap(p[0], nx), wrap(p[1], ny), wrap(p[2], nz))];
                if (alpha == 1 && L->walls_y && m[1] < 0) qm = -q[here];
                else qm = q[ora_index(L, wrap(m[0], nx), wrap(m[1], ny), wrap(m[2], nz))];
                dq[here] = (qp - qm) / (2.0 * L->lam[alpha]);
            }
}

/* ------------------------------------------------------------------- the step */

/*
 * One time step: f holds the post-streaming populations at time t, fn receives
 * those at t + 1.  Returns 0, or -1 if memory could not be obtained.
 */
int ora_step(const ora_lattice *L, const double *f, double *fn)
{
    const int D = L->D, Q = ora_Q(D);
    const long N = ora_cells(L);
    const double w = L->omega;
    double *rho = malloc(N * sizeof(double));
    double *u = malloc(3 * N * sizeof(double));
    double *q = malloc(3 * N * sizeof(double));
    double *d = calloc(3 * N, sizeof(double));
    if (!rho || !u || !q || !d) { free(rho); free(u); free(q); free(d); return -1; }

    /* (1) density and velocity, Eqs. density and momentum. */
    double fc[27];
    for (long x = 0; x < N; ++x) {
        for (int i = 0; i < Q; ++i) fc[i] = f[i * N + x];
        double uc[3];
        ora_cell_moments(D, fc, L->lam, &rho[x], uc);
        for (int a = 0; a < 3; ++a) u[a * N + x] = uc[a];
    }

    if (L->mode == ORA_EXTENDED) {
        /* (2) diagonal anomaly at every node, Eq. Deviation. */
        for (int a = 0; a < D; ++a)
            for (long x = 0; x < N; ++x)
                q[a * N + x] = ora_anomaly(rho[x], u[a * N + x], L->lam[a], L->T);
        /* (3) its central difference along its own axis, Eq. Paastar1. */
        for (int a = 0; a < D; ++a) ora_central_difference(L, q + a * N, a, d + a * N);
    }

    for (long x = 0; x < N; ++x) {
        for (int i = 0; i < Q; ++i) fc[i] = f[i * N + x];
        double r = rho[x], uc[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a) uc[a] = u[a * N + x];

        /* (4)-(5) extended pressure diagonal (Eqs. Paastar1, Paastar) and the
         * equilibrium that the populations relax to. */
        double feq[27];
        if (L->mode == ORA_SECOND_ORDER) {
            ora_second_order_equilibrium(D, r, uc, L->T, L->lam, feq);
        } else {
            double P[3] = {0, 0, 0};
            for (int a = 0; a < D; ++a) {
                P[a] = L->T + uc[a] * uc[a];
                if (L->mode == ORA_EXTENDED) P[a] += (2.0 - w) / (2.0 * r * w) * d[a * N + x];
            }
            ora_product(D, uc, P, L->lam, feq);       /* Eq. prod */
            for (int i = 0; i < Q; ++i) feq[i] *= r;  /* Eq. 27eqext */
        }

        /* (6) BGK relaxation, Eq. LBGK. */
        double fp[27];
        for (int i = 0; i < Q; ++i) fp[i] = fc[i] + w * (feq[i] - fc[i]);

        /* Body force, exact-difference reading: f' += f^eq(rho, u + g) - f^eq(rho, u). */
        if (L->g[0] != 0.0 || L->g[1] != 0.0 || L->g[2] != 0.0) {
            double ug[3] = {0, 0, 0}, e0[27], e1[27];
            for (int a = 0; a < D; ++a) ug[a] = uc[a] + L->g[a];
            ora_equilibrium(D, r, uc, L->T, L->lam, e0);
            ora_equilibrium(D, r, ug, L->T, L->lam, e1);
            for (int i = 0; i < Q; ++i) fp[i] += e1[i] - e0[i];
        }

        /* (7) streaming: population i moves one node along c_i, Eq. LBGK. */
        int x0 = (int)(x % L->n[0]);
        int y0 = (int)((x / L->n[0]) % L->n[1]);
        int z0 = (int)(x / ((long)L->n[0] * L->n[1]));
        for (int i = 0; i < Q; ++i) {
            int c[3];
            ora_velocity(D, i, c);
            int yt = y0 + c[1];
            if (L->walls_y && (yt < 0 || yt >= L->n[1])) {
                /* half-way bounce-back: the population returns reversed to its own node */
                fn[(Q - 1 - i) * N + x] = fp[i];
                continue;
            }
            long t = ora_index(L, wrap(x0 + c[0], L->n[0]), wrap(yt, L->n[1]),
                               wrap(z0 + c[2], L->n[2]));
            fn[i * N + t] = fp[i];
        }
    }
    free(rho); free(u); free(q); free(d);
    return 0;
}

/* Run `steps` steps in place on f (uses one scratch array).  Returns 0 or -1. */
int ora_run(const ora_lattice *L, double *f, int steps)
{
    long M = (long)ora_Q(L->D) * ora_cells(L);
    double *g = malloc(M * sizeof(double));
    if (!g) return -1;
    for (int s = 0; s < steps; ++s) {
        if (ora_step(L, f, g)) { free(g); return -1; }
        memcpy(f, g, M * sizeof(double));
    }
    free(g);
    return 0;
}
