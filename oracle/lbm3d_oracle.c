/*
 * lbm3d_oracle.c -- FP64 CPU oracle of the D3Q19 form of the method.
 *
 * TEST INFRASTRUCTURE ONLY, like lbm_oracle.c: plain loops restating what the
 * method computes, loaded only by the tests, the package smoke check and the
 * benchmark's CPU baseline; it shares nothing with the CUDA path.
 *
 * Section 2 uses D3Q19 for three-dimensional problems with the algorithms
 * unchanged, without listing its velocities and weights. They are taken here as
 * the rest velocity, the 6 face neighbours and the 12 edge neighbours of the
 * cubic lattice, with weights 1/3, 1/18 and 1/36 and c_s^2 = 1/3 (the unique
 * weights for these shells with sum w = 1, sum w e e = c_s^2 I and an isotropic
 * fourth moment). The update is the one of Section 2.2 with vectors of
 * three components:
 *     rho = sum_a f_a, j = sum_a e_a f_a
 *     u    = (j + eps rho G / 2) / (rho (1 + eps nu / (2 kappa)))          Eq. 6
 *     u_eq = 2 tau u + (1 - 2 tau) j / rho                                  Eq. 16
 *     f_eq = w rho (1 + e.u_eq / c_s^2)                                     Eq. 2
 *     f(x + e, t + 1) = f + (f_eq - f) / tau                                Eq. 13
 * Periodic in x, y and z; rest initial state (f = w rho0, rho0 = 1).
 * Layout: f[((z * ny + y) * nx + x) * 19 + a].
 *
 * With a tensor K* per cell instead of kappa (the coarse run, Eq. 18 in three
 * dimensions) Eq. 6 becomes the 3x3 solve (I + eps nu / 2 K*^-1) rho u = j + eps rho G / 2.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define Q3 19

typedef struct {
    int nx, ny, nz;
    double tau, nu, eps;
    double gx, gy, gz;        /* constant body force */
    const double *kappa;      /* [nz][ny][nx] permeability (may be +inf) */
    const double *ktensor;    /* [nz][ny][nx][9] K*_ij row-major, used when kappa == NULL */
} orc3_problem;

static int E3[Q3][3];
static double W3[Q3];
static int ready3 = 0;

/* The 19 vectors of {-1, 0, 1}^3 with at most two non-zero components, weighted by shell. */
static void lattice3_init(void)
{
    if (ready3) return;
    int a = 0;
    for (int shell = 0; shell <= 2; ++shell)
        for (int z = -1; z <= 1; ++z)
            for (int y = -1; y <= 1; ++y)
                for (int x = -1; x <= 1; ++x)
                    if (x * x + y * y + z * z == shell) {
                        E3[a][0] = x; E3[a][1] = y; E3[a][2] = z;
                        W3[a] = shell == 0 ? 1.0 / 3.0 : (shell == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
                        ++a;
                    }
    ready3 = 1;
}

void orc3_lattice(int *e_out /* [19][3] */, double *w_out /* [19] */)
{
    lattice3_init();
    for (int a = 0; a < Q3; ++a) {
        for (int k = 0; k < 3; ++k) e_out[3 * a + k] = E3[a][k];
        w_out[a] = W3[a];
    }
}

/* Inverse of the 3x3 matrix m (row-major) by cofactors: inv = adj(m) / det(m). */
static void inv3(const double m[9], double inv[9])
{
    const double c00 = m[4] * m[8] - m[5] * m[7], c01 = m[5] * m[6] - m[3] * m[8], c02 = m[3] * m[7] - m[4] * m[6];
    const double c10 = m[2] * m[7] - m[1] * m[8], c11 = m[0] * m[8] - m[2] * m[6], c12 = m[1] * m[6] - m[0] * m[7];
    const double c20 = m[1] * m[5] - m[2] * m[4], c21 = m[2] * m[3] - m[0] * m[5], c22 = m[0] * m[4] - m[1] * m[3];
    const double det = m[0] * c00 + m[1] * c01 + m[2] * c02;
    /* adj(m) is the transpose of the cofactor matrix */
    inv[0] = c00 / det; inv[1] = c10 / det; inv[2] = c20 / det;
    inv[3] = c01 / det; inv[4] = c11 / det; inv[5] = c21 / det;
    inv[6] = c02 / det; inv[7] = c12 / det; inv[8] = c22 / det;
}

/* Eq. 6 (or Eq. 18) for one cell: rho, j and the flow velocity u (Eq. 15). */
static void cell3(const orc3_problem *p, long c, const double *fc, double *rho_o, double j[3], double u[3])
{
    double rho = 0.0;
    j[0] = j[1] = j[2] = 0.0;
    for (int a = 0; a < Q3; ++a) {
        rho += fc[a];
        for (int k = 0; k < 3; ++k) j[k] += E3[a][k] * fc[a];
    }
    const double G[3] = {p->gx, p->gy, p->gz};
    *rho_o = rho;
    if (!p->kappa) {
        double r[3];
        for (int k = 0; k < 3; ++k) r[k] = j[k] + 0.5 * p->eps * rho * G[k];
        if (p->eps == 0.0 || p->nu == 0.0) {
            for (int k = 0; k < 3; ++k) u[k] = r[k] / rho;
            return;
        }
        /* Eq. 18: (I + h K*^-1) rho u = r, h = eps nu / 2 */
        double Ki[9], B[9], Bi[9];
        inv3(p->ktensor + 9 * c, Ki);
        const double h = 0.5 * p->eps * p->nu;
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) B[3 * i + k] = (i == k ? 1.0 : 0.0) + h * Ki[3 * i + k];
        inv3(B, Bi);
        for (int i = 0; i < 3; ++i) u[i] = (Bi[3 * i] * r[0] + Bi[3 * i + 1] * r[1] + Bi[3 * i + 2] * r[2]) / rho;
        return;
    }
    double drag = 0.0;                           /* eps nu / (2 kappa) */
    if (p->eps != 0.0 && p->nu != 0.0) {
        const double k = p->kappa[c];
        drag = isinf(k) ? 0.0 : (k == 0.0 ? INFINITY : p->eps * p->nu / (2.0 * k));
    }
    for (int k = 0; k < 3; ++k) {
        const double r = j[k] + 0.5 * p->eps * rho * G[k];
        u[k] = isinf(drag) ? 0.0 : r / (rho * (1.0 + drag));
    }
}

void orc3_init_rest(const orc3_problem *p, double *f)
{
    lattice3_init();
    const long n = (long)p->nx * p->ny * p->nz;
    for (long c = 0; c < n; ++c)
        for (int a = 0; a < Q3; ++a) f[c * Q3 + a] = W3[a];
}

/* One step f -> out: collide every cell (Eqs. 6, 16, 2, 13), then stream along e_a
 * with periodic wrap. The stored state is the streamed, pre-collision one, as in
 * the two-dimensional oracle. */
void orc3_step(const orc3_problem *p, const double *f, double *out)
{
    lattice3_init();
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const double tau = p->tau;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const long c = ((long)z * ny + y) * nx + x;
                const double *fc = f + c * Q3;
                double rho, j[3], u[3];
                cell3(p, c, fc, &rho, j, u);
                double ueq[3];
                for (int k = 0; k < 3; ++k) ueq[k] = 2.0 * tau * u[k] + (1.0 - 2.0 * tau) * j[k] / rho;
                for (int a = 0; a < Q3; ++a) {
                    const double eu = E3[a][0] * ueq[0] + E3[a][1] * ueq[1] + E3[a][2] * ueq[2];
                    const double feq = W3[a] * rho * (1.0 + 3.0 * eu);
                    const int xd = (x + E3[a][0] + nx) % nx, yd = (y + E3[a][1] + ny) % ny,
                              zd = (z + E3[a][2] + nz) % nz;
                    out[(((long)zd * ny + yd) * nx + xd) * Q3 + a] = fc[a] + (feq - fc[a]) / tau;
                }
            }
}

void orc3_run(const orc3_problem *p, double *f, long steps)
{
    const long n = (long)p->nx * p->ny * p->nz;
    double *g = (double *)malloc(sizeof(double) * n * Q3);
    for (long s = 0; s < steps; ++s) {
        orc3_step(p, f, g);
        memcpy(f, g, sizeof(double) * n * Q3);
    }
    free(g);
}

/* Density and flow velocity (Eq. 15) of every cell; any output may be NULL. */
void orc3_fields(const orc3_problem *p, const double *f, double *rho, double *u, double *v, double *w)
{
    lattice3_init();
    const long n = (long)p->nx * p->ny * p->nz;
    for (long c = 0; c < n; ++c) {
        double r, j[3], uc[3];
        cell3(p, c, f + c * Q3, &r, j, uc);
        if (rho) rho[c] = r;
        if (u) u[c] = uc[0];
        if (v) v[c] = uc[1];
        if (w) w[c] = uc[2];
    }
}

/* Volume average of the flow velocity (arithmetic mean over cells). */
void orc3_mean_velocity(const orc3_problem *p, const double *f, double out[3])
{
    lattice3_init();
    const long n = (long)p->nx * p->ny * p->nz;
    double s[3] = {0.0, 0.0, 0.0};
    for (long c = 0; c < n; ++c) {
        double r, j[3], uc[3];
        cell3(p, c, f + c * Q3, &r, j, uc);
        for (int k = 0; k < 3; ++k) s[k] += uc[k];
    }
    for (int k = 0; k < 3; ++k) out[k] = s[k] / n;
}

/* Mean flow velocity over the w^3 window at (x0, y0, z0) (the inner leaf of an oversampled cube). */
static void orc3_mean_velocity_window(const orc3_problem *p, const double *f, int x0, int y0, int z0, int w,
                                      double out[3])
{
    double s[3] = {0.0, 0.0, 0.0};
    for (int z = z0; z < z0 + w; ++z)
        for (int y = y0; y < y0 + w; ++y)
            for (int x = x0; x < x0 + w; ++x) {
                const long c = ((long)z * p->ny + y) * p->nx + x;
                double r, j[3], uc[3];
                cell3(p, c, f + c * Q3, &r, j, uc);
                for (int k = 0; k < 3; ++k) s[k] += uc[k];
            }
    for (int k = 0; k < 3; ++k) out[k] = s[k] / ((double)w * w * w);
}

/*
 * The oversampled form (the treatment the Conclusions name for high-contrast
 * media): kappa_ext is the leaf grown by `margin` cells on every side (se = s +
 * 2 margin, [z][y][x]); the periodic problem runs on the grown cube and the stop
 * test and Eq. 17 use the mean velocity over the inner s^3 leaf only. Otherwise
 * as orc3_local_keff below. Returns the number of drives that converged, or -1 if
 * the leaf would be empty.
 */
int orc3_local_keff_os(int se, int margin, const double *kappa_ext, double tau, double nu, double eps,
                       double gconst, double tol, long max_steps, int check_every, double keff[9], long steps[3])
{
    lattice3_init();
    const int s = se - 2 * margin;
    if (margin < 0 || s < 1) return -1;
    orc3_problem p;
    memset(&p, 0, sizeof p);
    p.nx = se; p.ny = se; p.nz = se; p.tau = tau; p.nu = nu; p.eps = eps; p.kappa = kappa_ext;
    const long n = (long)se * se * se;
    double *f = (double *)malloc(sizeof(double) * n * Q3);
    double *g = (double *)malloc(sizeof(double) * n * Q3);
    int nconv = 0;
    for (int d = 0; d < 3; ++d) {
        p.gx = d == 0 ? gconst : 0.0;
        p.gy = d == 1 ? gconst : 0.0;
        p.gz = d == 2 ? gconst : 0.0;
        orc3_init_rest(&p, f);
        double prev = 0.0, m[3];
        long st = 0;
        int conv = 0;
        while (st < max_steps) {
            orc3_step(&p, f, g);
            memcpy(f, g, sizeof(double) * n * Q3);
            ++st;
            if (check_every > 0 && st % check_every == 0) {
                orc3_mean_velocity_window(&p, f, margin, margin, margin, s, m);
                if (tol > 0.0 && st > check_every && fabs(m[d] - prev) <= tol * check_every * fabs(m[d])) {
                    conv = 1;
                    break;
                }
                prev = m[d];
            }
        }
        orc3_mean_velocity_window(&p, f, margin, margin, margin, s, m);
        for (int i = 0; i < 3; ++i) keff[3 * i + d] = nu / gconst * m[i];
        steps[d] = st;
        nconv += conv;
    }
    free(f);
    free(g);
    return nconv;
}

/*
 * One three-dimensional local problem (Section 3 with the D3Q19 lattice): the
 * s x s x s permeability cube `kappa_cube` ([z][y][x]) with periodic closure,
 * driven along x, y and z in turn by a body force of magnitude gconst, each from
 * rest until the driven component of the volume-averaged velocity settles:
 * every check_every steps n, |ubar_d(n) - ubar_d(n - k)| <= tol k |ubar_d(n)|
 * (tol <= 0 runs exactly max_steps). Eq. 17 in three dimensions: column d of K*
 * is nu / gconst times the mean velocity of drive d, so K*[i][d] = nu ubar_d,i / G.
 * keff [3][3] row-major (K*_ij, i the velocity component, j the drive);
 * steps[d] per drive; returns the number of drives that converged.
 */
int orc3_local_keff(int s, const double *kappa_cube, double tau, double nu, double eps, double gconst,
                    double tol, long max_steps, int check_every, double keff[9], long steps[3])
{
    lattice3_init();
    orc3_problem p;
    memset(&p, 0, sizeof p);
    p.nx = s; p.ny = s; p.nz = s; p.tau = tau; p.nu = nu; p.eps = eps; p.kappa = kappa_cube;
    const long n = (long)s * s * s;
    double *f = (double *)malloc(sizeof(double) * n * Q3);
    double *g = (double *)malloc(sizeof(double) * n * Q3);
    int nconv = 0;
    for (int d = 0; d < 3; ++d) {
        p.gx = d == 0 ? gconst : 0.0;
        p.gy = d == 1 ? gconst : 0.0;
        p.gz = d == 2 ? gconst : 0.0;
        orc3_init_rest(&p, f);
        double prev = 0.0, m[3];
        long st = 0;
        int conv = 0;
        while (st < max_steps) {
            orc3_step(&p, f, g);
            memcpy(f, g, sizeof(double) * n * Q3);
            ++st;
            if (check_every > 0 && st % check_every == 0) {
                orc3_mean_velocity(&p, f, m);
                if (tol > 0.0 && st > check_every && fabs(m[d] - prev) <= tol * check_every * fabs(m[d])) {
                    conv = 1;
                    break;
                }
                prev = m[d];
            }
        }
        orc3_mean_velocity(&p, f, m);
        for (int i = 0; i < 3; ++i) keff[3 * i + d] = nu / gconst * m[i];
        steps[d] = st;
        nconv += conv;
    }
    free(f);
    free(g);
    return nconv;
}
