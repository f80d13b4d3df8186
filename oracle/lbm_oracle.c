/*
 * lbm_oracle.c -- FP64 CPU oracle of the upscaled lattice Boltzmann method.
 *
 * TEST INFRASTRUCTURE ONLY. This file restates, slowly and in plain loops, what
 * the paper's method computes, so that the CUDA library can be checked against
 * it. Only the tests, the package smoke check and the benchmark's CPU baseline
 * load it. It shares no code, header or constant table with the CUDA path, and
 * the CUDA path never calls it.
 *
 * What it follows (Li & Brown, "Upscaled Lattice Boltzmann Method for
 * Simulations of Flows in Heterogeneous Porous Media"):
 *   - D2Q9 lattice: e_alpha and w_alpha as defined in Section 2 (theta formulas).
 *   - Simplified Shan-Chen evolution, Section 2.2:
 *       rho = sum_a f_a, j = sum_a e_a f_a
 *       u    = (j + dt/2 eps rho G) / (rho (1 + eps dt nu / (2 kappa)))    Eq. 6
 *              (valid for the Shan-Chen model, Section 2.2 below Eq. 15)
 *       u_eq = 2 tau u + (1 - 2 tau) j / rho                                 Eq. 16
 *       f_eq = w rho (1 + e.u_eq / c_s^2)                                    Eq. 2
 *       f(x + e dt, t + dt) = f + (f_eq - f) / tau                           Eq. 13
 *   - Tensor permeability (Eq. 18): f_m = -eps nu K*^-1 u + eps G, so that
 *       rho u = (I + dt/2 eps nu K*^-1)^-1 (j + dt/2 eps rho G)            (Eq. 15 + Eq. 18)
 *   - Local problems (Section 3): periodic subdomain, G1 = (G, 0) and
 *     G2 = (0, G), volume-averaged velocity, and Eq. 17 for K*.
 *
 * Lattice units throughout: dx = dt = 1, c = 1, c_s^2 = 1/3, rho0 = 1.
 * Layout: f[(y * nx + x) * 9 + a] (array of structures).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - initial state is rest, f = w rho0;
 *   - walls (when requested) are half-way bounce-back links at y = -1/2 and
 *     y = ny - 1/2; the paper itself uses periodic boundaries;
 *   - the averaged velocity is the flow velocity of Eq. 15 (half-force included),
 *     arithmetic mean over the cells;
 *   - nu = 0 or eps = 0 means no drag at all (then kappa is not used).
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

#define Q 9

typedef struct {
    int nx, ny;
    double tau, nu, eps;
    int walls;               /* 0: periodic in x and y; 1: bounce-back walls in y */
    double gx, gy;           /* constant body force, used when gfield == NULL */
    const double *kappa;     /* [ny][nx] scalar permeability (may be +inf), or NULL */
    const double *ktensor;   /* [ny][nx][4] (xx, xy, yx, yy), used when kappa == NULL */
    const double *gfield;    /* [2][ny][nx] body force, or NULL */
    int force_model;         /* 0: simplified Shan-Chen scheme (Section 2.2); 1: Guo scheme (Section 2.1) */
    const double *fixed;     /* [ny][nx][4] (flag, drho, u, v), or NULL: a cell with a non-zero flag
                                emits, every step, instead of its collision result, what a cell at
                                rest in the state (rho = 1 + drho, u, v) emits at tau = 1: the
                                equilibrium of Eq. 2 at its post-collision momentum rho u + rho f_m / 2
                                (f_m of Eq. 5 at u; zero where kappa = 0) (local-global ring) */
} orc_problem;

/* D2Q9 velocities and weights, built from the angle definitions of Section 2. */
static int E[Q][2];
static double W[Q];
static int OPP[Q];
static int lattice_ready = 0;

static void lattice_init(void)
{
    if (lattice_ready) return;
    const double pi = 3.14159265358979323846;
    E[0][0] = 0; E[0][1] = 0; W[0] = 4.0 / 9.0;
    for (int a = 1; a <= 4; ++a) {
        double th = (a - 1) * pi / 2.0;
        E[a][0] = (int)lround(cos(th));
        E[a][1] = (int)lround(sin(th));
        W[a] = 1.0 / 9.0;
    }
    for (int a = 5; a <= 8; ++a) {
        double th = (a - 5) * pi / 2.0 + pi / 4.0;
        E[a][0] = (int)lround(sqrt(2.0) * cos(th));
        E[a][1] = (int)lround(sqrt(2.0) * sin(th));
        W[a] = 1.0 / 36.0;
    }
    for (int a = 0; a < Q; ++a)
        for (int b = 0; b < Q; ++b)
            if (E[b][0] == -E[a][0] && E[b][1] == -E[a][1]) OPP[a] = b;
    lattice_ready = 1;
}

void orc_lattice(int *e_out /* [9][2] */, double *w_out /* [9] */)
{
    lattice_init();
    for (int a = 0; a < Q; ++a) {
        e_out[2 * a] = E[a][0];
        e_out[2 * a + 1] = E[a][1];
        w_out[a] = W[a];
    }
}

static void force_at(const orc_problem *p, long c, double *Gx, double *Gy)
{
    if (p->gfield) {
        long n = (long)p->nx * p->ny;
        *Gx = p->gfield[c];
        *Gy = p->gfield[n + c];
    } else {
        *Gx = p->gx;
        *Gy = p->gy;
    }
}

/*
 * Flow velocity of one cell from its (pre-collision) distributions:
 * Eq. 15 with f_m from Eq. 5 (scalar kappa, solved explicitly as Eq. 6) or
 * from Eq. 18 (tensor K*, a 2x2 solve). Also returns rho and j.
 */
static void cell_velocity(const orc_problem *p, long c, const double *fc,
                          double *rho_o, double *jx_o, double *jy_o,
                          double *ux_o, double *uy_o)
{
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int a = 0; a < Q; ++a) {
        rho += fc[a];
        jx += E[a][0] * fc[a];
        jy += E[a][1] * fc[a];
    }
    double Gx, Gy;
    force_at(p, c, &Gx, &Gy);
    const double dt = 1.0;
    double ux, uy;
    if (p->eps * p->nu == 0.0) {
        /* no drag: u = (j + dt/2 eps rho G) / rho */
        ux = (jx + 0.5 * dt * p->eps * rho * Gx) / rho;
        uy = (jy + 0.5 * dt * p->eps * rho * Gy) / rho;
    } else if (p->kappa) {
        double kap = p->kappa[c];
        double denom = rho * (1.0 + p->eps * dt * p->nu / (2.0 * kap));   /* Eq. 6 */
        ux = (jx + 0.5 * dt * p->eps * rho * Gx) / denom;
        uy = (jy + 0.5 * dt * p->eps * rho * Gy) / denom;
    } else {
        /* Eq. 18 in Eq. 15: (I + dt/2 eps nu K*^-1) rho u = j + dt/2 eps rho G */
        const double *k = p->ktensor + 4 * c;
        double det = k[0] * k[3] - k[1] * k[2];
        double ixx = k[3] / det, ixy = -k[1] / det, iyx = -k[2] / det, iyy = k[0] / det;
        double h = 0.5 * dt * p->eps * p->nu;
        double bxx = 1.0 + h * ixx, bxy = h * ixy, byx = h * iyx, byy = 1.0 + h * iyy;
        double rx = jx + 0.5 * dt * p->eps * rho * Gx;
        double ry = jy + 0.5 * dt * p->eps * rho * Gy;
        double bdet = bxx * byy - bxy * byx;
        double rux = (byy * rx - bxy * ry) / bdet;
        double ruy = (-byx * rx + bxx * ry) / bdet;
        ux = rux / rho;
        uy = ruy / rho;
    }
    *rho_o = rho; *jx_o = jx; *jy_o = jy;
    *ux_o = ux; *uy_o = uy;
}

/*
 * Force per unit mass f_m of Eq. 5 (scalar kappa) or Eq. 18 (tensor K*) at the
 * flow velocity u of Eq. 6. A blocked cell (kappa = 0) has u = 0 and its f_m
 * follows from Eq. 3 with u_eq = u = 0: f_m = -2 j / rho (reading; Eq. 5 is 0/0 there).
 */
static void force_per_mass(const orc_problem *p, long c, double rho, double jx, double jy, double ux, double uy,
                           double *fmx, double *fmy)
{
    double Gx, Gy;
    force_at(p, c, &Gx, &Gy);
    if (p->eps * p->nu == 0.0) {
        *fmx = p->eps * Gx;
        *fmy = p->eps * Gy;
    } else if (p->kappa) {
        double kap = p->kappa[c];
        if (kap == 0.0) {
            *fmx = -2.0 * jx / rho;
            *fmy = -2.0 * jy / rho;
        } else {
            *fmx = -p->eps * p->nu / kap * ux + p->eps * Gx;                 /* Eq. 5 */
            *fmy = -p->eps * p->nu / kap * uy + p->eps * Gy;
        }
    } else {
        const double *k = p->ktensor + 4 * c;                                /* Eq. 18 */
        double det = k[0] * k[3] - k[1] * k[2];
        double ixx = k[3] / det, ixy = -k[1] / det, iyx = -k[2] / det, iyy = k[0] / det;
        *fmx = -p->eps * p->nu * (ixx * ux + ixy * uy) + p->eps * Gx;
        *fmy = -p->eps * p->nu * (iyx * ux + iyy * uy) + p->eps * Gy;
    }
}

void orc_init_rest(const orc_problem *p, double *f)
{
    lattice_init();
    long n = (long)p->nx * p->ny;
    for (long c = 0; c < n; ++c)
        for (int a = 0; a < Q; ++a) f[c * Q + a] = W[a] * 1.0;
}

/* rho, u, v of the state f (Eq. 15); any output pointer may be NULL. */
void orc_velocity(const orc_problem *p, const double *f, double *rho, double *u, double *v)
{
    lattice_init();
    long n = (long)p->nx * p->ny;
    for (long c = 0; c < n; ++c) {
        double r, jx, jy, ux, uy;
        cell_velocity(p, c, f + c * Q, &r, &jx, &jy, &ux, &uy);
        if (rho) rho[c] = r;
        if (u) u[c] = ux;
        if (v) v[c] = uy;
    }
}

/* One time step f -> fnew: collide, then stream along e_a. Simplified Shan-Chen
 * scheme: Eqs. 6, 16, 2, 13. Guo scheme (force_model = 1): Eq. 6 for u, u_eq = u,
 * f_m by Eq. 5, the forcing term F_a of Eq. 4 and the update of Eq. 1. */
void orc_step(const orc_problem *p, const double *f, double *fnew)
{
    lattice_init();
    const int nx = p->nx, ny = p->ny;
    const double tau = p->tau, cs2 = 1.0 / 3.0;
#pragma omp parallel for schedule(static) if ((long)nx * ny >= 16384)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            long c = (long)y * nx + x;
            const double *fc = f + c * Q;
            double rho, jx, jy, ux, uy;
            cell_velocity(p, c, fc, &rho, &jx, &jy, &ux, &uy);
            double uex, uey, fmx = 0.0, fmy = 0.0;
            if (p->force_model == 1) {
                uex = ux;                                                    /* Guo: u_eq = u */
                uey = uy;
                force_per_mass(p, c, rho, jx, jy, ux, uy, &fmx, &fmy);
            } else {
                uex = 2.0 * tau * ux + (1.0 - 2.0 * tau) * jx / rho;        /* Eq. 16 */
                uey = 2.0 * tau * uy + (1.0 - 2.0 * tau) * jy / rho;
            }
            const double *fx = p->fixed && p->fixed[c * 4] != 0.0 ? p->fixed + c * 4 : NULL;
            for (int a = 0; a < Q; ++a) {
                double eu = E[a][0] * uex + E[a][1] * uey;
                double feq = W[a] * rho * (1.0 + eu / cs2);                 /* Eq. 2 */
                double fpost = fc[a] + (feq - fc[a]) / tau;                 /* Eq. 13 */
                if (p->force_model == 1) {
                    double ef = E[a][0] * fmx + E[a][1] * fmy;
                    fpost += W[a] * rho * (1.0 - 1.0 / (2.0 * tau)) * ef / cs2;   /* dt F_a, Eqs. 1, 4 */
                }
                if (fx) {
                    const double rb = 1.0 + fx[1];
                    double Gx, Gy, jpx = 0.0, jpy = 0.0;
                    force_at(p, c, &Gx, &Gy);
                    const double kap = p->kappa ? p->kappa[c] : INFINITY;
                    if (kap != 0.0) {
                        const double drag = (p->eps * p->nu == 0.0 || isinf(kap)) ? 0.0 : p->eps * p->nu / kap;
                        jpx = rb * fx[2] + 0.5 * rb * (p->eps * Gx - drag * fx[2]);
                        jpy = rb * fx[3] + 0.5 * rb * (p->eps * Gy - drag * fx[3]);
                    }
                    fpost = W[a] * (rb + (E[a][0] * jpx + E[a][1] * jpy) / cs2);
                }
                int xd = x + E[a][0];
                int yd = y + E[a][1];
                xd = (xd + nx) % nx;
                if (p->walls && (yd < 0 || yd >= ny)) {
                    /* half-way bounce-back: the particle returns to its own cell reversed */
                    fnew[c * Q + OPP[a]] = fpost;
                } else {
                    yd = (yd + ny) % ny;
                    fnew[((long)yd * nx + xd) * Q + a] = fpost;
                }
            }
        }
    }
}

static double max_abs_diff_uv(long n, const double *u0, const double *v0,
                              const double *u1, const double *v1, double *umax)
{
    double dm = 0.0, m = 0.0;
    for (long c = 0; c < n; ++c) {
        double du = fabs(u1[c] - u0[c]), dv = fabs(v1[c] - v0[c]);
        if (du > dm) dm = du;
        if (dv > dm) dm = dv;
        if (fabs(u1[c]) > m) m = fabs(u1[c]);
        if (fabs(v1[c]) > m) m = fabs(v1[c]);
    }
    *umax = m;
    return dm;
}

/*
 * Time stepping from the state in f (updated in place) for at most max_steps.
 * Every check_every steps (when > 0) the change of the flow velocity between
 * the last two steps is measured: resid = max|u^n - u^(n-1)| / max|u^n|
 * (max over cells and both components). Stops when tol > 0 and resid <= tol.
 * Returns the number of steps taken; *resid_out gets the last residual (or -1).
 * work: a second state of nx * ny * 9 doubles the steps alternate with (NULL:
 * allocated and freed here); after an odd number of steps the result is copied
 * back into f once.
 */
long orc_run(const orc_problem *p, double *f, double *work, long max_steps, double tol, int check_every,
             double *resid_out, int *converged)
{
    lattice_init();
    long n = (long)p->nx * p->ny;
    double *own = work ? NULL : (double *)malloc(sizeof(double) * n * Q);
    double *cur = f, *nxt = work ? work : own;
    double *u0 = NULL, *v0 = NULL, *u1 = NULL, *v1 = NULL;
    if (check_every > 0) {
        u0 = (double *)malloc(sizeof(double) * n);
        v0 = (double *)malloc(sizeof(double) * n);
        u1 = (double *)malloc(sizeof(double) * n);
        v1 = (double *)malloc(sizeof(double) * n);
    }
    double resid = -1.0;
    int conv = 0;
    long s = 0;
    /* u0/v0 hold u(f^(s-1)) whenever s is a check step (s % check_every == 0) */
    if (check_every == 1) orc_velocity(p, cur, NULL, u0, v0);
    while (s < max_steps) {
        orc_step(p, cur, nxt);
        double *t = cur;
        cur = nxt;
        nxt = t;
        ++s;
        if (check_every > 0) {
            if (s % check_every == 0) {
                double um;
                orc_velocity(p, cur, NULL, u1, v1);
                double d = max_abs_diff_uv(n, u0, v0, u1, v1, &um);
                resid = um > 0.0 ? d / um : d;
                if (tol > 0.0 && resid <= tol) { conv = 1; break; }
            }
            if ((s + 1) % check_every == 0) orc_velocity(p, cur, NULL, u0, v0);
        }
    }
    if (cur != f) memcpy(f, cur, sizeof(double) * n * Q);
    free(own); free(u0); free(v0); free(u1); free(v1);
    if (resid_out) *resid_out = resid;
    if (converged) *converged = conv;
    return s;
}

/* Thread count of the OpenMP loops (the timed CPU baseline runs at 1 and at all cores). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

/* Volume average (arithmetic mean over cells) of the flow velocity, Section 3. */
void orc_mean_velocity(const orc_problem *p, const double *f, double out[2])
{
    lattice_init();
    long n = (long)p->nx * p->ny;
    double su = 0.0, sv = 0.0;
    for (long c = 0; c < n; ++c) {
        double r, jx, jy, ux, uy;
        cell_velocity(p, c, f + c * Q, &r, &jx, &jy, &ux, &uy);
        su += ux;
        sv += uy;
    }
    out[0] = su / n;
    out[1] = sv / n;
}

/*
 * Steps f (in place) until the volume-averaged flow velocity settles: every
 * check_every steps, |ubar_d(n) - ubar_d(n - k)| <= tol * k * |ubar_d(n)| on
 * component d (0: x, 1: y). tol <= 0 runs exactly max_steps. Returns the
 * steps taken; *converged tells whether the test passed; ubar gets the final mean.
 */
long orc_run_mean_steady(const orc_problem *p, double *f, int d, double tol, long max_steps,
                         int check_every, double ubar[2], int *converged)
{
    lattice_init();
    long n = (long)p->nx * p->ny;
    double *g = (double *)malloc(sizeof(double) * n * Q);
    double prev = 0.0, m[2] = {0.0, 0.0};
    long st = 0;
    int conv = 0;
    while (st < max_steps) {
        orc_step(p, f, g);
        memcpy(f, g, sizeof(double) * n * Q);
        ++st;
        if (check_every > 0 && st % check_every == 0) {
            orc_mean_velocity(p, f, m);
            double cur = m[d];
            if (tol > 0.0 && st > check_every &&
                fabs(cur - prev) <= tol * check_every * fabs(cur)) {
                conv = 1;
                break;
            }
            prev = cur;
        }
    }
    orc_mean_velocity(p, f, ubar);
    free(g);
    if (converged) *converged = conv;
    return st;
}

/*
 * One local problem (Section 3): the s x s permeability patch `kappa_leaf`
 * (row-major) with periodic closure, driven by G1 = (gconst, 0) and then
 * G2 = (0, gconst), each from rest until the volume-averaged velocity settles
 * (orc_run_mean_steady on the driven component).
 * Eq. 17 then gives K* = nu / gconst * [[ubar1_x, ubar2_x], [ubar1_y, ubar2_y]].
 * keff = (xx, xy, yx, yy); ubar = (ubar1_x, ubar1_y, ubar2_x, ubar2_y);
 * steps[d] = steps taken per drive; returns the number of drives that converged.
 */
int orc_local_keff(int s, const double *kappa_leaf, double tau, double nu, double eps,
                   double gconst, double tol, long max_steps, int check_every,
                   double keff[4], double ubar[4], long steps[2])
{
    lattice_init();
    orc_problem p;
    memset(&p, 0, sizeof p);
    p.nx = s; p.ny = s; p.tau = tau; p.nu = nu; p.eps = eps;
    p.walls = 0; p.kappa = kappa_leaf;
    long n = (long)s * s;
    double *f = (double *)malloc(sizeof(double) * n * Q);
    int nconv = 0;
    for (int d = 0; d < 2; ++d) {
        p.gx = d == 0 ? gconst : 0.0;
        p.gy = d == 0 ? 0.0 : gconst;
        orc_init_rest(&p, f);
        int conv = 0;
        steps[d] = orc_run_mean_steady(&p, f, d, tol, max_steps, check_every, ubar + 2 * d, &conv);
        nconv += conv;
    }
    /* Eq. 17: columns are the two drives, rows the velocity components */
    keff[0] = nu / gconst * ubar[0];   /* K*_xx = nu/G ubar1 . (1,0) */
    keff[1] = nu / gconst * ubar[2];   /* K*_xy = nu/G ubar2 . (1,0) */
    keff[2] = nu / gconst * ubar[1];   /* K*_yx = nu/G ubar1 . (0,1) */
    keff[3] = nu / gconst * ubar[3];   /* K*_yy = nu/G ubar2 . (0,1) */
    free(f);
    return nconv;
}

/*
 * Oversampled local problem (the treatment named in the Conclusions for high-contrast,
 * channelised media): the leaf's s x s block is embedded in an se x se patch
 * (se = s + 2 margin, the block in the middle) which is solved with periodic closure
 * exactly as in orc_local_keff; the stop test and Eq. 17 use the mean velocity over
 * the inner s x s window only. margin = 0 is orc_local_keff.
 */
static void mean_velocity_window(const orc_problem *p, const double *f, int x0, int y0, int w, double out[2])
{
    double su = 0.0, sv = 0.0;
    for (int y = y0; y < y0 + w; ++y)
        for (int x = x0; x < x0 + w; ++x) {
            long c = (long)y * p->nx + x;
            double r, jx, jy, ux, uy;
            cell_velocity(p, c, f + c * Q, &r, &jx, &jy, &ux, &uy);
            su += ux;
            sv += uy;
        }
    out[0] = su / ((double)w * w);
    out[1] = sv / ((double)w * w);
}

/*
 * The local problem of orc_local_keff_os (leaf grown by `margin`, inner-window mean), each drive
 * starting from the state f_init + d * se * se * Q (d = 0: drive along x, 1: along y) instead of
 * rest. The stop test is Section 3's relative-change test applied to the whole mean velocity
 * vector, |ubar(t) - ubar(t - k)| <= tol k |ubar(t)|, rather than to its driven component only;
 * Eq. 17 as before.
 */
int orc_local_keff_from(int se, int margin, const double *kappa_ext, double tau, double nu, double eps,
                        double gconst, double tol, long max_steps, int check_every, const double *f_init,
                        double keff[4], double ubar[4], long steps[2])
{
    lattice_init();
    const int s = se - 2 * margin;
    if (margin < 0 || s < 1) return -1;
    orc_problem p;
    memset(&p, 0, sizeof p);
    p.nx = se; p.ny = se; p.tau = tau; p.nu = nu; p.eps = eps;
    p.walls = 0; p.kappa = kappa_ext;
    long n = (long)se * se;
    double *f = (double *)malloc(sizeof(double) * n * Q);
    double *g = (double *)malloc(sizeof(double) * n * Q);
    int nconv = 0;
    for (int d = 0; d < 2; ++d) {
        p.gx = d == 0 ? gconst : 0.0;
        p.gy = d == 0 ? 0.0 : gconst;
        memcpy(f, f_init + (long)d * n * Q, sizeof(double) * n * Q);
        /* from a start near the steady state the transverse mean velocity can still be moving
           when the driven one has stopped: the stop test takes the whole vector ubar */
        double prev[2] = {0.0, 0.0}, m[2];
        long st = 0;
        int conv = 0;
        while (st < max_steps) {
            orc_step(&p, f, g);
            memcpy(f, g, sizeof(double) * n * Q);
            ++st;
            if (check_every > 0 && st % check_every == 0) {
                mean_velocity_window(&p, f, margin, margin, s, m);
                const double dx = m[0] - prev[0], dy = m[1] - prev[1];
                if (tol > 0.0 && st > check_every &&
                    sqrt(dx * dx + dy * dy) <= tol * check_every * sqrt(m[0] * m[0] + m[1] * m[1])) {
                    conv = 1;
                    break;
                }
                prev[0] = m[0];
                prev[1] = m[1];
            }
        }
        mean_velocity_window(&p, f, margin, margin, s, ubar + 2 * d);
        steps[d] = st;
        nconv += conv;
    }
    keff[0] = nu / gconst * ubar[0];
    keff[1] = nu / gconst * ubar[2];
    keff[2] = nu / gconst * ubar[1];
    keff[3] = nu / gconst * ubar[3];
    free(f);
    free(g);
    return nconv;
}

/* Mean over the w x w window at (x0, y0) of the density gradient, by central differences cell by
   cell: (rho(x + 1, y) - rho(x - 1, y)) / 2 and (rho(x, y + 1) - rho(x, y - 1)) / 2. The window
   must leave one cell on every side inside the lattice. */
static void mean_density_gradient_window(const orc_problem *p, const double *f, int x0, int y0, int w,
                                         double out[2])
{
    double sx = 0.0, sy = 0.0;
    for (int y = y0; y < y0 + w; ++y)
        for (int x = x0; x < x0 + w; ++x) {
            double r[4] = {0.0, 0.0, 0.0, 0.0};
            const long nb[4] = {(long)y * p->nx + x + 1, (long)y * p->nx + x - 1, (long)(y + 1) * p->nx + x,
                                (long)(y - 1) * p->nx + x};
            for (int k = 0; k < 4; ++k)
                for (int a = 0; a < Q; ++a) r[k] += f[nb[k] * Q + a];
            sx += 0.5 * (r[0] - r[1]);
            sy += 0.5 * (r[2] - r[3]);
        }
    out[0] = sx / ((double)w * w);
    out[1] = sy / ((double)w * w);
}

/*
 * Local-global local problem (the treatment the Conclusions name beside oversampling for
 * high-contrast media): the leaf grown by `margin` >= 1 cells on every side (se = s + 2 margin),
 * under the constant drive G along x (d = 0) or y (d = 1) as in Section 3, but closed by a ring of
 * fixed cells instead of periodicity: the outermost cells of the patch emit, every step, the
 * equilibrium of a given state (drho, u, v) taken from a global coarse solution, and the whole
 * patch starts from the equilibrium of that state. Stop test as orc_local_keff_from (the whole
 * mean velocity vector of the inner window). state: [2][se][se][3] (drho, u, v per cell, one
 * block per drive). win: [2][4], per drive the inner window's mean u, mean v, mean d(rho)/dx and
 * mean d(rho)/dy.
 * ring = 1: the ring keeps the state's velocity. ring = 2 (pressure only): the ring keeps the
 * state's density, and its velocity follows the flow inside: at every check (every check_every
 * steps) each ring cell takes the velocity (Eq. 15) of its inward neighbour (the diagonal one at a
 * corner) in the state of that check, and emits with it from the second step after the check on.
 * K* follows from the Brinkman equation of Section 2 at steady state, averaged over the window:
 * <u> = (K* / nu) <F> with the force per unit mass F = G e_d - grad(p) / (eps rho0), p = c_s^2 rho,
 * rho0 = 1. With U and F the 2 x 2 matrices whose columns are the two drives, K* = nu U F^-1,
 * written to keff as (xx, xy, yx, yy). A periodic patch has <grad rho> = 0 and this is Eq. 17.
 */
int orc_local_lg(int se, int margin, const double *kappa_ext, double tau, double nu, double eps, double gconst,
                 double tol, long max_steps, int check_every, int ring, const double *state, double win[8],
                 double keff[4], long steps[2])
{
    lattice_init();
    const int s = se - 2 * margin;
    if (margin < 1 || s < 1) return -1;
    orc_problem p;
    memset(&p, 0, sizeof p);
    p.nx = se; p.ny = se; p.tau = tau; p.nu = nu; p.eps = eps;
    p.walls = 0; p.kappa = kappa_ext;
    long n = (long)se * se;
    double *f = (double *)malloc(sizeof(double) * n * Q);
    double *g = (double *)malloc(sizeof(double) * n * Q);
    double *fixed = (double *)malloc(sizeof(double) * n * 4);
    double *pend = (double *)malloc(sizeof(double) * n * 2);     /* ring velocities taken at a check */
    int nconv = 0;
    for (int d = 0; d < 2; ++d) {
        p.gx = d == 0 ? gconst : 0.0;
        p.gy = d == 0 ? 0.0 : gconst;
        const double *sd = state + (long)d * n * 3;
        for (long c = 0; c < n; ++c) {
            const int x = (int)(c % se), y = (int)(c / se);
            fixed[c * 4] = (x == 0 || y == 0 || x == se - 1 || y == se - 1) ? 1.0 : 0.0;
            fixed[c * 4 + 1] = sd[c * 3];
            fixed[c * 4 + 2] = sd[c * 3 + 1];
            fixed[c * 4 + 3] = sd[c * 3 + 2];
            const double rho = 1.0 + sd[c * 3];
            for (int a = 0; a < Q; ++a)
                f[c * Q + a] = W[a] * rho * (1.0 + 3.0 * (E[a][0] * sd[c * 3 + 1] + E[a][1] * sd[c * 3 + 2]));
        }
        p.fixed = fixed;
        double prev[2] = {0.0, 0.0}, m[2];
        long st = 0, apply_at = -1;
        int conv = 0;
        while (st < max_steps) {
            if (st == apply_at)
                for (long c = 0; c < n; ++c)
                    if (fixed[c * 4] != 0.0) {
                        fixed[c * 4 + 2] = pend[c * 2];
                        fixed[c * 4 + 3] = pend[c * 2 + 1];
                    }
            orc_step(&p, f, g);
            memcpy(f, g, sizeof(double) * n * Q);
            ++st;
            if (check_every > 0 && st % check_every == 0) {
                mean_velocity_window(&p, f, margin, margin, s, m);
                const double dx = m[0] - prev[0], dy = m[1] - prev[1];
                if (tol > 0.0 && st > check_every &&
                    sqrt(dx * dx + dy * dy) <= tol * check_every * sqrt(m[0] * m[0] + m[1] * m[1])) {
                    conv = 1;
                    break;
                }
                prev[0] = m[0];
                prev[1] = m[1];
                if (ring == 2) {
                    for (long c = 0; c < n; ++c) {
                        if (fixed[c * 4] == 0.0) continue;
                        const int x = (int)(c % se), y = (int)(c / se);
                        const int xi = x == 0 ? 1 : (x == se - 1 ? se - 2 : x);
                        const int yi = y == 0 ? 1 : (y == se - 1 ? se - 2 : y);
                        const long ci = (long)yi * se + xi;
                        double r2, jx2, jy2;
                        cell_velocity(&p, ci, f + ci * Q, &r2, &jx2, &jy2, pend + c * 2, pend + c * 2 + 1);
                    }
                    apply_at = st + 2;
                }
            }
        }
        mean_velocity_window(&p, f, margin, margin, s, win + 4 * d);
        mean_density_gradient_window(&p, f, margin, margin, s, win + 4 * d + 2);
        steps[d] = st;
        nconv += conv;
    }
    /* columns: drives; rows: components */
    const double u11 = win[0], u21 = win[1], u12 = win[4], u22 = win[5];
    const double f11 = gconst - win[2] / (3.0 * eps), f21 = -win[3] / (3.0 * eps);
    const double f12 = -win[6] / (3.0 * eps), f22 = gconst - win[7] / (3.0 * eps);
    const double det = f11 * f22 - f12 * f21;
    const double i11 = f22 / det, i12 = -f12 / det, i21 = -f21 / det, i22 = f11 / det;
    keff[0] = nu * (u11 * i11 + u12 * i21);   /* K*_xx */
    keff[1] = nu * (u11 * i12 + u12 * i22);   /* K*_xy */
    keff[2] = nu * (u21 * i11 + u22 * i21);   /* K*_yx */
    keff[3] = nu * (u21 * i12 + u22 * i22);   /* K*_yy */
    free(f);
    free(g);
    free(fixed);
    free(pend);
    return nconv;
}

int orc_local_keff_os(int se, int margin, const double *kappa_ext, double tau, double nu, double eps,
                      double gconst, double tol, long max_steps, int check_every,
                      double keff[4], double ubar[4], long steps[2])
{
    lattice_init();
    const int s = se - 2 * margin;
    if (margin < 0 || s < 1) return -1;
    orc_problem p;
    memset(&p, 0, sizeof p);
    p.nx = se; p.ny = se; p.tau = tau; p.nu = nu; p.eps = eps;
    p.walls = 0; p.kappa = kappa_ext;
    long n = (long)se * se;
    double *f = (double *)malloc(sizeof(double) * n * Q);
    double *g = (double *)malloc(sizeof(double) * n * Q);
    int nconv = 0;
    for (int d = 0; d < 2; ++d) {
        p.gx = d == 0 ? gconst : 0.0;
        p.gy = d == 0 ? 0.0 : gconst;
        orc_init_rest(&p, f);
        /* from a start near the steady state the transverse mean velocity can still be moving
           when the driven one has stopped: the stop test takes the whole vector ubar */
        double prev[2] = {0.0, 0.0}, m[2];
        long st = 0;
        int conv = 0;
        while (st < max_steps) {
            orc_step(&p, f, g);
            memcpy(f, g, sizeof(double) * n * Q);
            ++st;
            if (check_every > 0 && st % check_every == 0) {
                mean_velocity_window(&p, f, margin, margin, s, m);
                const double dx = m[0] - prev[0], dy = m[1] - prev[1];
                if (tol > 0.0 && st > check_every &&
                    sqrt(dx * dx + dy * dy) <= tol * check_every * sqrt(m[0] * m[0] + m[1] * m[1])) {
                    conv = 1;
                    break;
                }
                prev[0] = m[0];
                prev[1] = m[1];
            }
        }
        mean_velocity_window(&p, f, margin, margin, s, ubar + 2 * d);
        steps[d] = st;
        nconv += conv;
    }
    keff[0] = nu / gconst * ubar[0];   /* Eq. 17 on the inner window, as in orc_local_keff */
    keff[1] = nu / gconst * ubar[2];
    keff[2] = nu / gconst * ubar[1];
    keff[3] = nu / gconst * ubar[3];
    free(f);
    free(g);
    return nconv;
}

/* Mean of a [ny][nx] field over r x r blocks -> [ny/r][nx/r] (fine-to-coarse comparison). */
void orc_block_average(int nx, int ny, int r, const double *a, double *out)
{
    int cx = nx / r, cy = ny / r;
    for (int J = 0; J < cy; ++J)
        for (int I = 0; I < cx; ++I) {
            double s = 0.0;
            for (int y = J * r; y < (J + 1) * r; ++y)
                for (int x = I * r; x < (I + 1) * r; ++x) s += a[(long)y * nx + x];
            out[(long)J * cx + I] = s / ((double)r * r);
        }
}
