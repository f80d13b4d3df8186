// local.cu -- batched local problems of the upscaling scheme (Section 3):
// for every leaf (square subdomain) two periodic fine-grid runs driven by
// G1 = (G, 0) and G2 = (0, G), each until its volume-averaged velocity settles,
// then K* from Eq. 17. All jobs of a batch run in ONE persistent launch.
//
// Design (one CTA per SM, 1024 threads):
//  * A CTA owns CMAX = 4096 lattice cells in shared memory and works on one
//    leaf size s at a time: it holds nslots = min(CMAX / s^2, MAXSLOTS) jobs of
//    that size side by side ("slots"). Jobs are popped from a per-size device
//    queue with atomicAdd (no waiting, so nothing can hang). When a job's
//    steady-state test passes, its slot is refilled from the queue at once.
//  * The distributions of a slot stay resident in shared memory for the whole
//    job and are updated in place with the AA access pattern: on even steps a
//    cell reads its own nine values and writes the post-collision values into
//    the opposite slots of the same cell; on odd steps it reads them from its
//    neighbours' opposite slots and writes streamed values into its
//    neighbours' own slots. Each cell touches the same nine locations for both
//    reading and writing within a step, so only one barrier per step is needed
//    and one buffer suffices (64 x 64 leaves fit).
//  * The collision is the same simplified Shan-Chen update as the fine grid
//    (Eqs. 6, 16, 2, 13) in FP32 deviation form, periodic closure on the leaf.
//  * Every check_every steps of a job (and at max_steps) its mean velocity is
//    reduced in FP64 by one warp in a fixed order (bitwise reproducible); the
//    job ends when |ubar_d(t) - ubar_d(t - k)| <= tol k |ubar_d(t)| on the driven
//    component d (a job started from the Darcy state: the same test on the whole
//    vector ubar). Drive 1 writes K*_xx, K*_yx and drive 2 K*_xy, K*_yy (Eq. 17).
//  * A wall-clock limit (globaltimer) bounds the launch: past it every CTA
//    abandons its jobs with LBM_ETIMEOUT and returns.
//  * Variants of the same kernel (template MODE): jobs from rest (the paper's
//    local problems), jobs from the patch's Darcy state (warm_start), and
//    local-global jobs, whose patch is closed by a ring of cells held at a
//    coarse solution instead of periodicity (lbm_local_keff_lg).
#include "lbm_internal.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <vector>

namespace lbm {

lbm_status fail(lbm_status s, const char *fmt, ...);
bool is_device_ptr(const void *p);
int sm_count(int dev);
void count_launches(int64_t n);

namespace {

constexpr int LOCAL_THREADS = 1024;
// cells resident per CTA: 4096 in FP32 (leaves up to 64 x 64), 2048 in FP64 (up to 45 x 45);
// either way 12 values per cell fill 192 KiB of shared memory
template <typename T> struct LocalCfg {
    static constexpr int CMAX = sizeof(T) == 8 ? 2048 : 4096;
    static constexpr int CPT = CMAX / LOCAL_THREADS;   // cells per thread
    static constexpr size_t SMEM = (size_t)(9 + 1 + 2) * CMAX * sizeof(T);
};
constexpr int MAXSLOTS = 64;
constexpr int MAXCLASS = 64;

struct LocalArgs {
    const float *kappa;       // field [ny][nx]
    int nx, ny;
    int margin;               // oversampling margin: a job's patch is its leaf grown by margin cells
    const int *leaves;        // [n][3] (x0, y0, size)
    const int *jobs;          // job = 2 * leaf + drive, grouped by size class
    int nclass;
    int class_off[MAXCLASS + 1];
    int class_size[MAXCLASS];
    int *heads;               // [nclass] queue heads (zeroed before launch)
    const int *table;         // nullptr, or a device class table (layout DT_* in lbm_internal.h) that
                              // replaces nclass, class_off and class_size (heads then point into it)
    double omega, two_tau, omt, half_eps, gmag;
    float kf[4];              // collision constants (K_*) in FP32 and FP64, set by cell_consts()
    double kd[4];
    double eps_nu;            // eps * nu for the drag coefficient
    double nu_over_g;         // nu / G for Eq. 17
    int warm;                 // 1: patches of WARM_MIN cells or more (side a multiple of 8) start from
                              // their finite-volume Darcy state instead of rest (the kernel's WARM
                              // variant)
    double warm_rho;          // 3 eps G: density deviation per unit of the unit-drive Darcy pressure
    double warm_u;            // G / nu: velocity per unit of the unit-drive Darcy face flux
    const float *lg_state;    // local-global jobs: coarse (drho, u, v) [2 drives][3][lg_nyc][lg_nxc]
    int lg_r, lg_nxc, lg_nyc; // coarse cell size in fine cells, coarse lattice size
    int lg_ring;              // 1: the ring holds the coarse velocity; 2: pressure only (velocity
                              // refreshed from the inward neighbours at every check)
    double *lg_win;           // [n][2][4]: the inner window's mean u, v, d(drho)/dx, d(drho)/dy per drive
    double tol;
    int check_every;
    long long max_steps;
    double *keff;             // [n][4]
    int *status;              // [n] (zeroed before launch)
    int *steps;               // [n][2] or nullptr
    int *worst;               // [1] (zeroed)
    int *abort_flag;          // [1] (zeroed)
    unsigned long long time_limit_ns;
};

struct Slot {
    int job;                  // -1: empty
    int leaf, drive, x0, y0;
    double prev;              // driven mean velocity at the previous check
    double prev_t;            // transverse mean velocity at the previous check
};

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// drag fraction e = 1 - d = eps nu / (2 kappa + eps nu) of Eq. 6 (see the fine-grid step)
__device__ __forceinline__ double coef_e(float k, double eps_nu)
{
    if (!(k >= 0.0f)) return 1.0;
    if (eps_nu == 0.0 || isinf(k)) return 0.0;
    if (k == 0.0f) return 1.0;
    return eps_nu / (2.0 * (double)k + eps_nu);
}

// Per-slot values every cell reads each step, packed for one 16-byte shared load.
struct SlotHot {
    int tstart;       // CTA step of the job's step 0 (always even; differences taken modulo 2^32)
    int next_check;   // job step of the next steady-state check
    int flags;        // bit 0: active, bit 1: driven along y, bit 2: cells not yet set up
    int store;        // CTA step at which the cells store their velocity: tstart + min(next_check, max_steps)
};

// Collision constants (host-computed in the storage precision, so the FMAs read them from the
// constant bank): omega, Eq. 16's 2 tau and 1 - 2 tau, and eps G / 2.
enum { K_OMEGA, K_TWO_TAU, K_OMT, K_HG, K_N };

void cell_consts(LocalArgs &a)
{
    const double k[K_N] = {a.omega, a.two_tau, a.omt, a.half_eps * a.gmag};
    for (int i = 0; i < K_N; ++i) {
        a.kd[i] = k[i];
        a.kf[i] = (float)k[i];
    }
}

template <typename T> __device__ __forceinline__ T kc(const LocalArgs &a, int i);
template <> __device__ __forceinline__ float kc<float>(const LocalArgs &a, int i) { return a.kf[i]; }
template <> __device__ __forceinline__ double kc<double>(const LocalArgs &a, int i) { return a.kd[i]; }

// Eqs. 6, 16, 2 and 13 for one cell in deviation form with the D2Q9 sums written out (a product
// with a zero velocity component is not free in IEEE arithmetic): moments, r = j + eps rho G / 2,
// rho u = (1 - e) r, rho u_eq = 2 tau rho u + (1 - 2 tau) j, g_eq = w_a (drho + 3 e_a . rho u_eq),
// and BGK as g + omega (g_eq - g): the difference is formed first, so the rounding of the update
// stays at the size of the non-equilibrium part (FP32 solves in the Darcy regime depend on it).
// TAU1: tau = 1 exactly, where Eq. 16 reads rho u_eq = 2 rho u - j and Eq. 13 with omega = 1
// leaves the equilibrium itself, so g_eq is stored directly. Returns rho u and rho.
template <typename T, bool TAU1>
__device__ __forceinline__ void collide_d2q9(T (&g)[Q], T e, T hgx, T hgy, const LocalArgs &a, T &rux, T &ruy,
                                             T &rho, T &drho)
{
    const T s13 = g[1] + g[3], s24 = g[2] + g[4], s57 = g[5] + g[7], s68 = g[6] + g[8];
    drho = g[0] + ((s13 + s24) + (s57 + s68));
    const T d57 = g[5] - g[7], d86 = g[8] - g[6];
    const T jx = (g[1] - g[3]) + (d57 + d86);
    const T jy = (g[2] - g[4]) + (d57 - d86);
    rho = T(1) + drho;
    const T rx = fma(hgx, rho, jx), ry = fma(hgy, rho, jy);
    rux = fma(-e, rx, rx);
    ruy = fma(-e, ry, ry);
    T uex, uey;
    if constexpr (TAU1) {
        uex = fma(T(2), rux, -jx);
        uey = fma(T(2), ruy, -jy);
    } else {
        uex = fma(kc<T>(a, K_TWO_TAU), rux, kc<T>(a, K_OMT) * jx);
        uey = fma(kc<T>(a, K_TWO_TAU), ruy, kc<T>(a, K_OMT) * jy);
    }
    const T w1 = T(1.0 / 9.0), w2 = T(1.0 / 36.0);
    const T tx = T(3) * uex, ty = T(3) * uey, sp = tx + ty, sm = tx - ty;
    if constexpr (TAU1) {
        g[0] = T(4.0 / 9.0) * drho;
        g[1] = w1 * (drho + tx);
        g[3] = w1 * (drho - tx);
        g[2] = w1 * (drho + ty);
        g[4] = w1 * (drho - ty);
        g[5] = w2 * (drho + sp);
        g[7] = w2 * (drho - sp);
        g[8] = w2 * (drho + sm);
        g[6] = w2 * (drho - sm);
    } else {
        const T om = kc<T>(a, K_OMEGA);
        g[0] = fma(om, T(4.0 / 9.0) * drho - g[0], g[0]);
        g[1] = fma(om, w1 * (drho + tx) - g[1], g[1]);
        g[3] = fma(om, w1 * (drho - tx) - g[3], g[3]);
        g[2] = fma(om, w1 * (drho + ty) - g[2], g[2]);
        g[4] = fma(om, w1 * (drho - ty) - g[4], g[4]);
        g[5] = fma(om, w2 * (drho + sp) - g[5], g[5]);
        g[7] = fma(om, w2 * (drho - sp) - g[7], g[7]);
        g[8] = fma(om, w2 * (drho + sm) - g[8], g[8]);
        g[6] = fma(om, w2 * (drho - sm) - g[6], g[6]);
    }
}

// One lattice step of every active slot; ODD selects the half of the AA pattern. Job starts are
// aligned to even CTA steps, so the parity of a job's step is the CTA step's, the same for all.
// LG (local-global jobs): the patch's outermost cells emit a fixed state instead of their
// collision result: the equilibrium at density deviation D and momentum (UX, UY), set up when the
// job starts; the other cells also store their density deviation (RHO) with their velocity.
template <typename T, bool TAU1, bool ODD, bool LG>
__device__ __forceinline__ void local_step(T *F, const T *D, T *UX, T *UY, T *RHO, const int4 *hot,
                                           const int (&cgeo)[LocalCfg<T>::CPT], int s, int s2, unsigned Tcta, T hg,
                                           const LocalArgs &a, int tid)
{
    constexpr int CMAX = LocalCfg<T>::CMAX, CPT = LocalCfg<T>::CPT;
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
        const int geo = cgeo[i];
        if (geo < 0) continue;
        const int4 h = hot[geo >> 12];
        if (!(h.z & 1)) continue;
        const int c = tid + i * LOCAL_THREADS;
        T g[Q];
        // odd steps: the 8 neighbours with periodic closure on the leaf; cell x - e_a is read for
        // population a and cell x + e_a written, so each index serves both
        int n1 = 0, n2 = 0, n3 = 0, n4 = 0, n5 = 0, n6 = 0, n7 = 0, n8 = 0;
        if constexpr (!ODD) {
#pragma unroll
            for (int q = 0; q < Q; ++q) g[q] = F[q * CMAX + c];
        } else {
            const int cly = (geo >> 6) & 63, clx = geo & 63;
            const int row = c - clx;                                  // cell (0, cly) of the slot
            const int xm = (clx == 0 ? s : clx) - 1, xp = clx + 1 == s ? 0 : clx + 1;
            const int rm = cly == 0 ? row + s2 - s : row - s;        // row y - 1
            const int rp = cly + 1 == s ? row - s2 + s : row + s;    // row y + 1
            n1 = row + xp; n3 = row + xm; n2 = rp + clx; n4 = rm + clx;     // x + e_a for a = 1..4
            n5 = rp + xp; n6 = rp + xm; n7 = rm + xm; n8 = rm + xp;         // a = 5..8
            g[0] = F[c];
            g[1] = F[3 * CMAX + n3]; g[3] = F[1 * CMAX + n1];
            g[2] = F[4 * CMAX + n4]; g[4] = F[2 * CMAX + n2];
            g[5] = F[7 * CMAX + n7]; g[7] = F[5 * CMAX + n5];
            g[6] = F[8 * CMAX + n8]; g[8] = F[6 * CMAX + n6];
        }
        const T e = D[c];
        const bool along_y = (h.z & 2) != 0;
        T rux, ruy, rho, drho;
        collide_d2q9<T, TAU1>(g, e, along_y ? T(0) : hg, along_y ? hg : T(0), a, rux, ruy, rho, drho);
        bool ring = false;
        if constexpr (LG) {
            const int lx = geo & 63, ly = (geo >> 6) & 63;
            ring = lx == 0 || ly == 0 || lx == s - 1 || ly == s - 1;
            if (ring) {
                const T dr = D[c], tx = T(3) * UX[c], ty = T(3) * UY[c], sp = tx + ty, sm = tx - ty;
                const T w1 = T(1.0 / 9.0), w2 = T(1.0 / 36.0);
                g[0] = T(4.0 / 9.0) * dr;
                g[1] = w1 * (dr + tx); g[3] = w1 * (dr - tx);
                g[2] = w1 * (dr + ty); g[4] = w1 * (dr - ty);
                g[5] = w2 * (dr + sp); g[7] = w2 * (dr - sp);
                g[8] = w2 * (dr + sm); g[6] = w2 * (dr - sm);
            }
        }
        if (Tcta == (unsigned)h.w && !ring) {
            UX[c] = rux / rho;                                   // Eq. 15
            UY[c] = ruy / rho;
            if constexpr (LG) RHO[c] = drho;
        }
        if constexpr (!ODD) {
#pragma unroll
            for (int q = 0; q < Q; ++q) F[opp(q) * CMAX + c] = g[q];
        } else {
            F[c] = g[0];
            F[1 * CMAX + n1] = g[1]; F[3 * CMAX + n3] = g[3];
            F[2 * CMAX + n2] = g[2]; F[4 * CMAX + n4] = g[4];
            F[5 * CMAX + n5] = g[5]; F[7 * CMAX + n7] = g[7];
            F[6 * CMAX + n6] = g[6]; F[8 * CMAX + n8] = g[8];
        }
    }
}

// ---------------------------------------------------------------- the Darcy start
// Darcy flow through a patch under the job's drive, by finite volumes: the flux across the face
// between two neighbouring cells is k_f (p_i - p_j + G . (x_j - x_i)) with k_f the harmonic mean of
// the two cells, every cell conserves mass, and the patch is periodic. It is solved with a unit
// drive by conjugate gradients with the diagonal as preconditioner (the system's arrays live in
// the new job's own part of F, which is free until its distributions are written), then the
// run starts from g_a = w_a (drho + 3 e_a . j) with drho = 3 eps G p (the pressure p / rho0 = c_s^2
// drho balances the drive as in Darcy's law with porosity eps) and j = rho u, u the mean of the
// cell's two face fluxes along each axis times G / nu. Every fresh slot of the class is solved
// at once; each per-slot sum is taken warp by warp (in the storage precision: the 32 terms of a
// warp) and then over the slot's warps in FP64, in a fixed order, so the start, and everything
// after it, is bitwise reproducible.
constexpr int WARM_MIN = 16;
constexpr int WARM_MAXIT = 4000;

__device__ __forceinline__ double harmonic_face(double a, double b)
{
    if (isinf(a)) return isinf(b) ? a : 2.0 * b;
    if (isinf(b)) return 2.0 * a;
    return a + b > 0.0 ? 2.0 * a * b / (a + b) : 0.0;
}

// Geometry of cell c of a class of side s: its slot j, position (lx, ly) and the four neighbours
// within the slot (periodic closure).
struct WarmCell {
    int j, lx, ly, l, r, d, u;
};
__device__ __forceinline__ WarmCell warm_cell(int c, int s, int s2)
{
    WarmCell w;
    w.j = c / s2;
    const int loc = c - w.j * s2;
    w.ly = loc / s;
    w.lx = loc - w.ly * s;
    const int row = c - w.lx;
    w.l = row + (w.lx == 0 ? s - 1 : w.lx - 1);
    w.r = row + (w.lx + 1 == s ? 0 : w.lx + 1);
    w.d = w.ly == 0 ? c + s2 - s : c - s;
    w.u = w.ly + 1 == s ? c - s2 + s : c + s;
    return w;
}

// DIR (local-global patches): the patch's outermost ring is not periodic closure but Dirichlet
// data, its pressure held at the ring state's drho / (3 eps G) (D holds the ring's drho); only the
// inner cells are unknowns, and only they get the Darcy start.
template <typename T, bool DIR>
__device__ __forceinline__ void warm_start_fresh(const LocalArgs &a, T *F, const T *D, int4 *hot, const Slot *slots,
                                              int s, int nslots)
{
    constexpr int CMAX = LocalCfg<T>::CMAX, CPT = LocalCfg<T>::CPT, NW = LOCAL_THREADS / 32;
    __shared__ double w_rz[MAXSLOTS], w_stop[MAXSLOTS];
    __shared__ T w_alpha[MAXSLOTS], w_beta[MAXSLOTS];
    __shared__ int w_on[MAXSLOTS];
    __shared__ double w_red[CPT * NW][2];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int s2 = s * s, ncell = nslots * s2, nk = s2 / 32;
    T *KX = F, *KY = F + CMAX, *P = F + 2 * CMAX, *R = F + 3 * CMAX, *DV = F + 4 * CMAX, *AD = F + 5 * CMAX;
    T *IDG = F + 6 * CMAX;                           // 1 / diagonal (0 where the diagonal is 0)
    // this thread's cells: slot j and position (lx, ly), found once and packed as
    // j << 12 | ly << 6 | lx (s2 is a multiple of 64, so the 32 cells of a warp always belong to
    // one slot); bit i of `mine` marks a cell of a fresh slot
    int geo[CPT];
    unsigned mine = 0;
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
        const int c = tid + i * LOCAL_THREADS;
        const WarmCell w = warm_cell(c < ncell ? c : 0, s, s2);
        geo[i] = w.j << 12 | w.ly << 6 | w.lx;
        if (c < ncell && (hot[w.j].z & 5) == 5) mine |= 1u << i;
    }
    // DIR: bit i of `ringm` marks a ring cell of a fresh slot (fixed pressure, not an unknown)
    unsigned ringm = 0;
    if constexpr (DIR) {
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
            const int lx = geo[i] & 63, ly = (geo[i] >> 6) & 63;
            if ((mine >> i & 1) && (lx == 0 || ly == 0 || lx == s - 1 || ly == s - 1)) ringm |= 1u << i;
        }
    }
    const unsigned unk = mine & ~ringm;                      // the unknowns of this thread
    // the neighbours of cell i within its slot (periodic closure)
    auto cell = [&](int i) {
        const int c = tid + i * LOCAL_THREADS, lx = geo[i] & 63, ly = (geo[i] >> 6) & 63;
        WarmCell w;
        w.j = geo[i] >> 12;
        w.lx = lx;
        w.ly = ly;
        w.l = lx == 0 ? c + s - 1 : c - 1;
        w.r = lx + 1 == s ? c - s + 1 : c + 1;
        w.d = ly == 0 ? c + s2 - s : c - s;
        w.u = ly + 1 == s ? c - s2 + s : c + s;
        return w;
    };
    // per-slot sums of (x, y): the 32 cells of each warp in T, then the slot's warps in FP64 in
    // a fixed order
    auto slot_sum2 = [&](int i, T x, T y) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, off);
            y += __shfl_xor_sync(0xffffffffu, y, off);
        }
        if (lane == 0) {
            w_red[i * NW + wid][0] = (double)x;
            w_red[i * NW + wid][1] = (double)y;
        }
    };
    // each slot's warp sums folded by one warp (slot j by warp j mod NW: every lane a strided
    // share, then a butterfly), after which its lane 0 runs `then(j, x, y)`; one barrier before
    auto slot_fold = [&](auto then) {
        __syncthreads();
        for (int j = wid; j < nslots; j += NW) {
            double x = 0.0, y = 0.0;
            for (int k = j * nk + lane; k < (j + 1) * nk; k += 32) {
                x += w_red[k][0];
                y += w_red[k][1];
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                x += __shfl_xor_sync(0xffffffffu, x, off);
                y += __shfl_xor_sync(0xffffffffu, y, off);
            }
            if (lane == 0) then(j, x, y);
        }
    };
    auto kappa_at = [&](int j, int lx, int ly) {
        int gx = slots[j].x0 + lx, gy = slots[j].y0 + ly;
        gx = gx < 0 ? gx + a.nx : (gx >= a.nx ? gx - a.nx : gx);
        gy = gy < 0 ? gy + a.ny : (gy >= a.ny ? gy - a.ny : gy);
        return (double)a.kappa[(int64_t)gy * a.nx + gx];
    };

    // face permeabilities
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
        if (!(mine >> i & 1)) continue;
        const int c = tid + i * LOCAL_THREADS;
        const WarmCell w = cell(i);
        const double k = kappa_at(w.j, w.lx, w.ly);
        KX[c] = (T)harmonic_face(k, kappa_at(w.j, w.lx + 1 == s ? 0 : w.lx + 1, w.ly));
        KY[c] = (T)harmonic_face(k, kappa_at(w.j, w.lx, w.ly + 1 == s ? 0 : w.ly + 1));
    }
    __syncthreads();
    if constexpr (DIR) {
        // the ring's pressures, and zero directions there
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
            if (!(ringm >> i & 1)) continue;
            const int c = tid + i * LOCAL_THREADS;
            P[c] = D[c] / (T)a.warm_rho;
            DV[c] = T(0);
            R[c] = T(0);
            IDG[c] = T(0);
        }
        __syncthreads();
    }
    // start: p = 0 on the unknowns, r = b - A p, d = r / diag
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
        const int c = tid + i * LOCAL_THREADS;
        T x = T(0), y = T(0);
        if (unk >> i & 1) {
            const WarmCell w = cell(i);
            T b = (hot[w.j].z & 2) ? KY[w.d] - KY[c] : KX[w.l] - KX[c];
            if constexpr (DIR) {
                // minus A p for p = 0 here and the ring's pressures on its ring neighbours
                auto pr = [&](int n, int nl) { return nl ? P[n] : T(0); };
                const int lx = w.lx, ly = w.ly;
                b += KX[c] * pr(w.r, lx + 1 == s - 1) + KX[w.l] * pr(w.l, lx - 1 == 0) +
                     KY[c] * pr(w.u, ly + 1 == s - 1) + KY[w.d] * pr(w.d, ly - 1 == 0);
            }
            const T dg = KX[c] + KX[w.l] + KY[c] + KY[w.d];
            const T idg = dg > T(0) ? T(1) / dg : T(0);
            const T z = b * idg;
            IDG[c] = idg;
            P[c] = T(0);
            R[c] = b;
            DV[c] = z;
            x = b * b;
            y = b * z;
        }
        slot_sum2(i, x, y);
    }
    slot_fold([&](int j, double rr, double rz) {
        w_on[j] = (hot[j].z & 5) == 5 && rr > 0.0;
        w_rz[j] = rz;
        // (1e-5 relative residual)^2; with a Dirichlet ring the initial residual carries the ring's
        // whole pressure level, so the flow-carrying differences need 1e-7
        w_stop[j] = (DIR ? 1e-14 : 1e-10) * rr;
    });
    int any = __syncthreads_or(tid < nslots && w_on[tid]);
    for (int it = 0; any && it < WARM_MAXIT; ++it) {
        unsigned act = 0;                                    // unknowns of slots still iterating
#pragma unroll
        for (int i = 0; i < CPT; ++i)
            if ((unk >> i & 1) && w_on[geo[i] >> 12]) act |= 1u << i;
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
            const int c = tid + i * LOCAL_THREADS;
            T x = T(0);
            if (act >> i & 1) {
                const WarmCell w = cell(i);
                const T dc = DV[c];
                const T ad = KX[c] * (dc - DV[w.r]) + KX[w.l] * (dc - DV[w.l]) + KY[c] * (dc - DV[w.u]) +
                             KY[w.d] * (dc - DV[w.d]);
                AD[c] = ad;
                x = dc * ad;
            }
            slot_sum2(i, x, T(0));
        }
        slot_fold([&](int j, double dad, double) {
            if (!w_on[j]) return;
            if (!(dad > 0.0)) w_on[j] = 0;                   // a direction in the null space
            else w_alpha[j] = (T)(w_rz[j] / dad);
        });
        __syncthreads();
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
            const int c = tid + i * LOCAL_THREADS;
            T x = T(0), y = T(0);
            if ((act >> i & 1) && w_on[geo[i] >> 12]) {
                const T al = w_alpha[geo[i] >> 12];
                P[c] = fma(al, DV[c], P[c]);
                const T r = fma(-al, AD[c], R[c]);
                R[c] = r;
                x = r * r;
                y = r * r * IDG[c];
            }
            slot_sum2(i, x, y);
        }
        slot_fold([&](int j, double rr, double rz) {
            if (!w_on[j]) return;
            w_beta[j] = (T)(rz / w_rz[j]);
            w_rz[j] = rz;
            if (rr <= w_stop[j]) w_on[j] = 0;
        });
        any = __syncthreads_or(tid < nslots && w_on[tid]);
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
            const int c = tid + i * LOCAL_THREADS;
            if (!(act >> i & 1) || !w_on[geo[i] >> 12]) continue;
            DV[c] = fma(w_beta[geo[i] >> 12], DV[c], R[c] * IDG[c]);
        }
        __syncthreads();
    }
    // the start state: rho and j from the pressure and the face fluxes, staged in AD (drho) and
    // DV / R (j) so that every read of the pressure comes before the distributions are written
    // (DIR: the ring's cells keep their own start; they emit their fixed state from the first step)
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
        if (!(unk >> i & 1)) continue;
        const int c = tid + i * LOCAL_THREADS;
        const WarmCell w = cell(i);
        const bool ydrive = (hot[w.j].z & 2) != 0;
        const T gx = ydrive ? T(0) : T(1), gy = ydrive ? T(1) : T(0);
        const T qr = KX[c] * (P[c] - P[w.r] + gx), ql = KX[w.l] * (P[w.l] - P[c] + gx);
        const T qu = KY[c] * (P[c] - P[w.u] + gy), qd = KY[w.d] * (P[w.d] - P[c] + gy);
        const T drho = (T)a.warm_rho * P[c];
        const T rho = T(1) + drho;
        AD[c] = drho;
        DV[c] = rho * (T)(0.5 * a.warm_u) * (qr + ql);
        R[c] = rho * (T)(0.5 * a.warm_u) * (qu + qd);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
        if (!(unk >> i & 1)) continue;
        const int c = tid + i * LOCAL_THREADS;
        const T drho = AD[c], jx = DV[c], jy = R[c];
        const T w1 = T(1.0 / 9.0), w2 = T(1.0 / 36.0);
        F[c] = T(4.0 / 9.0) * drho;
        F[1 * CMAX + c] = w1 * (drho + T(3) * jx);
        F[3 * CMAX + c] = w1 * (drho - T(3) * jx);
        F[2 * CMAX + c] = w1 * (drho + T(3) * jy);
        F[4 * CMAX + c] = w1 * (drho - T(3) * jy);
        F[5 * CMAX + c] = w2 * (drho + T(3) * (jx + jy));
        F[7 * CMAX + c] = w2 * (drho - T(3) * (jx + jy));
        F[8 * CMAX + c] = w2 * (drho + T(3) * (jx - jy));
        F[6 * CMAX + c] = w2 * (drho - T(3) * (jx - jy));
    }
}

// ---------------------------------------------------------------- local-global jobs
// The job's patch (its leaf grown by the margin) is closed by a ring of fixed cells instead of
// periodicity. The coarse solution of the job's drive, (drho, u, v) at the coarse cell centres,
// is interpolated bilinearly (periodic) to every cell of the patch, drho taken relative to the
// block's own coarse cell; every cell starts from the
// equilibrium of that state, and the outermost cells keep emitting, every step, what a cell in
// that state emits after a collision at tau = 1: the equilibrium at density deviation drho and
// momentum rho u + rho f_m / 2 (f_m of Eq. 5 at u, the drive along the job's axis; zero momentum
// where kappa = 0).
// The momentum a ring cell emits with: rho u + rho f_m / 2 for its density 1 + D[c] and the
// velocity (ux, uy), f_m of Eq. 5 at the cell's own kappa (zero momentum where kappa = 0).
template <typename T>
__device__ __forceinline__ void lg_ring_momentum(const LocalArgs &a, const T *D, T *UX, T *UY, int c, const Slot &sl,
                                                 int lx, int ly, double ux, double uy)
{
    int gx = sl.x0 + lx, gy = sl.y0 + ly;
    gx = gx < 0 ? gx + a.nx : (gx >= a.nx ? gx - a.nx : gx);
    gy = gy < 0 ? gy + a.ny : (gy >= a.ny ? gy - a.ny : gy);
    const float kap = a.kappa[(int64_t)gy * a.nx + gx];
    const double rho = 1.0 + (double)D[c];
    double jpx = 0.0, jpy = 0.0;
    if (kap != 0.0f) {
        const double drag = (a.eps_nu == 0.0 || isinf(kap)) ? 0.0 : a.eps_nu / (double)kap;
        const double hg = a.half_eps * a.gmag;                     // eps G / 2 along the drive
        jpx = rho * ux + rho * ((sl.drive == 0 ? hg : 0.0) - 0.5 * drag * ux);
        jpy = rho * uy + rho * ((sl.drive == 1 ? hg : 0.0) - 0.5 * drag * uy);
    }
    UX[c] = (T)jpx;
    UY[c] = (T)jpy;
}

template <typename T>
__device__ __forceinline__ void lg_start_cell(const LocalArgs &a, T *F, T *D, T *UX, T *UY, int c, const Slot &sl,
                                              int geo, int s, float kap)
{
    constexpr int CMAX = LocalCfg<T>::CMAX;
    const int lx = geo & 63, ly = (geo >> 6) & 63;
    // position in coarse cell units (coarse centre i at fine x = (i + 1/2) r - 1/2)
    const double X = ((double)(sl.x0 + lx) + 0.5) / a.lg_r - 0.5;
    const double Y = ((double)(sl.y0 + ly) + 0.5) / a.lg_r - 0.5;
    const double fx0 = floor(X), fy0 = floor(Y);
    const double wx = X - fx0, wy = Y - fy0;
    int i0 = (int)fx0 % a.lg_nxc, j0 = (int)fy0 % a.lg_nyc;
    i0 += i0 < 0 ? a.lg_nxc : 0;
    j0 += j0 < 0 ? a.lg_nyc : 0;
    const int i1 = i0 + 1 == a.lg_nxc ? 0 : i0 + 1, j1 = j0 + 1 == a.lg_nyc ? 0 : j0 + 1;
    const int64_t nc = (int64_t)a.lg_nxc * a.lg_nyc;
    const float *S = a.lg_state + (int64_t)sl.drive * 3 * nc;
    double v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float *P = S + k * nc;
        const double f00 = P[(int64_t)j0 * a.lg_nxc + i0], f01 = P[(int64_t)j0 * a.lg_nxc + i1];
        const double f10 = P[(int64_t)j1 * a.lg_nxc + i0], f11 = P[(int64_t)j1 * a.lg_nxc + i1];
        v[k] = (1.0 - wy) * ((1.0 - wx) * f00 + wx * f01) + wy * ((1.0 - wx) * f10 + wx * f11);
    }
    // densities relative to the block's own coarse cell: the local problem keeps rho0 = 1 at the
    // block (the global pressure level is arbitrary and would swamp FP32 deviations)
    const int bxc = (sl.x0 + a.margin) / a.lg_r, byc = (sl.y0 + a.margin) / a.lg_r;
    v[0] -= (double)S[(int64_t)byc * a.lg_nxc + bxc];
    const double rho = 1.0 + v[0];
    const T drho = (T)v[0], jx = (T)(rho * v[1]), jy = (T)(rho * v[2]);
    const T w1 = T(1.0 / 9.0), w2 = T(1.0 / 36.0);
    F[c] = T(4.0 / 9.0) * drho;
    F[1 * CMAX + c] = w1 * (drho + T(3) * jx);
    F[3 * CMAX + c] = w1 * (drho - T(3) * jx);
    F[2 * CMAX + c] = w1 * (drho + T(3) * jy);
    F[4 * CMAX + c] = w1 * (drho - T(3) * jy);
    F[5 * CMAX + c] = w2 * (drho + T(3) * (jx + jy));
    F[7 * CMAX + c] = w2 * (drho - T(3) * (jx + jy));
    F[8 * CMAX + c] = w2 * (drho + T(3) * (jx - jy));
    F[6 * CMAX + c] = w2 * (drho - T(3) * (jx - jy));
    if (lx == 0 || ly == 0 || lx == s - 1 || ly == s - 1) {
        D[c] = drho;
        lg_ring_momentum<T>(a, D, UX, UY, c, sl, lx, ly, v[1], v[2]);
    } else {
        D[c] = (T)coef_e(kap, a.eps_nu);
    }
}

// MODE: 0 local problems from rest, 1 from the Darcy state (warm_start), 2 local-global jobs
enum { MODE_REST = 0, MODE_WARM = 1, MODE_LG = 2 };

template <typename T, bool TAU1, int MODE>
__global__ void __launch_bounds__(LOCAL_THREADS, 1) local_keff_kernel(LocalArgs a)
{
    constexpr int CMAX = LocalCfg<T>::CMAX, CPT = LocalCfg<T>::CPT;
    constexpr bool WARM = MODE == MODE_WARM, LG = MODE == MODE_LG;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *F = reinterpret_cast<T *>(smem_raw);   // [9][CMAX]
    T *D = F + 9 * CMAX;                      // [CMAX] drag fraction e of each cell (ring cells: drho)
    T *UX = D + CMAX;                         // [CMAX] (ring cells: emitted momentum x)
    T *UY = UX + CMAX;                        // [CMAX] (ring cells: emitted momentum y)
    T *RHO = UY + CMAX;                       // [CMAX] density deviation (local-global jobs only)
    __shared__ Slot slots[MAXSLOTS];
    __shared__ int4 hot[MAXSLOTS];            // SlotHot
    __shared__ int s_abort;
    __shared__ unsigned s_event;              // CTA step of the next velocity store of any slot

    __shared__ int s_nclass, s_csize[MAXCLASS], s_coff[MAXCLASS + 1];
    __shared__ unsigned long long s_t0;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const T hg = kc<T>(a, K_HG);
    if (tid == 0) {
        s_t0 = globaltimer();
        s_abort = 0;
        if (a.table) {      // built on the device by an earlier kernel of the same stream
            const int nc = a.table[DT_BAD] ? 0 : a.table[DT_NCLASS];
            s_nclass = nc;
            for (int c = 0; c < nc; ++c) {
                s_csize[c] = a.table[DT_SIZE + c];
                s_coff[c] = a.table[DT_OFF + c];
            }
            s_coff[nc] = a.table[DT_OFF + nc];
        } else {
            s_nclass = a.nclass;
            for (int c = 0; c < a.nclass; ++c) {
                s_csize[c] = a.class_size[c];
                s_coff[c] = a.class_off[c];
            }
            s_coff[a.nclass] = a.class_off[a.nclass];
        }
    }
    __syncthreads();

    for (int cls = 0; cls < s_nclass; ++cls) {
        const int s = s_csize[cls], s2 = s * s;
        int nslots = CMAX / s2;
        if (nslots > MAXSLOTS) nslots = MAXSLOTS;
        const int ncell = nslots * s2;

        // per-thread cell geometry for this size class, packed as slot << 12 | ly << 6 | lx
        int cgeo[CPT];
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
            const int c = tid + i * LOCAL_THREADS;
            if (c < ncell) {
                const int j = c / s2;
                const int loc = c - j * s2;
                const int ly = loc / s;
                cgeo[i] = (j << 12) | (ly << 6) | (loc - ly * s);
            } else {
                cgeo[i] = -1;
            }
        }
        __syncthreads();
        unsigned Tcta = 0;           // CTA step counter: the next step to run
        if (tid < nslots) {
            Slot sl;
            sl.job = -1;
            const int qbeg = s_coff[cls], qn = s_coff[cls + 1] - qbeg;
            int q = s_abort ? qn : atomicAdd(&a.heads[cls], 1);
            if (q < qn) {
                sl.job = a.jobs[qbeg + q];
                sl.leaf = sl.job >> 1;
                sl.drive = sl.job & 1;
                sl.x0 = a.leaves[3 * sl.leaf] - a.margin;
                sl.y0 = a.leaves[3 * sl.leaf + 1] - a.margin;
                sl.prev = 0.0;
                sl.prev_t = 0.0;
            }
            slots[tid] = sl;
            hot[tid] = make_int4(0, a.check_every, sl.job >= 0 ? 1 | (sl.drive << 1) | 4 : 0,
                                 min(a.check_every, (int)a.max_steps));
        }
        if (tid == 0) s_event = (unsigned)min(a.check_every, (int)a.max_steps);
        bool fresh = true;           // some slot was just (re)filled: set its cells up before stepping

        for (;;) {
            if (fresh) {
                // rest state (zero deviations) and the drag fraction of the cells of new jobs
                __syncthreads();
#pragma unroll
                for (int i = 0; i < CPT; ++i) {
                    const int geo = cgeo[i];
                    if (geo < 0) continue;
                    const int j = geo >> 12;
                    if (!(hot[j].z & 4)) continue;
                    const int c = tid + i * LOCAL_THREADS;
                    // patch origin may lie outside the field when oversampling: periodic wrap
                    int gx = slots[j].x0 + (geo & 63), gy = slots[j].y0 + ((geo >> 6) & 63);
                    gx = gx < 0 ? gx + a.nx : (gx >= a.nx ? gx - a.nx : gx);
                    gy = gy < 0 ? gy + a.ny : (gy >= a.ny ? gy - a.ny : gy);
                    const float kap = a.kappa[(int64_t)gy * a.nx + gx];
                    if constexpr (LG) {
                        lg_start_cell<T>(a, F, D, UX, UY, c, slots[j], geo, s, kap);
                    } else {
                        D[c] = (T)coef_e(kap, a.eps_nu);
#pragma unroll
                        for (int q = 0; q < Q; ++q) F[q * CMAX + c] = T(0);
                    }
                }
                __syncthreads();
                if constexpr (LG) {
                    // the Darcy start of the inner cells, the ring's pressures held (warm_start = 1)
                    if (a.warm && s % 8 == 0) {
                        warm_start_fresh<T, true>(a, F, D, hot, slots, s, nslots);
                        __syncthreads();
                    }
                }
                if constexpr (WARM) {
                    if (s >= WARM_MIN && s % 8 == 0) {
                        warm_start_fresh<T, false>(a, F, D, hot, slots, s, nslots);
                        __syncthreads();
                    }
                }
                if (tid < nslots) hot[tid].z &= ~4;
            }
            if (!__syncthreads_or(tid < nslots && (hot[tid].z & 1))) break;

            // ------------------------------------------------------ two steps (even, odd)
            local_step<T, TAU1, false, LG>(F, D, UX, UY, RHO, hot, cgeo, s, s2, Tcta, hg, a, tid);
            ++Tcta;
            __syncthreads();
            local_step<T, TAU1, true, LG>(F, D, UX, UY, RHO, hot, cgeo, s, s2, Tcta, hg, a, tid);
            ++Tcta;
            __syncthreads();

            // ------------------------------------- bookkeeping, only after a velocity store
            // (and every 256 steps for the wall-clock limit); s_event is uniform
            fresh = false;
            if ((int)(Tcta - s_event) <= 0 && (Tcta & 255u) != 0) continue;
            if (tid == 0 && !s_abort) {
                if (*(volatile int *)a.abort_flag) s_abort = 1;
                else if (globaltimer() - s_t0 > a.time_limit_ns) {
                    s_abort = 1;
                    atomicExch(a.abort_flag, 1);
                }
            }
            __syncthreads();
            const bool abort_now = s_abort != 0;
            for (int j = wid; j < nslots; j += LOCAL_THREADS / 32) {
                int4 h = hot[j];
                if (!(h.z & 1)) continue;
                Slot sl = slots[j];
                const bool check = (int)(Tcta - (unsigned)h.w) > 0;     // the store step has run
                if (!check && !abort_now) continue;
                // job step of the check (or, abandoned unchecked, the step reached)
                const int t = (int)((check ? (unsigned)h.w : Tcta) - (unsigned)h.x);
                int st = -1;   // -1: keep going
                double ux = 0.0, uy = 0.0, gxd = 0.0, gyd = 0.0;
                if (check) {
                    // mean over the leaf: all s2 cells, or the inner window when oversampling
                    const int m = a.margin, hi = s - m;
                    for (int c = j * s2 + lane; c < (j + 1) * s2; c += 32) {
                        const int loc = c - j * s2, ly = loc / s, lx = loc - ly * s;
                        if (m == 0 || (lx >= m && lx < hi && ly >= m && ly < hi)) {
                            ux += (double)UX[c];
                            uy += (double)UY[c];
                        }
                    }
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) {
                        ux += __shfl_xor_sync(0xffffffffu, ux, off);
                        uy += __shfl_xor_sync(0xffffffffu, uy, off);
                    }
                    const double inner = (double)(s - 2 * a.margin) * (double)(s - 2 * a.margin);
                    ux /= inner;
                    uy /= inner;
                    if constexpr (LG) {
                        // the inner window's mean density gradient by central differences, summed
                        // cell by cell, telescopes to its two edge columns (rows) and the ones beyond
                        double gxs = 0.0, gys = 0.0;
                        for (int c = j * s2 + lane; c < (j + 1) * s2; c += 32) {
                            const int loc = c - j * s2, ly = loc / s, lx = loc - ly * s;
                            const double rc = (double)RHO[c];
                            if (ly >= m && ly < hi) {
                                if (lx == hi - 1 || lx == hi) gxs += 0.5 * rc;
                                if (lx == m || lx == m - 1) gxs -= 0.5 * rc;
                            }
                            if (lx >= m && lx < hi) {
                                if (ly == hi - 1 || ly == hi) gys += 0.5 * rc;
                                if (ly == m || ly == m - 1) gys -= 0.5 * rc;
                            }
                        }
#pragma unroll
                        for (int off = 16; off > 0; off >>= 1) {
                            gxs += __shfl_xor_sync(0xffffffffu, gxs, off);
                            gys += __shfl_xor_sync(0xffffffffu, gys, off);
                        }
                        gxd = gxs / inner;
                        gyd = gys / inner;
                        if (a.lg_ring == 2) {
                            // pressure-only ring: each ring cell takes the velocity its inward
                            // neighbour stored at this check; the CTA's next step is the second
                            // after the check (checks fall on even job steps)
                            for (int c = j * s2 + lane; c < (j + 1) * s2; c += 32) {
                                const int loc = c - j * s2, ly = loc / s, lx = loc - ly * s;
                                if (!(lx == 0 || ly == 0 || lx == s - 1 || ly == s - 1)) continue;
                                const int xi = lx == 0 ? 1 : (lx == s - 1 ? s - 2 : lx);
                                const int yi = ly == 0 ? 1 : (ly == s - 1 ? s - 2 : ly);
                                const int ci = j * s2 + yi * s + xi;
                                lg_ring_momentum<T>(a, D, UX, UY, c, sl, lx, ly, (double)UX[ci], (double)UY[ci]);
                            }
                        }
                    }
                    const double cur = sl.drive == 0 ? ux : uy, cur_t = sl.drive == 0 ? uy : ux;
                    const bool regular = t == h.y;
                    if (regular) h.y += a.check_every;
                    bool settled;
                    if (LG || (WARM && s >= WARM_MIN && s % 8 == 0)) {
                        // a Darcy-started job: the whole mean velocity vector must have settled,
                        // since its transverse component can still carry the start's error after
                        // the driven one has stopped moving
                        const double dd = cur - sl.prev, dt = cur_t - sl.prev_t;
                        settled = sqrt(dd * dd + dt * dt) <=
                                  a.tol * a.check_every * sqrt(cur * cur + cur_t * cur_t);
                    } else {
                        settled = fabs(cur - sl.prev) <= a.tol * a.check_every * fabs(cur);
                    }
                    if (a.tol > 0.0 && t > a.check_every && regular && settled)
                        st = LBM_OK;
                    else if (t == (int)a.max_steps)
                        st = a.tol > 0.0 ? LBM_ENOTCONV : LBM_OK;
                    sl.prev = cur;
                    sl.prev_t = cur_t;
                    h.w = (int)((unsigned)h.x + (unsigned)min(h.y, (int)a.max_steps));
                }
                if (abort_now && st < 0) st = LBM_ETIMEOUT;
                if (lane == 0) {
                    if (st >= 0) {
                        // Eq. 17: column `drive` of K* from the mean velocity (NaN if abandoned unchecked)
                        const double kx = check ? a.nu_over_g * ux : __longlong_as_double(0x7ff8000000000000LL);
                        const double ky = check ? a.nu_over_g * uy : __longlong_as_double(0x7ff8000000000000LL);
                        if constexpr (LG) {
                            // K* needs both drives: the window means go out, K* is formed afterwards
                            double *w = a.lg_win + 4 * (2 * (int64_t)sl.leaf + sl.drive);
                            const double nan = __longlong_as_double(0x7ff8000000000000LL);
                            w[0] = check ? ux : nan;
                            w[1] = check ? uy : nan;
                            w[2] = check ? gxd : nan;
                            w[3] = check ? gyd : nan;
                        } else {
                            a.keff[4 * (int64_t)sl.leaf + (sl.drive == 0 ? 0 : 1)] = kx;
                            a.keff[4 * (int64_t)sl.leaf + (sl.drive == 0 ? 2 : 3)] = ky;
                        }
                        if (a.steps) a.steps[2 * (int64_t)sl.leaf + sl.drive] = t;
                        if (st != LBM_OK) {
                            atomicMax(&a.status[sl.leaf], st);
                            atomicMax(a.worst, st);
                        }
                        // refill the slot from this size's queue; the new job starts at the next
                        // (even) CTA step
                        const int qbeg = s_coff[cls], qn = s_coff[cls + 1] - qbeg;
                        int q = abort_now ? qn : atomicAdd(&a.heads[cls], 1);
                        if (q < qn) {
                            sl.job = a.jobs[qbeg + q];
                            sl.leaf = sl.job >> 1;
                            sl.drive = sl.job & 1;
                            sl.x0 = a.leaves[3 * sl.leaf] - a.margin;
                            sl.y0 = a.leaves[3 * sl.leaf + 1] - a.margin;
                            sl.prev = 0.0;
                            sl.prev_t = 0.0;
                            h = make_int4((int)Tcta, a.check_every, 1 | (sl.drive << 1) | 4,
                                          (int)(Tcta + (unsigned)min(a.check_every, (int)a.max_steps)));
                        } else {
                            sl.job = -1;
                            h.z = 0;
                        }
                    }
                    slots[j] = sl;
                    hot[j] = h;
                }
                __syncwarp();
            }
            __syncthreads();   // slot updates of every warp are visible before they are read
            // next event: the earliest velocity store of an active slot
            if (wid == 0) {
                unsigned best = 0xffffffffu;
                for (int j = lane; j < nslots; j += 32) {
                    const int4 h = hot[j];
                    if (h.z & 1) best = min(best, (unsigned)h.w - Tcta);
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, off));
                if (lane == 0) s_event = Tcta + best;
            }
            fresh = __syncthreads_or(tid < nslots && (hot[tid].z & 4)) != 0;
        }
    }
}

using LocalKernel = void (*)(LocalArgs);

// The solver variant for a storage type, tau (tau = 1 exactly has its own collision form) and
// the start (rest, or the Darcy state).
template <typename T>
LocalKernel local_kernel_t(bool t1, bool warm)
{
    if (warm) return t1 ? local_keff_kernel<T, true, MODE_WARM> : local_keff_kernel<T, false, MODE_WARM>;
    return t1 ? local_keff_kernel<T, true, MODE_REST> : local_keff_kernel<T, false, MODE_REST>;
}
LocalKernel local_kernel(bool f64, double tau, int warm)
{
    return f64 ? local_kernel_t<double>(tau == 1.0, warm != 0) : local_kernel_t<float>(tau == 1.0, warm != 0);
}
// local-global jobs: one more value per cell (the density deviation)
LocalKernel local_kernel_lg(bool f64, double tau)
{
    if (f64) return tau == 1.0 ? local_keff_kernel<double, true, MODE_LG> : local_keff_kernel<double, false, MODE_LG>;
    return tau == 1.0 ? local_keff_kernel<float, true, MODE_LG> : local_keff_kernel<float, false, MODE_LG>;
}
template <typename T> constexpr size_t lg_smem() { return LocalCfg<T>::SMEM + LocalCfg<T>::CMAX * sizeof(T); }

// K* of each local-global leaf from its two drives' window means (the Brinkman equation of
// Section 2 at steady state, averaged over the window): <u> = (K* / nu) <F> with
// F = G e_d - grad(drho) / (3 eps) per drive, so with U and F the 2 x 2 matrices whose columns
// are the drives, K* = nu U F^-1 (Eq. 17 when grad(drho) = 0).
// One warp per block: kuni[i] = kappa if every cell of the block's patch (the block grown by m,
// periodic) has the same kappa, else -1. Such a block's local-global K* is kappa I exactly (Darcy
// flow through a uniform medium under any boundary pressure), so it needs no local problem.
__global__ void lg_uniform_kernel(const float *kappa, int nx, int ny, int block, int m, int nbx, int64_t n,
                                  float *kuni)
{
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    const int by = (int)(w / nbx), bx = (int)(w - (int64_t)by * nbx), se = block + 2 * m;
    auto at = [&](int c) {
        const int ly = c / se, lx = c - ly * se;
        int x = bx * block - m + lx, y = by * block - m + ly;
        x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
        y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
        return kappa[(int64_t)y * nx + x];
    };
    const float k0 = at(0);
    bool same = k0 >= 0.0f;
    for (int c = lane; c < se * se && same; c += 32) same = at(c) == k0;
    same = __all_sync(0xffffffffu, same);
    if (lane == 0) kuni[w] = same ? k0 : -1.0f;
}

// Per block: a uniform patch takes K* = kappa I (status LBM_OK, no steps, window NaN). Otherwise
// K* from its two drives' window means (the Brinkman equation of Section 2 at steady state,
// averaged over the window): <u> = (K* / nu) <F> with F = G e_d - grad(drho) / (3 eps) per drive,
// so with U and F the 2 x 2 matrices whose columns are the drives, K* = nu U F^-1 (Eq. 17 when
// grad(drho) = 0). With fallback tensors (kref) such a block keeps its K*, symmetrised, only when
// its run met the tolerance, the symmetrised tensor is positive definite and the 2-norm condition
// number of F is at most LG_COND_MAX; otherwise it takes kref (counted in nfb).
constexpr double LG_COND_MAX = 10.0;
__global__ void lg_finish_kernel(int64_t n, const int *pos, const float *kuni, const double *win_h,
                                 const int32_t *status_h, const int32_t *steps_h, double nu, double g, double eps,
                                 const double *kref, double *keff, int32_t *status, int32_t *steps, double *window,
                                 int *nfb)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = pos[i];
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    if (j < 0) {
        const double k0 = kuni[i];
        keff[4 * i + 0] = k0;
        keff[4 * i + 1] = 0.0;
        keff[4 * i + 2] = 0.0;
        keff[4 * i + 3] = k0;
        status[i] = LBM_OK;
        if (steps) steps[2 * i] = steps[2 * i + 1] = 0;
        if (window)
            for (int q = 0; q < 8; ++q) window[8 * i + q] = nan;
        return;
    }
    const double *w = win_h + 8 * (int64_t)j;
    status[i] = status_h[j];
    if (steps) {
        steps[2 * i] = steps_h[2 * (int64_t)j];
        steps[2 * i + 1] = steps_h[2 * (int64_t)j + 1];
    }
    if (window)
        for (int q = 0; q < 8; ++q) window[8 * i + q] = w[q];
    const double u11 = w[0], u21 = w[1], u12 = w[4], u22 = w[5];
    const double f11 = g - w[2] / (3.0 * eps), f21 = -w[3] / (3.0 * eps);
    const double f12 = -w[6] / (3.0 * eps), f22 = g - w[7] / (3.0 * eps);
    const double det = f11 * f22 - f12 * f21;
    const double i11 = f22 / det, i12 = -f12 / det, i21 = -f21 / det, i22 = f11 / det;
    double k[4] = {nu * (u11 * i11 + u12 * i21), nu * (u11 * i12 + u12 * i22), nu * (u21 * i11 + u22 * i21),
                   nu * (u21 * i12 + u22 * i22)};
    if (kref) {
        const double sym = 0.5 * (k[1] + k[2]);
        // singular values of F from its Frobenius norm and determinant
        const double fro = f11 * f11 + f12 * f12 + f21 * f21 + f22 * f22;
        const double disc = sqrt(fmax(fro * fro - 4.0 * det * det, 0.0));
        const double smax = sqrt(0.5 * (fro + disc)), smin = sqrt(fmax(0.5 * (fro - disc), 0.0));
        const bool good = status_h[j] == LBM_OK && isfinite(k[0]) && isfinite(sym) && isfinite(k[3]) && k[0] > 0.0 &&
                          k[0] * k[3] - sym * sym > 0.0 && smin > 0.0 && smax <= LG_COND_MAX * smin;
        if (good) {
            k[1] = sym;
            k[2] = sym;
        } else {
            for (int q = 0; q < 4; ++q) k[q] = kref[4 * i + q];
            atomicAdd(nfb, 1);
        }
    }
    for (int q = 0; q < 4; ++q) keff[4 * i + q] = k[q];
}

// what the local-global variant of the solver needs beyond the plain local problems
struct LgInput {
    const float *state;   // coarse (drho, u, v) [2][3][nyc][nxc]
    int r, nxc, nyc;
    int ring;             // 1 or 2
    double *win;          // [n][2][4]
};

lbm_status local_keff_core(const lbm_params *p, const float *kappa_dev, const lbm_leaf *leaves_dev, int32_t n_leaves,
                           double g_const, double tol_rel, int64_t max_steps, int32_t check_every,
                           int32_t persistent, double *keff_dev, int32_t *status_dev, int32_t *steps_dev,
                           void *cuda_stream, double time_limit_s, const LgInput *lg)
{
    if (!p) return fail(LBM_EINVAL, "params is NULL");
    if (p->nx < 1 || p->ny < 1) return fail(LBM_EINVAL, "nx, ny must be >= 1");
    if (!std::isfinite(p->tau) || p->tau < 0.5) return fail(LBM_EINVAL, "tau must be finite and >= 0.5");
    if (!std::isfinite(p->nu) || !std::isfinite(p->eps) || p->eps < 0.0)
        return fail(LBM_EINVAL, "nu must be finite and eps finite and >= 0");
    if (n_leaves < 0) return fail(LBM_EINVAL, "n_leaves must be >= 0");
    if (!std::isfinite(g_const) || g_const == 0.0) return fail(LBM_EINVAL, "g_const must be finite and non-zero");
    if (!std::isfinite(tol_rel) || tol_rel < 0.0) return fail(LBM_EINVAL, "tol_rel must be finite and >= 0");
    if (max_steps < 1 || max_steps >= (int64_t)1 << 31) return fail(LBM_EINVAL, "max_steps must be in [1, 2^31 - 1]");
    if (check_every < 1) return fail(LBM_EINVAL, "check_every must be >= 1");
    if (p->warm_start != 0 && p->warm_start != 1) return fail(LBM_EINVAL, "warm_start must be 0 or 1");
    if (n_leaves == 0) return LBM_OK;
    if (!is_device_ptr(kappa_dev) || !is_device_ptr(leaves_dev) || !is_device_ptr(keff_dev) ||
        !is_device_ptr(status_dev) || (steps_dev && !is_device_ptr(steps_dev)))
        return fail(LBM_EINVAL, "kappa, leaves, keff, status (and steps) must be device pointers");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

#define LOC_CUDA(call)                                                                           \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            cudaGetLastError();                                                                  \
            return fail(e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s failed: %s", \
                        #call, cudaGetErrorString(e_));                                          \
        }                                                                                        \
    } while (0)

    // leaves come from the device; validate them on the host before any launch
    std::vector<lbm_leaf> lv(n_leaves);
    LOC_CUDA(cudaMemcpyAsync(lv.data(), leaves_dev, sizeof(lbm_leaf) * n_leaves, cudaMemcpyDeviceToHost, st));
    LOC_CUDA(cudaStreamSynchronize(st));
    const int m = p->margin;
    if (m < 0 || m > 32 || m >= p->nx || m >= p->ny)
        return fail(LBM_EINVAL, "margin %d outside [0, 32] or not below the field size", m);
    std::vector<int> sizes;
    for (int i = 0; i < n_leaves; ++i) {
        const lbm_leaf &L = lv[i];
        const int smax = p->storage == LBM_F64 ? 45 : 64;   // FP64 leaves hold 2048 cells per CTA
        if (L.size < 1 || L.size + 2 * m > smax)
            return fail(LBM_EINVAL, "leaf %d: size %d (+ 2 x margin %d) outside [1, %d]", i, L.size, m, smax);
        if (L.x0 < 0 || L.y0 < 0 || (int64_t)L.x0 + L.size > p->nx || (int64_t)L.y0 + L.size > p->ny)
            return fail(LBM_EINVAL, "leaf %d (%d, %d, %d) lies outside the %d x %d field", i, L.x0, L.y0, L.size,
                        p->nx, p->ny);
        sizes.push_back(L.size + 2 * m);
    }
    std::sort(sizes.begin(), sizes.end(), std::greater<int>());
    sizes.erase(std::unique(sizes.begin(), sizes.end()), sizes.end());
    if ((int)sizes.size() > MAXCLASS) return fail(LBM_EINVAL, "more than %d distinct leaf sizes", MAXCLASS);

    const double nu = p->nu < 0.0 ? (p->tau - 0.5) / 3.0 : p->nu;
    LocalArgs a{};
    a.kappa = kappa_dev;
    a.nx = p->nx;
    a.ny = p->ny;
    a.margin = m;
    a.leaves = reinterpret_cast<const int *>(leaves_dev);
    a.omega = (1.0 / p->tau);
    a.two_tau = (2.0 * p->tau);
    a.omt = (1.0 - 2.0 * p->tau);
    a.half_eps = (0.5 * p->eps);
    a.gmag = g_const;
    cell_consts(a);
    a.eps_nu = p->eps * nu;
    a.nu_over_g = nu / g_const;
    a.warm = p->warm_start;
    a.warm_rho = 3.0 * p->eps * g_const;
    a.warm_u = g_const / nu;
    if (lg) {
        a.lg_state = lg->state;
        a.lg_r = lg->r;
        a.lg_nxc = lg->nxc;
        a.lg_nyc = lg->nyc;
        a.lg_ring = lg->ring;
        a.lg_win = lg->win;
    }
    a.tol = tol_rel;
    a.check_every = check_every;
    a.max_steps = max_steps;
    a.keff = keff_dev;
    a.status = status_dev;
    a.steps = steps_dev;
    a.time_limit_ns = (unsigned long long)(time_limit_s * 1e9);

    // job lists: persistent -> grouped by size (largest first); per-leaf -> leaf order
    std::vector<int> jobs;
    jobs.reserve(2 * (size_t)n_leaves);
    std::vector<int> off;
    if (persistent) {
        for (int s : sizes) {
            off.push_back((int)jobs.size());
            for (int i = 0; i < n_leaves; ++i)
                if (lv[i].size + 2 * m == s) {
                    jobs.push_back(2 * i);
                    jobs.push_back(2 * i + 1);
                }
        }
        off.push_back((int)jobs.size());
    } else {
        for (int i = 0; i < n_leaves; ++i) {
            jobs.push_back(2 * i);
            jobs.push_back(2 * i + 1);
        }
    }
    const int nheads = persistent ? (int)sizes.size() : n_leaves;

    int *d_jobs = nullptr, *d_heads = nullptr, *d_flags = nullptr;
    auto cleanup = [&]() {
        cudaFree(d_jobs);
        cudaFree(d_heads);
        cudaFree(d_flags);
        cudaGetLastError();
    };
#define LOC_CUDA2(call)                                                                          \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            cudaGetLastError();                                                                  \
            cleanup();                                                                           \
            return fail(e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s failed: %s", \
                        #call, cudaGetErrorString(e_));                                          \
        }                                                                                        \
    } while (0)
    LOC_CUDA2(cudaMalloc(&d_jobs, sizeof(int) * jobs.size()));
    LOC_CUDA2(cudaMalloc(&d_heads, sizeof(int) * nheads));
    LOC_CUDA2(cudaMalloc(&d_flags, sizeof(int) * 2));
    LOC_CUDA2(cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(int) * jobs.size(), cudaMemcpyHostToDevice, st));
    LOC_CUDA2(cudaMemsetAsync(d_heads, 0, sizeof(int) * nheads, st));
    LOC_CUDA2(cudaMemsetAsync(d_flags, 0, sizeof(int) * 2, st));
    LOC_CUDA2(cudaMemsetAsync(status_dev, 0, sizeof(int32_t) * n_leaves, st));
    if (steps_dev) LOC_CUDA2(cudaMemsetAsync(steps_dev, 0, sizeof(int32_t) * 2 * n_leaves, st));
    a.jobs = d_jobs;
    a.worst = d_flags;
    a.abort_flag = d_flags + 1;

    const bool f64 = p->storage == LBM_F64;
    const LocalKernel kern = lg ? local_kernel_lg(f64, p->tau) : local_kernel(f64, p->tau, p->warm_start);
    const size_t smem = lg ? (f64 ? lg_smem<double>() : lg_smem<float>())
                           : f64 ? LocalCfg<double>::SMEM : LocalCfg<float>::SMEM;
    LOC_CUDA2(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0;
    LOC_CUDA2(cudaGetDevice(&dev));
    if (persistent) {
        a.nclass = (int)sizes.size();
        for (int c = 0; c < a.nclass; ++c) {
            a.class_off[c] = off[c];
            a.class_size[c] = sizes[c];
        }
        a.class_off[a.nclass] = off[a.nclass];
        a.heads = d_heads;
        int blocks = sm_count(dev);
        const int64_t max_useful = (int64_t)jobs.size();
        if (blocks > max_useful) blocks = (int)max_useful;
        kern<<<blocks, LOCAL_THREADS, smem, st>>>(a);
        LOC_CUDA2(cudaGetLastError());
        count_launches(1);
    } else {
        a.nclass = 1;
        for (int i = 0; i < n_leaves; ++i) {
            a.class_off[0] = 2 * i;
            a.class_off[1] = 2 * i + 2;
            a.class_size[0] = lv[i].size + 2 * m;
            a.heads = d_heads + i;
            kern<<<1, LOCAL_THREADS, smem, st>>>(a);
            LOC_CUDA2(cudaGetLastError());
        }
        count_launches(n_leaves);
    }
    int flags[2] = {0, 0};
    LOC_CUDA2(cudaMemcpyAsync(flags, d_flags, sizeof flags, cudaMemcpyDeviceToHost, st));
    LOC_CUDA2(cudaStreamSynchronize(st));
    cleanup();
    if (flags[1] || flags[0] == LBM_ETIMEOUT)
        return fail(LBM_ETIMEOUT, "local problems exceeded the %.3g s limit; unfinished leaves carry LBM_ETIMEOUT",
                    time_limit_s);
    if (flags[0] == LBM_ENOTCONV)
        return fail(LBM_ENOTCONV, "some leaves did not meet the tolerance within max_steps (status per leaf)");
    return LBM_OK;
#undef LOC_CUDA
#undef LOC_CUDA2
}

}  // namespace

lbm_status local_keff_impl(const lbm_params *p, const float *kappa_dev, const lbm_leaf *leaves_dev, int32_t n_leaves,
                           double g_const, double tol_rel, int64_t max_steps, int32_t check_every,
                           int32_t persistent, double *keff_dev, int32_t *status_dev, int32_t *steps_dev,
                           void *cuda_stream, double time_limit_s)
{
    return local_keff_core(p, kappa_dev, leaves_dev, n_leaves, g_const, tol_rel, max_steps, check_every, persistent,
                           keff_dev, status_dev, steps_dev, cuda_stream, time_limit_s, nullptr);
}

lbm_status local_keff_lg_impl(const lbm_params *p, const float *kappa_dev, int32_t block, const float *coarse_dev,
                              double g_const, double tol_rel, int64_t max_steps, int32_t check_every, int32_t ring,
                              const double *keff_fallback_dev, double *keff_dev, int32_t *status_dev,
                              int32_t *steps_dev, double *window_dev, int32_t *n_fallback, void *cuda_stream,
                              double time_limit_s)
{
    if (n_fallback) *n_fallback = 0;
    if (!p) return fail(LBM_EINVAL, "params is NULL");
    if (p->nx < 1 || p->ny < 1) return fail(LBM_EINVAL, "nx, ny must be >= 1");
    if (block < 1 || p->nx % block || p->ny % block)
        return fail(LBM_EINVAL, "nx, ny must be multiples of block %d", block);
    const int m = p->margin;
    const int smax = p->storage == LBM_F64 ? 45 : 64;   // FP64 patches hold 2048 cells per CTA
    if (m < 2 || block + 2 * m > smax)
        return fail(LBM_EINVAL, "local-global patches need margin >= 2 and block + 2 x margin <= %d (got %d, %d)",
                    smax, block, m);
    if (m >= p->nx || m >= p->ny) return fail(LBM_EINVAL, "margin %d is not below the field size", m);
    if (p->warm_start != 0 && p->warm_start != 1) return fail(LBM_EINVAL, "warm_start must be 0 or 1");
    if (!(p->eps > 0.0) || !std::isfinite(p->eps)) return fail(LBM_EINVAL, "eps must be finite and > 0");
    if (ring != 1 && ring != 2) return fail(LBM_EINVAL, "ring must be 1 (state held) or 2 (pressure only)");
    if (check_every < 2 || check_every % 2) return fail(LBM_EINVAL, "local-global checks need an even check_every");
    if (!coarse_dev || !is_device_ptr(coarse_dev)) return fail(LBM_EINVAL, "coarse_dev must be a device pointer");
    if (keff_fallback_dev && !is_device_ptr(keff_fallback_dev))
        return fail(LBM_EINVAL, "keff_fallback_dev must be a device pointer");
    if (window_dev && !is_device_ptr(window_dev)) return fail(LBM_EINVAL, "window_dev must be a device pointer");
    if (!keff_dev || !status_dev || !is_device_ptr(keff_dev) || !is_device_ptr(status_dev) ||
        (steps_dev && !is_device_ptr(steps_dev)))
        return fail(LBM_EINVAL, "keff, status (and steps) must be device pointers");
    const int nbx = p->nx / block, nby = p->ny / block;
    const int64_t n = (int64_t)nbx * nby;
    if (n > INT32_MAX / 2) return fail(LBM_EINVAL, "too many blocks");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    lbm_leaf *d_leaves = nullptr;
    double *d_win = nullptr;
    int *d_nfb = nullptr, *d_pos = nullptr;
    int32_t *d_status = nullptr, *d_steps = nullptr;
    float *d_kuni = nullptr;
    auto release = [&]() {
        cudaFree(d_leaves);
        cudaFree(d_win);
        cudaFree(d_nfb);
        cudaFree(d_pos);
        cudaFree(d_status);
        cudaFree(d_steps);
        cudaFree(d_kuni);
        cudaGetLastError();
    };
#define LG_CUDA(call)                                                                            \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            release();                                                                           \
            return fail(e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s failed: %s", \
                        #call, cudaGetErrorString(e_));                                          \
        }                                                                                        \
    } while (0)
    // blocks whose whole patch is uniform need no local problem
    LG_CUDA(cudaMalloc(&d_kuni, sizeof(float) * n));
    lg_uniform_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(kappa_dev, p->nx, p->ny, block, m, nbx, n,
                                                                         d_kuni);
    LG_CUDA(cudaGetLastError());
    count_launches(1);
    std::vector<float> kuni((size_t)n);
    LG_CUDA(cudaMemcpyAsync(kuni.data(), d_kuni, sizeof(float) * n, cudaMemcpyDeviceToHost, st));
    LG_CUDA(cudaStreamSynchronize(st));
    std::vector<lbm_leaf> lv;
    std::vector<int> pos((size_t)n, -1);
    for (int64_t i = 0; i < n; ++i)
        if (!(kuni[i] >= 0.0f)) {
            pos[i] = (int)lv.size();
            const int by = (int)(i / nbx), bx = (int)(i - (int64_t)by * nbx);
            lv.push_back(lbm_leaf{bx * block, by * block, block});
        }
    const int64_t nh = (int64_t)lv.size();
    LG_CUDA(cudaMalloc(&d_pos, sizeof(int) * n));
    LG_CUDA(cudaMalloc(&d_nfb, sizeof(int)));
    LG_CUDA(cudaMemsetAsync(d_nfb, 0, sizeof(int), st));
    LG_CUDA(cudaMemcpyAsync(d_pos, pos.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    const int64_t nal = nh > 0 ? nh : 1;
    LG_CUDA(cudaMalloc(&d_leaves, sizeof(lbm_leaf) * nal));
    LG_CUDA(cudaMalloc(&d_win, sizeof(double) * 8 * nal));
    LG_CUDA(cudaMalloc(&d_status, sizeof(int32_t) * nal));
    LG_CUDA(cudaMalloc(&d_steps, sizeof(int32_t) * 2 * nal));
    lbm_status s = LBM_OK;
    if (nh > 0) {
        LG_CUDA(cudaMemcpyAsync(d_leaves, lv.data(), sizeof(lbm_leaf) * nh, cudaMemcpyHostToDevice, st));
        LgInput lg{coarse_dev, block, nbx, nby, ring, d_win};
        s = local_keff_core(p, kappa_dev, d_leaves, (int32_t)nh, g_const, tol_rel, max_steps, check_every, 1, keff_dev,
                            d_status, d_steps, cuda_stream, time_limit_s, &lg);
    }
    if (s == LBM_OK || s == LBM_ENOTCONV || s == LBM_ETIMEOUT) {
        const double nu = p->nu < 0.0 ? (p->tau - 0.5) / 3.0 : p->nu;
        lg_finish_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, d_pos, d_kuni, d_win, d_status, d_steps, nu,
                                                                      g_const, p->eps, keff_fallback_dev, keff_dev,
                                                                      status_dev, steps_dev, window_dev, d_nfb);
        LG_CUDA(cudaGetLastError());
        count_launches(1);
        int nfb = 0;
        LG_CUDA(cudaMemcpyAsync(&nfb, d_nfb, sizeof(int), cudaMemcpyDeviceToHost, st));
        LG_CUDA(cudaStreamSynchronize(st));
        if (n_fallback) *n_fallback = nfb;
    }
    release();
    return s;
#undef LG_CUDA
}

lbm_status launch_local_from_table(const lbm_params *p, const float *kappa_dev, const lbm_leaf *leaves_dev,
                                   const int *jobs, int *table, double g_const, double tol_rel, int64_t max_steps,
                                   int32_t check_every, double *keff_dev, int32_t *status_dev, int32_t *steps_dev,
                                   cudaStream_t st, double time_limit_s)
{
    // parameters were validated by the caller (lbm_surrogate_keff)
    const double nu = p->nu < 0.0 ? (p->tau - 0.5) / 3.0 : p->nu;
    LocalArgs a{};
    a.kappa = kappa_dev;
    a.nx = p->nx;
    a.ny = p->ny;
    a.margin = p->margin;
    a.leaves = reinterpret_cast<const int *>(leaves_dev);
    a.jobs = jobs;
    a.table = table;
    a.heads = table + DT_HEADS;
    a.omega = (1.0 / p->tau);
    a.two_tau = (2.0 * p->tau);
    a.omt = (1.0 - 2.0 * p->tau);
    a.half_eps = (0.5 * p->eps);
    a.gmag = g_const;
    cell_consts(a);
    a.eps_nu = p->eps * nu;
    a.nu_over_g = nu / g_const;
    a.warm = p->warm_start;
    a.warm_rho = 3.0 * p->eps * g_const;
    a.warm_u = g_const / nu;
    a.tol = tol_rel;
    a.check_every = check_every;
    a.max_steps = max_steps;
    a.keff = keff_dev;
    a.status = status_dev;
    a.steps = steps_dev;
    a.worst = table + DT_WORST;
    a.abort_flag = table + DT_ABORT;
    a.time_limit_ns = (unsigned long long)(time_limit_s * 1e9);
    const bool f64 = p->storage == LBM_F64;
    const LocalKernel kern = local_kernel(f64, p->tau, p->warm_start);
    const size_t smem = f64 ? LocalCfg<double>::SMEM : LocalCfg<float>::SMEM;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ECUDA, "local solver set-up: %s", cudaGetErrorString(e));
    }
    // one CTA per SM; CTAs of an empty table find no class and return at once
    kern<<<sm_count(dev), LOCAL_THREADS, smem, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LBM_ECUDA, "local solver launch: %s", cudaGetErrorString(e));
    count_launches(1);
    return LBM_OK;
}

}  // namespace lbm

namespace {
double g_time_limit_s = 600.0;
}

extern "C" {

lbm_status lbm_local_keff_batch(const lbm_params *p, const float *kappa_dev, const lbm_leaf *leaves_dev,
                                int32_t n_leaves, double g_const, double tol_rel, int64_t max_steps,
                                int32_t check_every, int32_t persistent, double *keff_dev, int32_t *status_dev,
                                int32_t *steps_dev, void *cuda_stream)
{
    return lbm::local_keff_impl(p, kappa_dev, leaves_dev, n_leaves, g_const, tol_rel, max_steps, check_every,
                                persistent, keff_dev, status_dev, steps_dev, cuda_stream, g_time_limit_s);
}

lbm_status lbm_local_keff_lg(const lbm_params *p, const float *kappa_dev, int32_t block, const float *coarse_dev,
                             double g_const, double tol_rel, int64_t max_steps, int32_t check_every, int32_t ring,
                             const double *keff_fallback_dev, double *keff_dev, int32_t *status_dev,
                             int32_t *steps_dev, double *window_dev, int32_t *n_fallback, void *cuda_stream)
{
    return lbm::local_keff_lg_impl(p, kappa_dev, block, coarse_dev, g_const, tol_rel, max_steps, check_every, ring,
                                   keff_fallback_dev, keff_dev, status_dev, steps_dev, window_dev, n_fallback,
                                   cuda_stream, g_time_limit_s);
}

lbm_status lbm_set_time_limit(double seconds)
{
    if (!(seconds > 0.0) || !std::isfinite(seconds))
        return lbm::fail(LBM_EINVAL, "time limit must be finite and > 0");
    g_time_limit_s = seconds;
    return LBM_OK;
}

}  // extern "C"

namespace lbm {
double local_time_limit() { return g_time_limit_s; }
}  // namespace lbm

// ---------------------------------------------------------------------------
// Allocation-free variant of the batched local problems.
//
// For callers that must not allocate device memory themselves or through the
// library: code running where cudaMalloc is not allowed or not wanted (inside
// a host that owns a fixed memory pool, under a strict memory budget, or next
// to an allocator that must not be bypassed). The work queue, the per-size
// class table and the status flags live in the file-scope device array below
// instead of cudaMalloc'd scratch. The array holds at most NOALLOC_MAX_LEAVES
// leaves (1 MiB plus a small header); every GPU that loads this library keeps
// it until the process exits. Its device address is looked up with
// cudaGetSymbolAddress once per device, by the first call on that device with
// the device current. Every call also reads the class table and the status flags
// back to the host and synchronises the stream before it returns. All calls
// share the array and it keeps the last call's contents, so each call clears
// what must start at zero; calls that overlap on the GPU (different streams or
// threads) race on it. storage = LBM_F64 runs the FP64 solver (leaves up to 45
// cells), any other storage the FP32 one, as in lbm_local_keff_batch.
// ---------------------------------------------------------------------------
namespace lbm {
namespace {

constexpr int NOALLOC_MAX_LEAVES = 131072;
constexpr int NA_COUNTS = 0;                  // [65] leaves per size
constexpr int NA_CURSOR = 65;                 // [65] scatter cursors per size
constexpr int NA_HEADS = 130;                 // [64] queue heads per class
constexpr int NA_FLAGS = 194;                 // [4]  bad-leaf flag, worst status, abort flag, spare
constexpr int NA_TABLE = 198;                 // [1 + 64 + 65] nclass, class_size[], class_off[]
constexpr int NA_HEADER = 328;                // ints before the job list (keeps it 32-byte aligned)
constexpr int NA_JOBS = NA_HEADER;            // [2 * NOALLOC_MAX_LEAVES]
constexpr int NA_TOTAL = NA_JOBS + 2 * NOALLOC_MAX_LEAVES;

static __device__ __align__(256) int g_noalloc_scratch[NA_TOTAL];

std::atomic<int *> g_noalloc_ptr[64];   // device address of the array, per device

// smax: the largest leaf the solver's shared memory holds (64 in FP32, 45 in FP64)
__global__ void noalloc_count_kernel(const int *leaves, int n, int nx, int ny, int smax, int *scr)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int x0 = leaves[3 * i], y0 = leaves[3 * i + 1], s = leaves[3 * i + 2];
        if (s < 1 || s > smax || x0 < 0 || y0 < 0 || (long long)x0 + s > nx || (long long)y0 + s > ny) {
            atomicOr(&scr[NA_FLAGS], 1);
            continue;
        }
        atomicAdd(&scr[NA_COUNTS + s], 1);
    }
}

// one thread: classes in descending size, offsets of their job ranges
__global__ void noalloc_table_kernel(int *scr)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int nclass = 0, off = 0;
    for (int s = 64; s >= 1; --s) {
        const int c = scr[NA_COUNTS + s];
        if (c == 0) continue;
        scr[NA_TABLE + 1 + nclass] = s;
        scr[NA_TABLE + 65 + nclass] = off;
        scr[NA_CURSOR + s] = off;
        off += 2 * c;
        ++nclass;
    }
    scr[NA_TABLE + 65 + nclass] = off;
    scr[NA_TABLE] = nclass;
}

__global__ void noalloc_scatter_kernel(const int *leaves, int n, int *scr)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int s = leaves[3 * i + 2];
        const int pos = atomicAdd(&scr[NA_CURSOR + s], 2);
        scr[NA_JOBS + pos] = 2 * i;
        scr[NA_JOBS + pos + 1] = 2 * i + 1;
    }
}

}  // namespace
}  // namespace lbm

extern "C" lbm_status lbm_local_keff_batch_noalloc(const lbm_params *p, const float *kappa_dev,
                                                   const lbm_leaf *leaves_dev, int32_t n_leaves, double g_const,
                                                   double tol_rel, int64_t max_steps, int32_t check_every,
                                                   double *keff_dev, int32_t *status_dev, int32_t *steps_dev,
                                                   void *cuda_stream)
{
    using namespace lbm;
    if (!p) return fail(LBM_EINVAL, "params is NULL");
    if (p->nx < 1 || p->ny < 1) return fail(LBM_EINVAL, "nx, ny must be >= 1");
    if (!std::isfinite(p->tau) || p->tau < 0.5) return fail(LBM_EINVAL, "tau must be finite and >= 0.5");
    if (!std::isfinite(p->nu) || !std::isfinite(p->eps) || p->eps < 0.0)
        return fail(LBM_EINVAL, "nu must be finite and eps finite and >= 0");
    if (n_leaves < 0) return fail(LBM_EINVAL, "n_leaves must be >= 0");
    if (p->margin != 0) return fail(LBM_EINVAL, "the allocation-free entry point solves plain local problems (margin 0)");
    if (n_leaves > NOALLOC_MAX_LEAVES)
        return fail(LBM_EINVAL, "n_leaves %d exceeds the %d leaves the static scratch holds", n_leaves,
                    NOALLOC_MAX_LEAVES);
    if (!std::isfinite(g_const) || g_const == 0.0) return fail(LBM_EINVAL, "g_const must be finite and non-zero");
    if (!std::isfinite(tol_rel) || tol_rel < 0.0) return fail(LBM_EINVAL, "tol_rel must be finite and >= 0");
    if (max_steps < 1 || max_steps >= (int64_t)1 << 31) return fail(LBM_EINVAL, "max_steps must be in [1, 2^31 - 1]");
    if (check_every < 1) return fail(LBM_EINVAL, "check_every must be >= 1");
    if (p->warm_start != 0 && p->warm_start != 1) return fail(LBM_EINVAL, "warm_start must be 0 or 1");
    if (n_leaves == 0) return LBM_OK;
    if (!is_device_ptr(kappa_dev) || !is_device_ptr(leaves_dev) || !is_device_ptr(keff_dev) ||
        !is_device_ptr(status_dev) || (steps_dev && !is_device_ptr(steps_dev)))
        return fail(LBM_EINVAL, "kappa, leaves, keff, status (and steps) must be device pointers");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return fail(LBM_ECUDA, "no usable current device");
    }
    if (!g_noalloc_ptr[dev].load()) {
        // set-up, once per device, with that device current: the host-side name of a
        // __device__ array is not its device address, so ask the runtime for it
        int *ptr = nullptr;
        e = cudaGetSymbolAddress((void **)&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return fail(LBM_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
        }
        g_noalloc_ptr[dev].store(ptr);
    }
    int *scr = g_noalloc_ptr[dev].load();
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
#define NA_CUDA(call)                                                                            \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            cudaGetLastError();                                                                  \
            return fail(LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));              \
        }                                                                                        \
    } while (0)
    // the array keeps the previous call's contents: clear the header (counts, cursors,
    // heads, flags, class table) and the caller's status / steps outputs
    NA_CUDA(cudaMemsetAsync(scr, 0, sizeof(int) * NA_HEADER, st));
    NA_CUDA(cudaMemsetAsync(status_dev, 0, sizeof(int32_t) * n_leaves, st));
    if (steps_dev) NA_CUDA(cudaMemsetAsync(steps_dev, 0, sizeof(int32_t) * 2 * n_leaves, st));
    const int *lv = reinterpret_cast<const int *>(leaves_dev);
    const int nb = (n_leaves + 255) / 256 < 1024 ? (n_leaves + 255) / 256 : 1024;
    const bool f64 = p->storage == LBM_F64;           // the FP64 solver, as lbm_local_keff_batch
    const int smax = f64 ? 45 : 64;
    noalloc_count_kernel<<<nb, 256, 0, st>>>(lv, n_leaves, p->nx, p->ny, smax, scr);
    noalloc_table_kernel<<<1, 32, 0, st>>>(scr);
    NA_CUDA(cudaGetLastError());
    int head[NA_HEADER];
    NA_CUDA(cudaMemcpyAsync(head, scr, sizeof head, cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaStreamSynchronize(st));
    count_launches(2);
    if (head[NA_FLAGS])
        return fail(LBM_EINVAL, "a leaf has a size outside [1, %d] or lies outside the field", smax);
    noalloc_scatter_kernel<<<nb, 256, 0, st>>>(lv, n_leaves, scr);
    NA_CUDA(cudaGetLastError());
    count_launches(1);

    const double nu = p->nu < 0.0 ? (p->tau - 0.5) / 3.0 : p->nu;
    LocalArgs a{};
    a.kappa = kappa_dev;
    a.nx = p->nx;
    a.ny = p->ny;
    a.margin = 0;
    a.leaves = lv;
    a.jobs = scr + NA_JOBS;
    a.nclass = head[NA_TABLE];
    for (int c = 0; c < a.nclass; ++c) {
        a.class_size[c] = head[NA_TABLE + 1 + c];
        a.class_off[c] = head[NA_TABLE + 65 + c];
    }
    a.class_off[a.nclass] = head[NA_TABLE + 65 + a.nclass];
    a.heads = scr + NA_HEADS;
    a.omega = (1.0 / p->tau);
    a.two_tau = (2.0 * p->tau);
    a.omt = (1.0 - 2.0 * p->tau);
    a.half_eps = (0.5 * p->eps);
    a.gmag = g_const;
    cell_consts(a);
    a.eps_nu = p->eps * nu;
    a.nu_over_g = nu / g_const;
    a.warm = p->warm_start;
    a.warm_rho = 3.0 * p->eps * g_const;
    a.warm_u = g_const / nu;
    a.tol = tol_rel;
    a.check_every = check_every;
    a.max_steps = max_steps;
    a.keff = keff_dev;
    a.status = status_dev;
    a.steps = steps_dev;
    a.worst = scr + NA_FLAGS + 1;
    a.abort_flag = scr + NA_FLAGS + 2;
    a.time_limit_ns = (unsigned long long)(g_time_limit_s * 1e9);
    const LocalKernel kern = local_kernel(f64, p->tau, p->warm_start);
    const size_t smem = f64 ? LocalCfg<double>::SMEM : LocalCfg<float>::SMEM;
    NA_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int blocks = sm_count(dev);
    if (blocks > 2 * n_leaves) blocks = 2 * n_leaves;
    kern<<<blocks, LOCAL_THREADS, smem, st>>>(a);
    NA_CUDA(cudaGetLastError());
    count_launches(1);
    int flags[2] = {0, 0};
    NA_CUDA(cudaMemcpyAsync(flags, scr + NA_FLAGS + 1, sizeof flags, cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaStreamSynchronize(st));
#undef NA_CUDA
    if (flags[1] || flags[0] == LBM_ETIMEOUT)
        return fail(LBM_ETIMEOUT, "local problems exceeded the time limit; unfinished leaves carry LBM_ETIMEOUT");
    if (flags[0] == LBM_ENOTCONV)
        return fail(LBM_ENOTCONV, "some leaves did not meet the tolerance within max_steps (status per leaf)");
    return LBM_OK;
}
