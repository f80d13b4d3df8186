/*
 * lbm.h -- C ABI of the GB300 upscaled lattice Boltzmann library (liblbm.so).
 *
 * The library steps the D2Q9 simplified Shan-Chen lattice Boltzmann scheme for
 * Brinkman/Darcy flow in heterogeneous porous media (Li & Brown, "Upscaled
 * Lattice Boltzmann Method for Simulations of Flows in Heterogeneous Porous
 * Media", Section 2.2), solves the local problems that give the effective
 * permeability tensor K* of each subdomain (Section 3, Eq. 17), and runs the
 * coarse upscaled simulation with K* (Section 3, Eq. 18; Section 4.3).
 *
 * Units. Everything is in lattice units: dx = dt = 1, c = 1, c_s^2 = 1/3 and
 * rho0 = 1. tau sets nu_eff = (tau - 1/2) / 3 (Section 2.1). nu is the Darcy
 * viscosity of the drag term (Eq. 5), independent of nu_eff; kappa is the
 * permeability in cells^2; G is the body force per unit mass.
 *
 * Conventions shared by every call.
 *   - Arrays are row-major [ny][nx] (x fastest). Array arguments named *_dev
 *     are DEVICE pointers owned by the caller; the library never frees them.
 *     Passing a host pointer where a device pointer is expected returns
 *     LBM_EINVAL. Only the opaque handles (lbm_grid) own device memory.
 *   - `cuda_stream` is a cudaStream_t (NULL: the legacy default stream). Work is
 *     ordered on that stream; every call synchronises the stream before it
 *     returns, so outputs are ready when it returns LBM_OK.
 *   - Every call returns an lbm_status. On failure lbm_last_error() returns a
 *     thread-local message. LBM_EINVAL is returned before any device work when
 *     the arguments can be checked on the host; device-resident inputs (kappa)
 *     are validated by a kernel and reported as LBM_EINVAL as well.
 *   - The library uses one GPU: the current CUDA device at the call.
 */
#ifndef LBM_H
#define LBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,     /* invalid argument (nothing was launched or changed)          */
    LBM_ENOMEM = 2,     /* device or pinned host allocation failed                     */
    LBM_ECUDA = 3,      /* a CUDA runtime call failed (message has the CUDA error)     */
    LBM_ENOTCONV = 4,   /* stopping tolerance not met within max_steps (results valid) */
    LBM_ETIMEOUT = 5    /* a bounded device-side wait gave up (results not valid)      */
} lbm_status;

typedef enum {
    LBM_F32 = 0,        /* distributions stored as FP32 deviations g = f - w rho0     */
    LBM_F16 = 1,        /* FP16 deviations scaled by a power of two S, FP32 arithmetic */
    LBM_F64 = 2         /* FP64 deviations and FP64 arithmetic                        */
} lbm_storage;

typedef enum {
    LBM_BC_PERIODIC = 0,  /* periodic in x and y (the paper's choice, Section 3)       */
    LBM_BC_WALLS_Y = 1    /* periodic in x; half-way bounce-back walls at y = -1/2 and
                             y = ny - 1/2 (no-slip channel walls)                      */
} lbm_bc;

typedef struct {
    int32_t nx, ny;       /* lattice size in cells, each >= 1                          */
    double  tau;          /* BGK relaxation time, tau >= 1/2; nu_eff = (tau - 1/2)/3    */
    double  nu;           /* Darcy viscosity in f_m = -(eps nu / kappa) u + eps G (Eq. 5);
                             a negative value selects nu = nu_eff                       */
    double  eps;          /* porosity epsilon, >= 0                                     */
    double  gx, gy;       /* constant body force, used when no force field is given     */
    int32_t bc;           /* lbm_bc                                                     */
    int32_t storage;      /* lbm_storage                                                */
    double  scale;        /* LBM_F16 only: power-of-two storage scale S; 0 picks S from
                             the largest finite kappa, |G| and nu                        */
    int32_t force_model;  /* 0: simplified Shan-Chen scheme (Section 2.2, Eqs. 13-16);
                             1: Guo scheme (Section 2.1, Eqs. 1-6: u_eq = u and the
                             forcing term F_a of Eq. 4). With the linear equilibrium of
                             Eq. 2 both give the same update up to rounding.          */
    int32_t margin;       /* local problems (lbm_local_keff_batch, lbm_upscale): oversampling
                             margin m >= 0 in cells, the treatment the Conclusions name for
                             channelised, high-contrast media. Each leaf's problem is solved
                             on the leaf grown by m cells on every side (taken from the field
                             with periodic wrap) with periodic closure, and the stop test and
                             Eq. 17 average the inner leaf only. 0 is the plain local problem
                             of Section 3. Ignored by the grid calls.                    */
    int32_t warm_start;   /* local problems: 0 starts every run from rest (Section 3 is silent
                             on the start; rest is the reading used throughout); 1 starts a
                             run on a patch of 16 cells or more from the patch's finite-volume
                             Darcy state instead: the pressure and the cell velocities of
                             Darcy flow through the same patch under the same drive (harmonic
                             face permeabilities, periodic), solved in shared memory when the
                             run begins, as g_a = w_a (drho + 3 e_a . j) with drho = 3 eps G p
                             and j = rho u. The steady state is the same. The stop test of
                             such a run takes the relative change of the whole mean velocity
                             vector, not of its driven component only (from a start near the
                             steady state the transverse component can still be moving when
                             the driven one has stopped). The slow diffusive start is skipped,
                             so runs stop sooner, and K* differs from the rest start only
                             within the stop test's band. With lbm_local_keff_lg: the
                             inner cells start from the Darcy flow with the ring's
                             pressures held. Ignored by the grid calls.                   */
} lbm_params;

/* Thread-local description of the last failure of any call in this thread. */
const char *lbm_last_error(void);

/* Number of kernels this library has launched in this process (graph launches
 * count each kernel node). Lets a caller check that the device path ran. */
int64_t lbm_launch_count(void);

/* ------------------------------------------------------------------ grids ---
 * A grid is one lattice with its permeability and force, stepped by the
 * simplified Shan-Chen scheme of Section 2.2:
 *   rho = sum_a f_a, j = sum_a e_a f_a,
 *   u = (j + eps rho G / 2) / (rho (1 + eps nu / (2 kappa)))      (Eq. 6, Eq. 15)
 *   u_eq = 2 tau u + (1 - 2 tau) j / rho                            (Eq. 16)
 *   f_eq = w_a rho (1 + e_a . u_eq / c_s^2)                        (Eq. 2)
 *   f_a(x + e_a, t + 1) = f_a + (f_eq - f_a) / tau                  (Eq. 13)
 * starting from rest (f = w_a rho0). */
typedef struct lbm_grid lbm_grid;

/* Creates a grid. kappa_dev: float [ny][nx] permeability, each >= 0 (0 blocks the
 * cell completely, +inf means no drag); NaN or negative values give LBM_EINVAL.
 * g_field_dev: NULL for the constant (gx, gy), else float [2][ny][nx] (x plane,
 * then y plane). Both are read during the call only (the grid keeps its own
 * derived copy). On success *out owns two distribution buffers of
 * 9 * nx * ny elements of the storage type plus per-cell coefficients. */
lbm_status lbm_grid_create(const lbm_params *p, const float *kappa_dev, const float *g_field_dev,
                           void *cuda_stream, lbm_grid **out);

/* Frees a grid and everything it owns. NULL is accepted. */
lbm_status lbm_grid_destroy(lbm_grid *g);

/* Advances the grid by up to max_steps time steps (fused pull-stream + collide,
 * replayed as CUDA graphs). With check_every = k > 0, after every step count t
 * that is a multiple of k (counted from grid creation) the residual
 *   r = max_x,i |u_i^t - u_i^(t-1)| / max_x,i |u_i^t|
 * is computed in FP64; when tol_rel > 0 and r <= tol_rel the call stops and
 * returns LBM_OK. tol_rel <= 0 runs exactly max_steps and returns LBM_OK.
 * If tol_rel > 0 and the test never passes, returns LBM_ENOTCONV (the state is
 * valid). steps_done (may be NULL) receives the steps taken by this call;
 * residual (may be NULL) the last residual computed in this call, or -1. */
lbm_status lbm_step(lbm_grid *g, int64_t max_steps, double tol_rel, int32_t check_every,
                    int64_t *steps_done, double *residual);

/* Density and flow velocity (Eq. 15) of the current state into caller-owned
 * float [ny][nx] device arrays; any of the three may be NULL. */
lbm_status lbm_get_fields(lbm_grid *g, float *rho_dev, float *u_dev, float *v_dev);

/* Volume average of the flow velocity over all cells (Section 3), reduced in
 * FP64 in a fixed order (bitwise reproducible). out_mean_uv is HOST memory. */
lbm_status lbm_mean_velocity(lbm_grid *g, double out_mean_uv[2]);

/* Total steps taken since creation (host value). */
int64_t lbm_grid_steps(const lbm_grid *g);

/* Checkpoint: copies the grid's state to or from caller-owned DEVICE memory of
 * exactly lbm_grid_state_bytes(g) bytes (nbytes must equal it, else LBM_EINVAL),
 * together with the step count. The first 256 bytes are a header: magic
 * "LBM2CKPT", version, storage type, nx, ny, the FP16 scale S and a hash of the
 * parameters the update depends on (tau, nu, eps, G, bc, force model, scalar or
 * tensor drag, force field or not). Loading compares it with the loading grid's
 * own and returns LBM_EINVAL on any difference, so a state saved by a grid of
 * another size, storage, scale or parameter set is never misread. The header is
 * followed by both distribution buffers, the current one first (the previous one
 * is kept so that the convergence test after a restart compares the same two
 * states as an uninterrupted run). Each buffer holds 9 planes of the storage
 * type, plane a at offset a * plane where plane = nx * ny rounded up to a
 * multiple of 64, cell (x, y) at y * nx + x; the values are deviations from
 * w_a rho0, multiplied by the FP16 scale for LBM_F16. The permeability field is
 * not part of the state: load it into a grid created on the same field. */
int64_t lbm_grid_state_bytes(const lbm_grid *g);
lbm_status lbm_grid_save_state(lbm_grid *g, void *state_dev, int64_t nbytes, int64_t *steps);
lbm_status lbm_grid_load_state(lbm_grid *g, const void *state_dev, int64_t nbytes, int64_t steps);

/* Storage scale S in use (1 for LBM_F32 / LBM_F64). */
double lbm_grid_scale(const lbm_grid *g);

/* --------------------------------------------------------- local problems ---
 * Section 3 of the paper: each subdomain ("leaf") is solved twice on the fine
 * grid with periodic closure, driven by G1 = (g_const, 0) and G2 = (0, g_const),
 * from rest until its volume-averaged flow velocity ubar settles; then
 *   K* = nu / g_const [[ubar1_x, ubar2_x], [ubar1_y, ubar2_y]]        (Eq. 17)
 * which reproduces the mean flux of the heterogeneous leaf when the leaf is
 * re-run with the uniform tensor K* (Eqs. 19-21). */
typedef struct {
    int32_t x0, y0;       /* lower-left cell of the leaf in the field                 */
    int32_t size;         /* side s in cells, 1 <= s <= 64                            */
} lbm_leaf;

/* Solves all leaves in one launch. p: nx, ny are the FIELD dimensions and tau,
 * nu (< 0: nu_eff), eps the lattice parameters; bc, gx, gy and scale are
 * ignored (leaves are periodic). storage = LBM_F64 runs the solver in FP64
 * (deviations and arithmetic; leaves up to 45 cells including twice the
 * margin); any other value runs it with FP32 deviations and FP32 arithmetic
 * (leaves up to 64 cells). The mean velocities are reduced in FP64 either way.
 * kappa_dev: float [ny][nx] field; leaves_dev: DEVICE array of n_leaves leaves,
 * each inside the field. Stopping test per drive d, every check_every steps t:
 *   |ubar_d(t) - ubar_d(t - check_every)| <= tol_rel * check_every * |ubar_d(t)|;
 * tol_rel = 0 runs exactly max_steps. Outputs (caller-owned DEVICE memory):
 *   keff_dev   double [n_leaves][4] = (K*_xx, K*_xy, K*_yx, K*_yy), lattice units;
 *   status_dev int32  [n_leaves]   = LBM_OK, LBM_ENOTCONV (max_steps reached with
 *                                    tol_rel > 0) or LBM_ETIMEOUT (abandoned);
 *   steps_dev  int32  [n_leaves][2] steps taken per drive, or NULL.
 * persistent != 0: one persistent launch fed by a device work queue, leaves
 * resident in shared memory with per-leaf exit; persistent == 0: one launch
 * per leaf (the same solver, for comparison). Returns the worst per-leaf
 * status (LBM_OK, LBM_ENOTCONV or LBM_ETIMEOUT); invalid leaves give
 * LBM_EINVAL before any launch. Uses device scratch for the queue. */
lbm_status lbm_local_keff_batch(const lbm_params *p, const float *kappa_dev, const lbm_leaf *leaves_dev,
                                int32_t n_leaves, double g_const, double tol_rel, int64_t max_steps,
                                int32_t check_every, int32_t persistent, double *keff_dev, int32_t *status_dev,
                                int32_t *steps_dev, void *cuda_stream);

/* Allocation-free variant of lbm_local_keff_batch (the paper has no counterpart;
 * it exists for callers of this library). Some callers cannot allocate device
 * memory: code that runs inside a host application owning a fixed device pool,
 * under a hard memory budget, or beside an allocator that must not be bypassed.
 * This call allocates no device or pinned memory (no cudaMalloc, cudaFree or
 * cudaMallocHost, directly or through another library); the caller passes the
 * inputs and outputs exactly as for lbm_local_keff_batch, and the work queue
 * lives in a static device array built into the library (1 MiB, held on every
 * GPU that loads it until the process exits). Differences from
 * lbm_local_keff_batch: always one persistent launch; at most 131072 leaves
 * per call (more gives LBM_EINVAL); p->margin must be 0 (plain local
 * problems); leaves are validated on the device (a bad leaf gives LBM_EINVAL
 * before the solver starts). storage selects the FP32 or FP64 solver exactly as
 * for lbm_local_keff_batch (leaves up to 45 cells in FP64). The first call on
 * each device looks up the array's device address (cudaGetSymbolAddress).
 * Every call reads the class table and the status flags back to the
 * host and synchronises the stream before it returns. Every call reuses the same
 * array (it is cleared at the start of each call), so calls that overlap on the
 * GPU (other streams or threads) race on it and must be serialised by the
 * caller. The results are those of lbm_local_keff_batch with persistent != 0,
 * bit for bit. */
lbm_status lbm_local_keff_batch_noalloc(const lbm_params *p, const float *kappa_dev, const lbm_leaf *leaves_dev,
                                        int32_t n_leaves, double g_const, double tol_rel, int64_t max_steps,
                                        int32_t check_every, double *keff_dev, int32_t *status_dev,
                                        int32_t *steps_dev, void *cuda_stream);

/* Local-global local problems: the Conclusions name local-global treatments,
 * beside oversampling, for channelised and high-contrast media, without detail;
 * this is the library's reading. Every block x block block of the field is a
 * leaf; its patch is the block grown by p->margin cells on every side (periodic
 * wrap at the field's edges), driven by G = g_const along x, then along y, as
 * in Section 3, but closed by a ring of fixed cells instead of periodicity.
 * The ring holds a global coarse solution: coarse_dev is a caller-owned DEVICE
 * float [2][3][ny/block][nx/block] array with, for the coarse run driven along
 * x and then the one driven along y, the density deviation rho - 1 and the
 * velocity components u and v of each coarse cell (Eq. 15, lbm_coarse_run's
 * rho/u/v outputs; coarse and fine lattice units share the velocity and
 * density scale). That state is interpolated bilinearly (periodic) from the
 * coarse cell centres to every cell of the patch, the density deviation taken
 * relative to the block's own coarse cell (rho0 = 1 at the block: the global
 * pressure level is arbitrary); all cells start from its equilibrium, or, with
 * p->warm_start = 1 and block + 2 margin a multiple of 8, the inner cells start
 * from the Darcy flow through the patch with the ring's pressures held (finite
 * volumes as for warm_start on periodic patches, the ring's rho - 1 as
 * 3 eps G p on the boundary; conjugate gradients to a relative residual of
 * 1e-7 in shared memory when the job starts). Each ring
 * cell emits, every step, what a cell at its density emits after a collision at
 * tau = 1: the equilibrium (Eq. 2) at momentum rho u + rho f_m / 2 (f_m of Eq. 5
 * at the ring cell's own kappa; zero where kappa = 0). ring = 1: u is the coarse
 * state's velocity. ring = 2 (pressure only): u starts there and is refreshed at
 * every check from the velocity of the ring cell's inward neighbour (diagonal at
 * corners), acting from the second step after the check; check_every must be
 * even. A run stops on the relative change of the inner window's whole mean
 * velocity vector (test as for warm_start = 1). K* follows from Section 2's
 * Brinkman equation at steady state averaged over the block (the inner window):
 * <u> = (K* / nu) <F> with F = G e_d - grad(rho) / (3 eps) (p = c_s^2 rho,
 * rho0 = 1), grad(rho) by central differences cell by cell; with U and F the
 * 2 x 2 matrices of the two drives' window means, K* = nu U F^-1 (Eq. 17 when
 * the window's mean density gradient vanishes). A block whose whole patch has
 * one kappa runs no local problem: Darcy flow through a uniform medium gives
 * K* = kappa I under any boundary pressure; it gets that, status LBM_OK, 0 steps
 * and a NaN window.
 * keff_fallback_dev: NULL (K* as computed, not symmetrised), or a caller-owned
 * DEVICE double [ny/block][nx/block][4] of tensors to fall back to (e.g. the
 * periodic local problems' K*): a block then keeps its K*, symmetrised, only
 * when its run met the tolerance, the symmetrised tensor is positive definite
 * and the 2-norm condition number of its F is at most 10; otherwise it takes
 * the fallback, and *n_fallback (HOST, may be NULL) counts those blocks.
 * Requirements: nx, ny multiples of block; p->margin >= 2, below nx and ny, and
 * block + 2 margin <= 64 (<= 45 with storage = LBM_F64, which runs the local
 * problems in FP64); warm_start 0 or 1; eps > 0. Outputs (caller-owned DEVICE memory):
 *   keff_dev   double [ny/block][nx/block][4] (xx, xy, yx, yy), fine lattice units;
 *   status_dev int32  [ny/block][nx/block] as lbm_local_keff_batch;
 *   steps_dev  int32  [ny/block][nx/block][2], or NULL;
 *   window_dev double [ny/block][nx/block][2][4], or NULL: per drive the window's
 *              mean u, mean v, mean d(rho)/dx and mean d(rho)/dy.
 * Returns as lbm_local_keff_batch; synchronises the stream. */
lbm_status lbm_local_keff_lg(const lbm_params *p, const float *kappa_dev, int32_t block, const float *coarse_dev,
                             double g_const, double tol_rel, int64_t max_steps, int32_t check_every, int32_t ring,
                             const double *keff_fallback_dev, double *keff_dev, int32_t *status_dev,
                             int32_t *steps_dev, double *window_dev, int32_t *n_fallback, void *cuda_stream);

/* Wall-clock bound (seconds, > 0) of one local-problem launch; past it the
 * kernel abandons its remaining jobs with LBM_ETIMEOUT instead of running on.
 * Process-wide; default 600 s. */
lbm_status lbm_set_time_limit(double seconds);

/* -------------------------------------------------------- K* surrogate ---
 * A learned shortcut for the local problems, not part of the paper (which
 * obtains every K* by local LBM, Section 3): an ensemble of small CNNs maps a
 * subdomain's permeability patch to (log K*_xx, log K*_yy); local LBM stays the
 * fallback for doubtful patches and the arbiter of the surrogate's error.
 * Network per model: six 3x3 'same' convolutions 9 -> 32 -> 32 -> 64 -> 64 ->
 * 64 -> 64 with ReLU, global average pooling, a 64 -> 2 linear head; BF16
 * activations and weights on the tensor cores with FP32 accumulation, FP32
 * master weights, Adam. Inputs are the nine planes lbm_patches writes. */
typedef struct lbm_surrogate lbm_surrogate;

/* Number of FP32 parameters of one model; layout: for layer l = 0..5 the weights
 * [c_out][c_in][3][3] then the bias [c_out] (c_in = 9, 32, 32, 64, 64, 64;
 * c_out = 32, 32, 64, 64, 64, 64), then the head [2][64] and its bias [2]. */
int64_t lbm_surrogate_param_count(void);

/* Creates n_models (1..16) models with seeded He-normal weights (splitmix64). */
lbm_status lbm_surrogate_create(int32_t n_models, uint64_t seed, lbm_surrogate **out);
lbm_status lbm_surrogate_destroy(lbm_surrogate *s);
/* Copy one model's FP32 parameters to / from HOST memory (checkpoints, tests). */
lbm_status lbm_surrogate_get_params(const lbm_surrogate *s, int32_t model, float *host_out);
lbm_status lbm_surrogate_set_params(lbm_surrogate *s, int32_t model, const float *host_in);
/* Normalisation and gate range, HOST float[13]: input shift and scale of the
 * log-K planes, target mean/std of log K*_xx and log K*_yy, then (low, high) of
 * each patch statistic (mean, std, gradient energy of log K), then the target
 * mode: the networks learn (log K* - c) / w per component with, per leaf,
 * 0: c = mean log K, w = 1; 1: c = midpoint of the log layered-medium bounds
 * (rows as parallel series tubes below, columns as series parallel slabs above)
 * of the leaf's 64 x 64 log-K plane (see lbm_patches), w = 1; 2: that midpoint
 * and w = half the log width (at least 0.05); 3: c = log of the leaf's Darcy K*
 * (finite volumes on the leaf, harmonic face permeabilities, periodic, unit
 * drive along x and along y; solved on the device by preconditioned conjugate
 * gradients in FP64), w = 1, so the networks learn the Brinkman and
 * discretisation correction to Darcy flow. lbm_surrogate_train sets every
 * entry but the mode from its data and keeps the mode set before it (2 for a
 * new ensemble). */
lbm_status lbm_surrogate_set_normalization(lbm_surrogate *s, const float norm[13]);   /* mode not 0-3: EINVAL */
lbm_status lbm_surrogate_get_normalization(const lbm_surrogate *s, float norm[13]);

/* Leaf -> surrogate input. For each leaf (size s dividing 32, or a multiple of
 * 64 up to 1024) the leaf's log K is put on a 64 x 64 plane (each cell repeated
 * 64/s times per axis for s <= 32, the leaf itself for s = 64, the mean of log K
 * over (s/64)^2 blocks above) and x_dev[i] receives nine float [32][32] planes:
 * plane 2a + b holds that plane's cell (2 row + a, 2 column + b), so a 64-cell
 * leaf enters at full resolution; plane 4 is the constant log2(s)/6; planes 5-8
 * are the context of the 32 x 32 mean of the four phase planes: the harmonic and
 * the arithmetic mean of K along each of its rows (repeated across the row),
 * then along each column (repeated down the column), as log K.
 * stats_dev[i] = (mean, standard deviation, gradient energy) of that 32 x 32
 * mean patch. kappa must be > 0. */
lbm_status lbm_patches(const float *kappa_dev, int32_t nx, int32_t ny, const lbm_leaf *leaves_dev, int32_t n,
                       float *x_dev, float *stats_dev, void *cuda_stream);

/* Trains every model on n samples x_dev [n][9][32][32] (lbm_patches), targets
 * y_dev [n][2] (log K*_xx, log K*_yy), stats_dev [n][3] from lbm_patches. The
 * networks learn (log K* - c) / w with the per-leaf base (c, w) of the target
 * mode (see lbm_surrogate_set_normalization), standardised; lbm_surrogate_predict
 * undoes both. Adam (0.9, 0.999, 1e-8), learning rate lr with cosine decay to
 * lr/10, mini-batches of `batch` (<= 1024) from a seeded shuffle per epoch.
 * loss_host (HOST, may be NULL) receives [n_models][epochs] mean training loss
 * on standardised targets. */
lbm_status lbm_surrogate_train(lbm_surrogate *s, const float *x_dev, const float *y_dev, const float *stats_dev,
                               int32_t n, int32_t epochs, int32_t batch, double lr, uint64_t seed, float *loss_host,
                               void *cuda_stream);

/* Predictions of every model for inputs x_dev [n][9][32][32]:
 * y_dev [n_models][n][2] = log K*_xx, log K*_yy. */
lbm_status lbm_surrogate_predict(lbm_surrogate *s, const float *x_dev, int32_t n, float *y_dev, void *cuda_stream);

/* Per-size gate of lbm_surrogate_keff (and lbm_upscale) when it is called with
 * spread_max = 0: HOST float[7], the relative spread limit for leaves of 1, 2, 4,
 * 8, 16, 32 and 64 cells (each > 0; default 0.03). */
lbm_status lbm_surrogate_set_gate(lbm_surrogate *s, const float spread_by_log2size[7]);
lbm_status lbm_surrogate_get_gate(const lbm_surrogate *s, float spread_by_log2size[7]);

/* K* of arbitrary leaves by the ensemble, with local LBM (Section 3, Eq. 17) for
 * the leaves the gate rejects, all enqueued on the device: patches (lbm_patches),
 * inference of every model, the gate, and the persistent local solver whose work
 * queue the gate fills on the device (no host round trip between them; one
 * stream synchronisation at the end). A leaf (size s a power of two from 1 to
 * 64, or to 45 cells with the margin for LBM_F64 storage; inside the field) is
 * accepted when, for log K*_xx and log K*_yy, the members' sample standard
 * deviation is at most ln(1 + spread) and their mean is finite, and each patch
 * statistic lies in the range seen in training; spread = spread_max when > 0,
 * else the ensemble's per-size value (lbm_surrogate_set_gate). Accepted leaves
 * get K* = diag(exp(mean log K*_xx), exp(mean log K*_yy)); the others are solved
 * as by lbm_local_keff_batch (p: tau, nu, eps, storage, margin; check every 64
 * steps) and get its K*. Outputs (caller-owned DEVICE memory): keff_dev double
 * [n][4] (xx, xy, yx, yy), fallback_dev int32 [n] (0 accepted, 1 local LBM; may
 * be NULL), status_dev int32 [n] (LBM_OK for accepted leaves, the local solver's
 * status otherwise; may be NULL); *n_fallback (HOST, may be NULL) the number of
 * leaves solved by local LBM. An invalid leaf gives LBM_EINVAL after the device
 * work (it is found there) with no local problem solved; otherwise returns the
 * worst status as lbm_local_keff_batch. Work buffers are kept in the ensemble
 * and reused by later calls (no allocation once they are large enough). */
lbm_status lbm_surrogate_keff(lbm_surrogate *s, const lbm_params *p, const float *kappa_dev,
                              const lbm_leaf *leaves_dev, int32_t n, double spread_max, double g_const,
                              double tol_rel, int64_t max_steps, double *keff_dev, int32_t *fallback_dev,
                              int32_t *status_dev, int32_t *n_fallback, void *cuda_stream);

/* One forward and backward pass of one model on n <= 1024 inputs with
 * targets t_dev [n][2] in standardised units: HOST outputs (each may be NULL)
 * grad_host [param_count] = d mean((y - t)^2) / d params, *loss_host, and the
 * raw outputs y_host [n][2]. For gradient checks against an independent code. */
lbm_status lbm_surrogate_grad(lbm_surrogate *s, int32_t model, const float *x_dev, const float *t_dev, int32_t n,
                              float *grad_host, float *loss_host, float *y_host, void *cuda_stream);

/* ------------------------------------------------------------- upscaling ---
 * Section 3: the field is cut into block x block subdomains, one coarse point
 * each (row-major, coarse cell (I, J) <-> fine cells [I r, (I+1) r) x [J r, (J+1) r)).
 * K* of every subdomain comes from its local problems (lbm_local_keff_batch).
 * keff_coarse_dev: caller-owned DEVICE double [ny/r][nx/r][4] (xx, xy, yx, yy) in
 * FINE lattice units. With sur == NULL every block is solved by local LBM. With
 * an ensemble, lbm_surrogate_keff runs on one leaf per block: its prediction
 * (K*_xx = exp(mean log K*_xx), likewise yy, zero off-diagonal) is used for a
 * block unless the ensemble's spread (standard deviation across models of either
 * log K*) exceeds ln(1 + spread_max) (spread_max = 0: the ensemble's per-size
 * limit) or a patch statistic lies outside the range seen in training; such
 * blocks fall back to local LBM. *n_fallback (HOST, may be NULL) receives the
 * number of blocks solved by local LBM. Status as for lbm_local_keff_batch
 * (check_every = 64, persistent launch). */
lbm_status lbm_upscale(const lbm_params *p, const float *kappa_dev, int32_t block, const lbm_surrogate *sur,
                       double spread_max, double g_const, double tol_rel, int64_t max_steps,
                       double *keff_coarse_dev, int32_t *n_fallback, void *cuda_stream);

/* Local-global upscaling in one call (the treatment of lbm_local_keff_lg):
 * K* of every block x block block by the periodic local problems of Section 3
 * (lbm_upscale with margin 0, from rest), then `passes` local-global passes:
 * each runs the coarse model with the current K* (lbm_coarse_run, from rest,
 * at most coarse_max_steps steps, stopping test coarse_tol; periodic, FP32)
 * driven by G = g_const along x and along y, and solves lbm_local_keff_lg on the two
 * steady states (p->margin >= 2, the pressure-only ring, p->warm_start for its
 * Darcy start, check_every 64) with the periodic K* as the fallback tensors.
 * p: as for lbm_local_keff_lg (nx, ny the fine field; gx, gy ignored).
 * keff_coarse_dev: caller-owned DEVICE double [ny/block][nx/block][4], the
 * final K* (the periodic K* when passes = 0). *n_fallback (HOST, may be NULL):
 * blocks of the last pass that took the periodic K*. Returns the worst status
 * of the local problems (LBM_OK, LBM_ENOTCONV or LBM_ETIMEOUT), or the error of
 * a failing step. Synchronises the stream. */
lbm_status lbm_upscale_lg(const lbm_params *p, const float *kappa_dev, int32_t block, int32_t passes,
                          double g_const, double tol_rel, int64_t max_steps, int64_t coarse_max_steps,
                          double coarse_tol, double *keff_coarse_dev, int32_t *n_fallback, void *cuda_stream);

/* Coarse lattice parameters for a fine set-up coarsened by `block` (= r):
 * nx/r x ny/r cells, tau_c = 1/2 + (tau_f - 1/2)/r, nu_c = nu_f/r, G_c = r G_f,
 * same eps, bc and storage (the paper keeps rho0, nu_eff, eps, nu and G and
 * scales dx and dt by r; Section 3 and Section 4.3). */
lbm_status lbm_coarse_params(const lbm_params *fine_p, int32_t block, lbm_params *coarse_out);

/* The coarse (upscaled) run of Section 3 / Section 4.3: the simplified
 * Shan-Chen step on the coarse lattice with the tensor drag of Eq. 18,
 *   rho u = (I + eps nu_c K*_c^-1 / 2)^-1 (j + eps rho G_c / 2),  K*_c = K*_f / r^2,
 * from rest for up to max_steps (stopping test as lbm_step). keff_coarse_dev is
 * [ny/r][nx/r][4] in FINE lattice units (as lbm_upscale writes it); each K* must
 * be finite with K*_c + (eps nu_c / 2) I invertible. g_coarse_dev: NULL for the
 * constant force of fine_p, else float [2][ny/r][nx/r] holding G sampled at the
 * coarse cell centres in FINE lattice units (the call multiplies it by r).
 * rho/u/v_dev (any may be NULL): caller-owned float [ny/r][nx/r] outputs (Eq. 15).
 * The grid is created and destroyed inside the call. */
lbm_status lbm_coarse_run(const lbm_params *fine_p, int32_t block, const double *keff_coarse_dev,
                          const float *g_coarse_dev, int64_t max_steps, double tol_rel, int32_t check_every,
                          float *rho_dev, float *u_dev, float *v_dev, int64_t *steps_done, void *cuda_stream);

/* Mean of a float [ny][nx] device field over block x block tiles into float
 * [ny/block][nx/block] (accumulated in FP64, fixed order): the fine-grid
 * averages the coarse run is compared with (Section 4.3.1). */
lbm_status lbm_block_average(const float *in_dev, int32_t nx, int32_t ny, int32_t block, float *out_dev,
                             void *cuda_stream);

/* ------------------------------------------------------ 3-D grids (D3Q19) ---
 * Section 2 uses the D3Q19 lattice for three-dimensional problems with the
 * algorithms unchanged. These calls step the scheme on it (rest, 6 face and 12 edge velocities,
 * weights 1/3, 1/18, 1/36, c_s^2 = 1/3) with the same update as the 2-D grid
 * (Eqs. 6, 16, 2, 13 with three-component vectors), periodic in x, y and z,
 * constant body force, scalar permeability (a tensor K* per cell for the coarse
 * grid below), from rest. Arrays are [nz][ny][nx] (x fastest), caller-owned
 * device memory. */
typedef struct {
    int32_t nx, ny, nz;   /* lattice size, each >= 1; ny, nz <= 65535                   */
    double  tau, nu, eps; /* as in lbm_params (nu < 0 selects nu_eff)                  */
    double  gx, gy, gz;   /* constant body force                                        */
    int32_t storage;      /* LBM_F32, LBM_F64, or LBM_F16 (scalar-kappa grids only:   */
                          /* deviations scaled by an automatic power of two S with    */
                          /* S max|g| near 2^12, FP32 arithmetic, 80 B per update)    */
    int32_t margin;       /* lbm3d_local_keff_batch only: oversampling margin m in     */
                          /* [0, 32] (0: plain local problems); grids ignore it        */
} lbm3d_params;
typedef struct lbm3d_grid lbm3d_grid;

/* Creates a 3-D grid: two distribution buffers of 19 planes of the storage type
 * and the per-cell drag fraction; kappa_dev float [nz][ny][nx] is read during the
 * call only (>= 0, +inf allowed; NaN or negative give LBM_EINVAL). */
lbm_status lbm3d_grid_create(const lbm3d_params *p, const float *kappa_dev, void *cuda_stream, lbm3d_grid **out);
lbm_status lbm3d_grid_destroy(lbm3d_grid *g);
/* Advances the grid by `steps` time steps (fused pull-stream + collide). */
lbm_status lbm3d_step(lbm3d_grid *g, int64_t steps);
/* Density and flow velocity (Eq. 15) into caller-owned float [nz][ny][nx] device
 * arrays; any of the four may be NULL. */
lbm_status lbm3d_get_fields(lbm3d_grid *g, float *rho_dev, float *u_dev, float *v_dev, float *w_dev);
/* Volume average of the flow velocity, FP64 in a fixed order; HOST out[3]. */
lbm_status lbm3d_mean_velocity(lbm3d_grid *g, double out_mean_uvw[3]);
/* Checkpoint: copies the grid's current state to or from caller-owned DEVICE
 * memory of exactly lbm3d_grid_state_bytes(g) bytes (-1 for NULL; nbytes must
 * equal it, else LBM_EINVAL): a 256-byte header (magic "LBM3CKPT", version,
 * storage, nx, ny, nz, the FP16 scale S and a hash of tau, nu, eps, G and the
 * scalar or tensor drag), then 19 planes of the storage type, plane a at offset
 * a * plane with plane = nx ny nz rounded up to a multiple of 64, holding the
 * deviations from w_a rho0 (times S for LBM_F16). Loading a state whose header
 * differs from the loading grid's own gives LBM_EINVAL. A grid created with the
 * same parameters and field continues bit for bit. */
int64_t lbm3d_grid_state_bytes(const lbm3d_grid *g);
lbm_status lbm3d_grid_save_state(lbm3d_grid *g, void *state_dev, int64_t nbytes);
lbm_status lbm3d_grid_load_state(lbm3d_grid *g, const void *state_dev, int64_t nbytes);

/* Coarse-grid parameters for blocks of block^3 fine cells (Section 3 in 3-D: the
 * same rho0, nu_eff, eps, nu and G in physical units with dx and dt scaled by
 * r = block): nx, ny, nz / r, tau_c = 1/2 + (tau - 1/2) / r, nu_c = nu / r (nu < 0
 * first becomes nu_eff), G_c = r G. nx, ny, nz must be multiples of block, else
 * LBM_EINVAL. HOST in and out. */
lbm_status lbm3d_coarse_params(const lbm3d_params *fine_p, int32_t block, lbm3d_params *coarse_out);
/* Creates the coarse 3-D grid of the upscaled model (Eq. 18 in 3-D): parameters
 * from lbm3d_coarse_params, and per coarse cell the tensor K* of
 * keff_coarse_dev double [nz/r][ny/r][nx/r][3][3] (row i = velocity component,
 * column j = drive, as lbm3d_local_keff_batch writes it, in FINE lattice units;
 * divided by r^2 here). The step then uses rho u = (I + (eps nu / 2) K*^-1)^-1
 * (j + eps rho G / 2), stored per cell as the 9 planes of E = (eps nu / 2)
 * (K* + (eps nu / 2) I)^-1 (188 B per FP32 update). keff is read during the call
 * only; non-finite entries or a singular K* + (eps nu / 2) I give LBM_EINVAL.
 * Step, fields and mean velocity are the lbm3d_* calls above. */
lbm_status lbm3d_coarse_grid_create(const lbm3d_params *fine_p, int32_t block, const double *keff_coarse_dev,
                                    void *cuda_stream, lbm3d_grid **out);
/* Mean of a float [nz][ny][nx] device field over block^3 cubes into float
 * [nz/block][ny/block][nx/block] (FP64 accumulation, fixed order): the fine-grid
 * averages a 3-D coarse run is compared with. Sizes must be multiples of block. */
lbm_status lbm3d_block_average(const float *in_dev, int32_t nx, int32_t ny, int32_t nz, int32_t block,
                               float *out_dev, void *cuda_stream);

/* Three-dimensional local problems (Section 3 with the D3Q19 lattice). For each
 * cubic leaf (x0, y0, z0, size) of the field kappa_dev [nz][ny][nx] (p->nx, ny,
 * nz are the field size; tau, nu, eps as for a 3-D grid; storage LBM_F32 or
 * LBM_F64; the force is ignored) three periodic runs from rest, driven by g_const along x, y and z,
 * each until its volume-averaged velocity settles: every check_every steps t,
 * |ubar_d(t) - ubar_d(t - check_every)| <= tol_rel * check_every * |ubar_d(t)|
 * on the driven component d (tol_rel = 0 runs exactly max_steps). Eq. 17 in 3-D
 * gives column d of K*: K*_id = nu ubar_d,i / g_const. Outputs (caller-owned
 * DEVICE memory): keff_dev double [n][3][3] (row i = velocity component, column
 * d = drive), status_dev int32 [n] (LBM_OK, LBM_ENOTCONV, or LBM_ETIMEOUT when
 * the lbm_set_time_limit bound ran out first; keff then not valid), steps_dev
 * int32 [n][3] or NULL. Cubes that fit the shared memory of a thread-block
 * cluster of at most 16 CTAs (up to 32 cells wide in FP32, 22 in FP64) run one
 * job per cluster entirely on chip; larger cubes run with their 3 n jobs stacked
 * in device memory (allocated and freed by the call); the environment variable
 * LBM_LOCAL3_GLOBAL=1 sends every size that second way. With p->margin = m > 0
 * (oversampling) each run is on the leaf grown by m cells on every side, cut from
 * the field with periodic wrap at its edges, and the stop test and Eq. 17 use the
 * mean over the inner leaf only. Returns the worst status; leaves outside the
 * field, size + 2 m outside [1, 256] or m outside [0, min(32, nx, ny, nz)] give
 * LBM_EINVAL. */
typedef struct { int32_t x0, y0, z0, size; } lbm3d_leaf;
/* The upscaling step in 3-D: K* of every block^3 block of the field (one cubic
 * leaf per coarse cell, three drives, check every 64 steps, p->margin as
 * above) into keff_coarse_dev double [nz/r][ny/r][nx/r][3][3], fine lattice
 * units, the layout lbm3d_coarse_grid_create reads. n_notconv (HOST, may be
 * NULL) receives the number of blocks whose status is not LBM_OK. nx, ny, nz
 * must be multiples of block; returns the worst status, as
 * lbm3d_local_keff_batch. Allocates and frees the leaf list and the status. */
lbm_status lbm3d_upscale(const lbm3d_params *p, const float *kappa_dev, int32_t block, double g_const,
                         double tol_rel, int64_t max_steps, double *keff_coarse_dev, int32_t *n_notconv,
                         void *cuda_stream);
lbm_status lbm3d_local_keff_batch(const lbm3d_params *p, const float *kappa_dev, const lbm3d_leaf *leaves_dev,
                                  int32_t n_leaves, double g_const, double tol_rel, int64_t max_steps,
                                  int32_t check_every, double *keff_dev, int32_t *status_dev, int32_t *steps_dev,
                                  void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
