// lbm_internal.h -- declarations shared by the library's translation units.
// Nothing here is part of the public ABI (see include/lbm.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/lbm.h"

namespace lbm {

// D2Q9 velocity set, ordered as in Section 2 of the paper:
// 0 rest, 1..4 axis directions at angles (a-1) pi/2, 5..8 diagonals at (a-5) pi/2 + pi/4.
constexpr int Q = 9;
__host__ __device__ constexpr int ex(int a) { return a == 1 || a == 5 || a == 8 ? 1 : (a == 3 || a == 6 || a == 7 ? -1 : 0); }
__host__ __device__ constexpr int ey(int a) { return a == 2 || a == 5 || a == 6 ? 1 : (a == 4 || a == 7 || a == 8 ? -1 : 0); }
__host__ __device__ constexpr int opp(int a) { return a == 0 ? 0 : (a <= 4 ? ((a + 1) & 3) + 1 : ((a - 3) & 3) + 5); }

enum CoefMode { COEF_SCALAR = 0, COEF_TENSOR = 1 };

// Everything one launch of the fused step (or the moment/check pass) needs.
// src/dst are the storage-type planes [9][plane]; coefficient and force planes
// use CT (float for FP32/FP16 storage, double for FP64).
template <typename T, typename CT>
struct StepArgs {
    int nx, ny;
    int64_t plane;        // elements between consecutive population planes
    CT omega;             // 1 / tau
    CT two_tau;           // 2 tau             (Eq. 16)
    CT one_m_two_tau;     // 1 - 2 tau         (Eq. 16)
    CT half_eps;          // eps dt / 2        (Eq. 6)
    CT gx, gy;            // constant force when gfield == nullptr
    CT rho0;              // rest density in storage units (the FP16 scale S, else 1)
    int guo;              // 1: Guo forcing (u_eq = u plus the forcing term of Eq. 4)
    CT guo_c;             // 6 (1 - 1/(2 tau)): F_a = w_a guo_c e_a . (rho u - j)
    const T *src;         // post-collision state of the previous step
    T *dst;
    const CT *coef;       // COEF_SCALAR: e [plane] (rho u = (1 - e) r); COEF_TENSOR: E [4][plane] (rho u = (I - E) r)
    const CT *gfield;     // [2][plane] or nullptr
};

// Moments / residual pass: reads the current (and optionally previous) state.
template <typename T, typename CT>
struct MomArgs {
    StepArgs<T, CT> s;    // s.src = current state; dst unused
    const T *prev;        // previous state (nullptr: no residual)
    CT inv_scale;         // 1 / S
    float *rho, *u, *v;   // optional field outputs [ny][nx]
    double *partials;     // [gridDim.x][4]: max|du|, max|u|, sum u, sum v
};

struct GridLaunch {
    int step_blocks;      // persistent grid for the fused step
    int step_threads;     // threads per block (<= 512)
    int step_vec;         // cells per thread (0: the default for the storage and row length)
    int mom_blocks;
    int mom_threads;
};

// ---- launchers (step.cu) -----------------------------------------------------
// storage: lbm_storage; coef_mode: CoefMode. All return cudaGetLastError().
cudaError_t launch_step(int storage, int coef_mode, bool gfield, bool walls, const void *args,
                        const GridLaunch &L, cudaStream_t st);
cudaError_t launch_moments(int storage, int coef_mode, bool gfield, bool walls, const void *args,
                           const GridLaunch &L, cudaStream_t st);
cudaError_t launch_reduce_partials(const double *partials, int n, double *out4, cudaStream_t st);
cudaError_t launch_coef_scalar(int storage, const float *kappa, void *coef, int64_t n, int64_t plane,
                               double eps_nu, unsigned *flags, unsigned *kmax_bits, cudaStream_t st);
cudaError_t launch_coef_tensor(int storage, const double *kstar, void *coef, int64_t n, int64_t plane,
                               double c, unsigned *flags, cudaStream_t st);
cudaError_t launch_copy_force(int storage, const float *g, void *dst, int64_t n, int64_t plane,
                              double scale_unused, cudaStream_t st);
int step_vec(int storage, int nx);   // cells per thread used for this storage and row length
int step_blocks_per_sm(int storage, int coef_mode, bool gfield, bool walls, int nx, int threads, int vec = 0);
bool step_vec_ok(int storage, int nx, int vec);   // is this cells-per-thread variant built and usable

// ---- launch counter (lbm_api.cu) ----------------------------------------------
void count_launches(int64_t n);

}  // namespace lbm

namespace lbm {

// ---- checkpoints (lbm_api.cu, d3q19.cu) -----------------------------------------
// A saved state starts with this 256-byte header, then the distribution planes.
// Loading compares every field with the loading grid's own header, so a state
// saved by a grid of another size, storage type, FP16 scale or parameter set is
// rejected instead of being misread.
constexpr int64_t CKPT_HEADER_BYTES = 256;
struct CkptHeader {
    char magic[8];          // "LBM2CKPT" (D2Q9) or "LBM3CKPT" (D3Q19)
    int32_t version;        // 1
    int32_t storage;        // lbm_storage
    int64_t nx, ny, nz;     // nz = 1 for D2Q9
    double scale;           // FP16 storage scale S (1 otherwise)
    uint64_t params_hash;   // FNV-1a over the parameters the update depends on
    int64_t steps;          // steps taken when saved (D2Q9; 0 for D3Q19)
    uint8_t pad[CKPT_HEADER_BYTES - 64];
};
static_assert(sizeof(CkptHeader) == CKPT_HEADER_BYTES, "checkpoint header is 256 bytes");

// 64-bit FNV-1a (Fowler, Noll, Vo) of a byte range, continuing from h.
inline uint64_t fnv1a(const void *data, size_t n, uint64_t h = 0xcbf29ce484222325ull)
{
    const unsigned char *b = static_cast<const unsigned char *>(data);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

}  // namespace lbm

namespace lbm {

// ---- device-built work queue of the local problems (surrogate.cu -> local.cu) ------------
// int array in device memory: the per-size class table the persistent local solver reads at
// start, filled by kernels of the same stream, so no host round trip is needed between the
// gate that picks the leaves and the solver that takes them.
enum DeviceTable {
    DT_NCLASS = 0,            // number of size classes
    DT_SIZE = 1,              // [64] class sizes, descending
    DT_OFF = 65,              // [65] job offsets of the classes (jobs = 2 leaf + drive)
    DT_CURSOR = 130,          // [65] scatter cursor per patch size (index = size)
    DT_COUNT = 195,           // [65] leaves per patch size (index = size)
    DT_HEADS = 260,           // [64] queue heads per class
    DT_BAD = 324,             // non-zero: an invalid leaf was found (nothing is solved)
    DT_WORST = 325,           // worst per-leaf status of the solver
    DT_ABORT = 326,           // the solver's wall-clock limit ran out
    DT_NFALLBACK = 327,       // leaves sent to the solver
    DT_INTS = 384
};

// Launches the persistent local solver on the jobs of a device-built table (the table's job
// list `jobs` holds 2 leaf + drive for leaves of `leaves_dev`; per-leaf outputs are indexed by
// leaf). Enqueues only: no host synchronisation; the caller reads DT_WORST / DT_ABORT later.
lbm_status launch_local_from_table(const lbm_params *p, const float *kappa_dev, const lbm_leaf *leaves_dev,
                                   const int *jobs, int *table, double g_const, double tol_rel, int64_t max_steps,
                                   int32_t check_every, double *keff_dev, int32_t *status_dev, int32_t *steps_dev,
                                   cudaStream_t st, double time_limit_s);

}  // namespace lbm
