// coarse.cu -- the upscaled (coarse-grid) run of Section 3 and its inputs:
// K* per coarse cell from the local problems (lbm_upscale), the coarse run with
// the tensor drag of Eq. 18 (lbm_coarse_run), and r x r block averages of fine
// fields for comparison (lbm_block_average).
//
// Coarse lattice parameters. The paper keeps rho0, nu_eff, eps, nu and G the
// same on both grids and scales dx and dt by the same factor r (so c is the
// same). In lattice units of the coarse grid that is
//   tau_c = 1/2 + (tau_f - 1/2) / r,  nu_c = nu_f / r,  K*_c = K*_f / r^2,  G_c = r G_f,
// and lattice velocities are directly comparable between the grids.
#include "lbm_internal.h"

#include <cmath>
#include <vector>

namespace lbm {

lbm_status fail(lbm_status s, const char *fmt, ...);
bool is_device_ptr(const void *p);
void count_launches(int64_t n);
lbm_status validate_params(const lbm_params *p);
lbm_status grid_create_impl(const lbm_params *p, const float *kappa_dev, const double *kstar_dev,
                            double kstar_scale, const float *g_field_dev, void *cuda_stream, lbm_grid **out);
lbm_status local_keff_impl(const lbm_params *p, const float *kappa_dev, const lbm_leaf *leaves_dev, int32_t n_leaves,
                           double g_const, double tol_rel, int64_t max_steps, int32_t check_every,
                           int32_t persistent, double *keff_dev, int32_t *status_dev, int32_t *steps_dev,
                           void *cuda_stream, double time_limit_s);
double local_time_limit();
lbm_status upscale_with_surrogate(const lbm_params *p, const float *kappa_dev, int32_t block, lbm_surrogate *s,
                                  double spread_max, double g_const, double tol_rel, int64_t max_steps,
                                  double *keff_dev, int32_t *n_fallback, void *cuda_stream);

namespace {

// mean over r x r blocks, accumulated in double in a fixed order (one thread per block)
__global__ void __launch_bounds__(256) block_average_kernel(const float *in, int nx, int ny, int r, float *out)
{
    const int cx = nx / r, cy = ny / r;
    const int64_t nb = (int64_t)cx * cy;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
        const int J = (int)(b / cx), I = (int)(b - (int64_t)J * cx);
        double s = 0.0;
        for (int y = J * r; y < (J + 1) * r; ++y) {
            const float *row = in + (int64_t)y * nx + (int64_t)I * r;
            for (int x = 0; x < r; ++x) s += (double)row[x];
        }
        out[b] = (float)(s / ((double)r * r));
    }
}

// scale a [2][n] force field from fine to coarse lattice units (G_c = r G_f)
__global__ void __launch_bounds__(256) scale_force_kernel(const float *in, float *out, int64_t n2, float r)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i] * r;
}

// rho -> rho - 1 in place (the coarse run's density to the deviation the local-global ring takes)
__global__ void __launch_bounds__(256) minus_one_kernel(float *a, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] -= 1.0f;
}

int blocks_for(int64_t n)
{
    int64_t b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" {

lbm_status lbm_block_average(const float *in_dev, int32_t nx, int32_t ny, int32_t block, float *out_dev,
                             void *cuda_stream)
{
    if (nx < 1 || ny < 1 || block < 1 || nx % block || ny % block)
        return fail(LBM_EINVAL, "nx, ny must be positive multiples of block");
    if (!is_device_ptr(in_dev) || !is_device_ptr(out_dev)) return fail(LBM_EINVAL, "in/out must be device pointers");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int64_t nb = (int64_t)(nx / block) * (ny / block);
    block_average_kernel<<<blocks_for(nb), 256, 0, st>>>(in_dev, nx, ny, block, out_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LBM_ECUDA, "block average launch: %s", cudaGetErrorString(e));
    count_launches(1);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(LBM_ECUDA, "block average: %s", cudaGetErrorString(e));
    return LBM_OK;
}

lbm_status lbm_coarse_params(const lbm_params *fine_p, int32_t block, lbm_params *coarse_out)
{
    lbm_status s = validate_params(fine_p);
    if (s != LBM_OK) return s;
    if (!coarse_out) return fail(LBM_EINVAL, "coarse_out is NULL");
    if (block < 1 || fine_p->nx % block || fine_p->ny % block)
        return fail(LBM_EINVAL, "nx, ny must be multiples of block %d", block);
    const double r = block;
    const double nu_f = fine_p->nu < 0.0 ? (fine_p->tau - 0.5) / 3.0 : fine_p->nu;
    lbm_params c = *fine_p;
    c.nx = fine_p->nx / block;
    c.ny = fine_p->ny / block;
    c.tau = 0.5 + (fine_p->tau - 0.5) / r;
    c.nu = nu_f / r;
    c.gx = fine_p->gx * r;
    c.gy = fine_p->gy * r;
    c.margin = 0;
    c.warm_start = 0;
    *coarse_out = c;
    return LBM_OK;
}

lbm_status lbm_coarse_run(const lbm_params *fine_p, int32_t block, const double *keff_coarse_dev,
                          const float *g_coarse_dev, int64_t max_steps, double tol_rel, int32_t check_every,
                          float *rho_dev, float *u_dev, float *v_dev, int64_t *steps_done, void *cuda_stream)
{
    if (steps_done) *steps_done = 0;
    lbm_params c;
    lbm_status s = lbm_coarse_params(fine_p, block, &c);
    if (s != LBM_OK) return s;
    if (!keff_coarse_dev || !is_device_ptr(keff_coarse_dev)) return fail(LBM_EINVAL, "keff_coarse_dev must be a device pointer");
    if (g_coarse_dev && !is_device_ptr(g_coarse_dev)) return fail(LBM_EINVAL, "g_coarse_dev must be a device pointer");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int64_t n = (int64_t)c.nx * c.ny;
    float *gscaled = nullptr;
    if (g_coarse_dev) {
        cudaError_t e = cudaMalloc(&gscaled, sizeof(float) * 2 * n);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(LBM_ENOMEM, "coarse force buffer: %s", cudaGetErrorString(e));
        }
        scale_force_kernel<<<blocks_for(2 * n), 256, 0, st>>>(g_coarse_dev, gscaled, 2 * n, (float)block);
        count_launches(1);
    }
    lbm_grid *g = nullptr;
    s = grid_create_impl(&c, nullptr, keff_coarse_dev, 1.0 / ((double)block * block), gscaled, cuda_stream, &g);
    cudaFree(gscaled);
    if (s != LBM_OK) return s;
    int64_t done = 0;
    double resid = -1.0;
    lbm_status sr = lbm_step(g, max_steps, tol_rel, check_every, &done, &resid);
    if (sr != LBM_OK && sr != LBM_ENOTCONV) {
        lbm_grid_destroy(g);
        return sr;
    }
    lbm_status sf = lbm_get_fields(g, rho_dev, u_dev, v_dev);
    lbm_grid_destroy(g);
    if (sf != LBM_OK) return sf;
    if (steps_done) *steps_done = done;
    return sr == LBM_ENOTCONV ? fail(LBM_ENOTCONV, "coarse run: residual %.3e above tolerance after %lld steps",
                                     resid, (long long)done)
                              : LBM_OK;
}

lbm_status lbm_upscale(const lbm_params *p, const float *kappa_dev, int32_t block, const lbm_surrogate *sur,
                       double spread_max, double g_const, double tol_rel, int64_t max_steps,
                       double *keff_coarse_dev, int32_t *n_fallback, void *cuda_stream)
{
    if (n_fallback) *n_fallback = 0;
    lbm_status s = validate_params(p);
    if (s != LBM_OK) return s;
    if (block < 1 || block > 64 || p->nx % block || p->ny % block)
        return fail(LBM_EINVAL, "block must be in [1, 64] and divide nx, ny");
    // the ensemble is logically const here: only its internal work buffers are reused
    if (sur) return upscale_with_surrogate(p, kappa_dev, block, const_cast<lbm_surrogate *>(sur), spread_max, g_const,
                                           tol_rel, max_steps, keff_coarse_dev, n_fallback, cuda_stream);
    const int cx = p->nx / block, cy = p->ny / block;
    const int64_t nl = (int64_t)cx * cy;
    if (nl > (int64_t)1 << 30) return fail(LBM_EINVAL, "too many blocks");
    std::vector<lbm_leaf> lv((size_t)nl);
    for (int J = 0; J < cy; ++J)
        for (int I = 0; I < cx; ++I) lv[(size_t)J * cx + I] = lbm_leaf{I * block, J * block, block};
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    lbm_leaf *d_leaves = nullptr;
    int32_t *d_status = nullptr;
    cudaError_t e = cudaMalloc(&d_leaves, sizeof(lbm_leaf) * nl);
    if (e == cudaSuccess) e = cudaMalloc(&d_status, sizeof(int32_t) * nl);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_leaves, lv.data(), sizeof(lbm_leaf) * nl, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_leaves);
        cudaFree(d_status);
        return fail(e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "upscale set-up: %s",
                    cudaGetErrorString(e));
    }
    s = local_keff_impl(p, kappa_dev, d_leaves, (int32_t)nl, g_const, tol_rel, max_steps, 64, 1, keff_coarse_dev,
                        d_status, nullptr, cuda_stream, local_time_limit());
    cudaFree(d_leaves);
    cudaFree(d_status);
    if (n_fallback) *n_fallback = (int32_t)nl;
    return s;
}

lbm_status lbm_upscale_lg(const lbm_params *p, const float *kappa_dev, int32_t block, int32_t passes,
                          double g_const, double tol_rel, int64_t max_steps, int64_t coarse_max_steps,
                          double coarse_tol, double *keff_coarse_dev, int32_t *n_fallback, void *cuda_stream)
{
    if (n_fallback) *n_fallback = 0;
    lbm_status s = validate_params(p);
    if (s != LBM_OK) return s;
    if (passes < 0) return fail(LBM_EINVAL, "passes must be >= 0");
    if (block < 1 || block > 64 || p->nx % block || p->ny % block)
        return fail(LBM_EINVAL, "block must be in [1, 64] and divide nx, ny");
    if (coarse_max_steps < 1 || !std::isfinite(coarse_tol) || coarse_tol < 0.0)
        return fail(LBM_EINVAL, "coarse_max_steps must be >= 1 and coarse_tol finite and >= 0");
    if (!keff_coarse_dev || !is_device_ptr(keff_coarse_dev))
        return fail(LBM_EINVAL, "keff_coarse_dev must be a device pointer");
    const int64_t nb = (int64_t)(p->nx / block) * (p->ny / block);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    double *kref = nullptr;
    float *cs = nullptr;
    int32_t *status = nullptr;
    auto release = [&]() {
        cudaFree(kref);
        cudaFree(cs);
        cudaFree(status);
        cudaGetLastError();
    };
    cudaError_t e = cudaMalloc(&kref, sizeof(double) * 4 * nb);
    if (e == cudaSuccess) e = cudaMalloc(&cs, sizeof(float) * 6 * nb);
    if (e == cudaSuccess) e = cudaMalloc(&status, sizeof(int32_t) * nb);
    if (e != cudaSuccess) {
        release();
        return fail(e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "upscale set-up: %s",
                    cudaGetErrorString(e));
    }
    // the paper's local problems: periodic, from rest
    lbm_params p0 = *p;
    p0.margin = 0;
    p0.warm_start = 0;
    s = lbm_upscale(&p0, kappa_dev, block, nullptr, 0.0, g_const, tol_rel, max_steps, kref, nullptr, cuda_stream);
    if (s != LBM_OK && s != LBM_ENOTCONV) {
        release();
        return s;
    }
    lbm_status worst = s;
    const double *kcur = kref;
    for (int pass = 0; pass < passes; ++pass) {
        // the global coarse solutions driven along x and along y, to steady state
        for (int d = 0; d < 2; ++d) {
            lbm_params pd = p0;
            pd.gx = d == 0 ? g_const : 0.0;
            pd.gy = d == 1 ? g_const : 0.0;
            pd.bc = LBM_BC_PERIODIC;
            pd.storage = LBM_F32;
            pd.scale = 0.0;
            float *c = cs + (int64_t)3 * d * nb;
            s = lbm_coarse_run(&pd, block, kcur, nullptr, coarse_max_steps, coarse_tol, 64, c, c + nb, c + 2 * nb,
                               nullptr, cuda_stream);
            if (s != LBM_OK && s != LBM_ENOTCONV) {
                release();
                return s;
            }
            minus_one_kernel<<<blocks_for(nb), 256, 0, st>>>(c, nb);
            count_launches(1);
        }
        int32_t nfb = 0;
        s = lbm_local_keff_lg(p, kappa_dev, block, cs, g_const, tol_rel, max_steps, 64, 2, kref, keff_coarse_dev,
                              status, nullptr, nullptr, &nfb, cuda_stream);
        if (s != LBM_OK && s != LBM_ENOTCONV && s != LBM_ETIMEOUT) {
            release();
            return s;
        }
        if (s > worst) worst = s;
        if (n_fallback) *n_fallback = nfb;
        kcur = keff_coarse_dev;
    }
    if (passes == 0) {
        e = cudaMemcpyAsync(keff_coarse_dev, kref, sizeof(double) * 4 * nb, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            release();
            return fail(LBM_ECUDA, "upscale copy: %s", cudaGetErrorString(e));
        }
    }
    release();
    return worst;
}

}  // extern "C"
