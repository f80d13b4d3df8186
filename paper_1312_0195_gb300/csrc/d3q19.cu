// d3q19.cu -- the method on the D3Q19 lattice, which Section 2 uses for
// three-dimensional problems with the algorithms unchanged: periodic in x, y and
// z, constant body force, scalar permeability, FP32 or FP64 deviation storage.
//
// The step is the fine-grid step of step.cu with 19 populations: pull-stream,
// moments, rho u = (1 - e) r with r = j + eps rho G / 2 and the per-cell drag
// fraction e = eps nu / (2 kappa + eps nu) (Eq. 6), rho u_eq = 2 tau rho u +
// (1 - 2 tau) j (Eq. 16), the linear equilibrium w_a (drho + 3 e_a . rho u_eq) of
// Eq. 2 in deviation form, and BGK (Eq. 13). One thread per cell; x runs along
// the threads of a block, so every population plane is read and written
// coalesced. HBM-bound: 19 x 4 x 2 + 4 = 156 bytes per lattice update in FP32.
#include "lbm_internal.h"

#include <cmath>

namespace lbm {

lbm_status fail(lbm_status s, const char *fmt, ...);
bool is_device_ptr(const void *p);
void count_launches(int64_t n);

namespace {

constexpr int Q19 = 19;
// D3Q19 velocities: 0 rest; 1-6 faces (+x, -x, +y, -y, +z, -z); 7-18 edges in opposite pairs
__host__ __device__ constexpr int cx(int a)
{
    return (a == 1 || a == 7 || a == 9 || a == 11 || a == 13) ? 1 : ((a == 2 || a == 8 || a == 10 || a == 12 || a == 14) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int a)
{
    return (a == 3 || a == 7 || a == 10 || a == 15 || a == 17) ? 1 : ((a == 4 || a == 8 || a == 9 || a == 16 || a == 18) ? -1 : 0);
}
__host__ __device__ constexpr int cz(int a)
{
    return (a == 5 || a == 11 || a == 14 || a == 15 || a == 18) ? 1 : ((a == 6 || a == 12 || a == 13 || a == 16 || a == 17) ? -1 : 0);
}
__host__ __device__ constexpr double w19(int a) { return a == 0 ? 1.0 / 3.0 : (a <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }

// a +/- v for a component c in {-1, 0, 1} known at compile time (no multiplication by 0 or 1)
template <int C, typename T> __device__ __forceinline__ T addc(T acc, T v)
{
    return C == 1 ? acc + v : (C == -1 ? acc - v : acc);
}

template <typename T>
struct Step3Args {
    const T *src;
    T *dst;
    const T *coef;          // e per cell
    int nx, ny, nz;
    int64_t plane;          // elements per population plane
    T omega, two_tau, omt, hgx, hgy, hgz;   // 1/tau, 2 tau, 1 - 2 tau, eps G / 2
};

// Index of cell (x - e_x, y - e_y, z - e_z) from the wrapped neighbour offsets.
struct Nbr {
    int64_t z[3], y[3];
    int x[3];
    template <int A> __device__ __forceinline__ int64_t from() const { return z[1 - cz(A)] + y[1 - cy(A)] + x[1 - cx(A)]; }
};

__device__ __forceinline__ Nbr neighbours(int x, int y, int z, int nx, int ny, int nz)
{
    Nbr n;
    const int64_t pz = (int64_t)ny * nx;
    n.x[0] = x == 0 ? nx - 1 : x - 1;
    n.x[1] = x;
    n.x[2] = x + 1 == nx ? 0 : x + 1;
    n.y[0] = (int64_t)(y == 0 ? ny - 1 : y - 1) * nx;
    n.y[1] = (int64_t)y * nx;
    n.y[2] = (int64_t)(y + 1 == ny ? 0 : y + 1) * nx;
    n.z[0] = (z == 0 ? nz - 1 : z - 1) * pz;
    n.z[1] = z * pz;
    n.z[2] = (z + 1 == nz ? 0 : z + 1) * pz;
    return n;
}

template <int A, typename T>
__device__ __forceinline__ void pull_one(const T *__restrict__ src, int64_t plane, const Nbr &nb, T (&g)[Q19])
{
    g[A] = __ldg(src + A * plane + nb.template from<A>());
}
template <typename T, int... As>
__device__ __forceinline__ void pull_all(const T *src, int64_t plane, const Nbr &nb, T (&g)[Q19])
{
    (pull_one<As>(src, plane, nb, g), ...);
}
template <typename T> __device__ __forceinline__ void pull19(const T *src, int64_t plane, const Nbr &nb, T (&g)[Q19])
{
    pull_all<T, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18>(src, plane, nb, g);
}

template <int A, typename T> __device__ __forceinline__ void moment_one(const T (&g)[Q19], T &d, T &jx, T &jy, T &jz)
{
    d += g[A];
    jx = addc<cx(A)>(jx, g[A]);
    jy = addc<cy(A)>(jy, g[A]);
    jz = addc<cz(A)>(jz, g[A]);
}
template <typename T, int... As>
__device__ __forceinline__ void moments_all(const T (&g)[Q19], T &d, T &jx, T &jy, T &jz)
{
    (moment_one<As>(g, d, jx, jy, jz), ...);
}
// drho = sum_a g_a and j = sum_a e_a g_a
template <typename T> __device__ __forceinline__ void moments19(const T (&g)[Q19], T &d, T &jx, T &jy, T &jz)
{
    d = T(0);
    jx = jy = jz = T(0);
    moments_all<T, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18>(g, d, jx, jy, jz);
}

template <int A, typename T>
__device__ __forceinline__ void relax_one(T (&g)[Q19], T drho, T ux, T uy, T uz, T om)
{
    T eu = T(0);
    eu = addc<cx(A)>(eu, ux);
    eu = addc<cy(A)>(eu, uy);
    eu = addc<cz(A)>(eu, uz);
    const T geq = T(w19(A)) * (drho + eu);                // ux, uy, uz carry the factor 3 already
    g[A] = fma(om, geq - g[A], g[A]);
}
template <typename T, int... As>
__device__ __forceinline__ void relax_all(T (&g)[Q19], T drho, T ux, T uy, T uz, T om)
{
    (relax_one<As>(g, drho, ux, uy, uz, om), ...);
}

template <typename T>
__global__ void __launch_bounds__(256) step3d_kernel(Step3Args<T> a)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= a.nx) return;
    const T *__restrict__ src = a.src;
    T *__restrict__ dst = a.dst;
    const Nbr nb = neighbours(x, y, z, a.nx, a.ny, a.nz);
    T g[Q19];
    pull19(src, a.plane, nb, g);
    const int64_t c = nb.z[1] + nb.y[1] + x;
    const T e = __ldg(a.coef + c);
    T drho, jx, jy, jz;
    moments19(g, drho, jx, jy, jz);
    const T rho = T(1) + drho;
    const T rx = fma(a.hgx, rho, jx), ry = fma(a.hgy, rho, jy), rz = fma(a.hgz, rho, jz);
    const T rux = fma(-e, rx, rx), ruy = fma(-e, ry, ry), ruz = fma(-e, rz, rz);       // Eq. 6 times rho
    // 3 rho u_eq (Eq. 16 times 3 rho), so that g_eq = w (drho + e . (3 rho u_eq))
    const T u3x = T(3) * fma(a.two_tau, rux, a.omt * jx);
    const T u3y = T(3) * fma(a.two_tau, ruy, a.omt * jy);
    const T u3z = T(3) * fma(a.two_tau, ruz, a.omt * jz);
    relax_all<T, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18>(g, drho, u3x, u3y, u3z, a.omega);
#pragma unroll
    for (int q = 0; q < Q19; ++q) dst[q * a.plane + c] = g[q];
}

// Density and flow velocity (Eq. 15) of the streamed state, optional FP64 block sums of u.
template <typename T>
__global__ void __launch_bounds__(128) fields3d_kernel(Step3Args<T> a, float *rho_o, float *u_o, float *v_o,
                                                       float *w_o, double *partials)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    double su = 0.0, sv = 0.0, sw = 0.0;
    if (x < a.nx) {
        const Nbr nb = neighbours(x, y, z, a.nx, a.ny, a.nz);
        T g[Q19];
        pull19(a.src, a.plane, nb, g);
        const int64_t c = nb.z[1] + nb.y[1] + x;
        const T e = a.coef[c];
        T drho, jx, jy, jz;
        moments19(g, drho, jx, jy, jz);
        const T rho = T(1) + drho;
        const T rx = fma(a.hgx, rho, jx), ry = fma(a.hgy, rho, jy), rz = fma(a.hgz, rho, jz);
        const T ux = fma(-e, rx, rx) / rho, uy = fma(-e, ry, ry) / rho, uz = fma(-e, rz, rz) / rho;
        if (rho_o) rho_o[c] = (float)rho;
        if (u_o) u_o[c] = (float)ux;
        if (v_o) v_o[c] = (float)uy;
        if (w_o) w_o[c] = (float)uz;
        su = ux;
        sv = uy;
        sw = uz;
    }
    if (!partials) return;
    // fixed-order block sum: warp shuffles, then warp 0 over the 4 warp sums
    __shared__ double ws[3][4];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        su += __shfl_down_sync(0xffffffffu, su, off);
        sv += __shfl_down_sync(0xffffffffu, sv, off);
        sw += __shfl_down_sync(0xffffffffu, sw, off);
    }
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        ws[0][wid] = su;
        ws[1][wid] = sv;
        ws[2][wid] = sw;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const double s = (ws[threadIdx.x][0] + ws[threadIdx.x][1]) + (ws[threadIdx.x][2] + ws[threadIdx.x][3]);
        const int64_t b = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        partials[3 * b + threadIdx.x] = s;
    }
}

// One block: each thread sums a fixed stride of the partials, then a fixed tree.
__global__ void __launch_bounds__(1024) reduce3_kernel(const double *partials, int64_t nb, double scale, double *out)
{
    __shared__ double s[3][1024];
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int64_t b = threadIdx.x; b < nb; b += 1024) {
        a0 += partials[3 * b];
        a1 += partials[3 * b + 1];
        a2 += partials[3 * b + 2];
    }
    s[0][threadIdx.x] = a0;
    s[1][threadIdx.x] = a1;
    s[2][threadIdx.x] = a2;
    __syncthreads();
    for (int h = 512; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int k = 0; k < 3; ++k) s[k][threadIdx.x] += s[k][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 3) out[threadIdx.x] = s[threadIdx.x][0] * scale;
}

// e = eps nu / (2 kappa + eps nu) per cell; flags bit 0: kappa NaN or negative
template <typename T>
__global__ void __launch_bounds__(256) coef3d_kernel(const float *kappa, T *coef, int64_t n, double eps_nu, unsigned *flags)
{
    unsigned bad = 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float k = kappa[i];
        double e;
        if (!(k >= 0.0f)) { bad = 1u; e = 1.0; }
        else if (eps_nu == 0.0 || isinf(k)) e = 0.0;
        else if (k == 0.0f) e = 1.0;
        else e = eps_nu / (2.0 * (double)k + eps_nu);
        coef[i] = (T)e;
    }
    if (bad) atomicOr(flags, 1u);
}

}  // namespace
}  // namespace lbm

struct lbm3d_grid {
    lbm3d_params p;
    int dev = 0;
    cudaStream_t st = nullptr;
    void *buf[2] = {nullptr, nullptr};
    void *coef = nullptr;
    double *partials = nullptr, *mean = nullptr;
    unsigned *flags = nullptr;
    int cur = 0;
    int64_t n = 0, plane = 0, nblocks = 0;
    size_t esz = 4;
};

using namespace lbm;

namespace {

template <typename T>
Step3Args<T> args3(const lbm3d_grid *g, int src)
{
    Step3Args<T> a;
    a.src = static_cast<const T *>(g->buf[src]);
    a.dst = static_cast<T *>(g->buf[1 - src]);
    a.coef = static_cast<const T *>(g->coef);
    a.nx = g->p.nx;
    a.ny = g->p.ny;
    a.nz = g->p.nz;
    a.plane = g->plane;
    a.omega = (T)(1.0 / g->p.tau);
    a.two_tau = (T)(2.0 * g->p.tau);
    a.omt = (T)(1.0 - 2.0 * g->p.tau);
    a.hgx = (T)(0.5 * g->p.eps * g->p.gx);
    a.hgy = (T)(0.5 * g->p.eps * g->p.gy);
    a.hgz = (T)(0.5 * g->p.eps * g->p.gz);
    return a;
}

dim3 grid3(const lbm3d_grid *g, int threads) { return dim3((g->p.nx + threads - 1) / threads, g->p.ny, g->p.nz); }

void free3(lbm3d_grid *g)
{
    cudaFree(g->buf[0]);
    cudaFree(g->buf[1]);
    cudaFree(g->coef);
    cudaFree(g->partials);
    cudaFree(g->mean);
    cudaFree(g->flags);
    if (g->st) cudaStreamSynchronize(g->st);
    cudaGetLastError();
    delete g;
}

#define L3_CUDA(call)                                                                            \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            cudaGetLastError();                                                                  \
            return fail(e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s failed: %s", \
                        #call, cudaGetErrorString(e_));                                          \
        }                                                                                        \
    } while (0)

}  // namespace

extern "C" {

lbm_status lbm3d_grid_create(const lbm3d_params *p, const float *kappa_dev, void *cuda_stream, lbm3d_grid **out)
{
    if (!p || !out) return fail(LBM_EINVAL, "params and out must not be NULL");
    *out = nullptr;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->ny > 65535 || p->nz > 65535)
        return fail(LBM_EINVAL, "nx, ny, nz must be >= 1 (ny, nz <= 65535)");
    if (!std::isfinite(p->tau) || p->tau < 0.5) return fail(LBM_EINVAL, "tau must be finite and >= 0.5");
    if (!std::isfinite(p->nu) || !std::isfinite(p->eps) || p->eps < 0.0)
        return fail(LBM_EINVAL, "nu must be finite and eps finite and >= 0");
    if (!std::isfinite(p->gx) || !std::isfinite(p->gy) || !std::isfinite(p->gz))
        return fail(LBM_EINVAL, "G must be finite");
    if (p->storage != LBM_F32 && p->storage != LBM_F64) return fail(LBM_EINVAL, "storage must be LBM_F32 or LBM_F64");
    if (!is_device_ptr(kappa_dev)) return fail(LBM_EINVAL, "kappa_dev must be a device pointer");
    lbm3d_grid *g = new lbm3d_grid;
    g->p = *p;
    cudaGetDevice(&g->dev);
    g->st = static_cast<cudaStream_t>(cuda_stream);
    g->n = (int64_t)p->nx * p->ny * p->nz;
    g->plane = (g->n + 63) / 64 * 64;
    g->esz = p->storage == LBM_F64 ? 8 : 4;
    const dim3 gr = grid3(g, 128);
    g->nblocks = (int64_t)gr.x * gr.y * gr.z;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaMalloc(&g->buf[k], Q19 * g->plane * g->esz);
    if (e == cudaSuccess) e = cudaMalloc(&g->coef, g->n * g->esz);
    if (e == cudaSuccess) e = cudaMalloc(&g->partials, sizeof(double) * 3 * g->nblocks);
    if (e == cudaSuccess) e = cudaMalloc(&g->mean, sizeof(double) * 3);
    if (e == cudaSuccess) e = cudaMalloc(&g->flags, sizeof(unsigned));
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaMemsetAsync(g->buf[k], 0, Q19 * g->plane * g->esz, g->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->flags, 0, sizeof(unsigned), g->st);
    if (e != cudaSuccess) {
        free3(g);
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "3-D grid allocation: %s",
                    cudaGetErrorString(e));
    }
    const double nu = p->nu < 0.0 ? (p->tau - 0.5) / 3.0 : p->nu;
    const int nb = (int)std::min<int64_t>((g->n + 255) / 256, 8192);
    if (g->esz == 8)
        coef3d_kernel<double><<<nb, 256, 0, g->st>>>(kappa_dev, static_cast<double *>(g->coef), g->n, p->eps * nu, g->flags);
    else
        coef3d_kernel<float><<<nb, 256, 0, g->st>>>(kappa_dev, static_cast<float *>(g->coef), g->n, p->eps * nu, g->flags);
    count_launches(1);
    unsigned flags = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, g->flags, sizeof flags, cudaMemcpyDeviceToHost, g->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
    if (e != cudaSuccess) {
        free3(g);
        return fail(LBM_ECUDA, "3-D coefficient pass: %s", cudaGetErrorString(e));
    }
    if (flags) {
        free3(g);
        return fail(LBM_EINVAL, "kappa holds NaN or negative values");
    }
    *out = g;
    return LBM_OK;
}

lbm_status lbm3d_grid_destroy(lbm3d_grid *g)
{
    if (g) free3(g);
    return LBM_OK;
}

lbm_status lbm3d_step(lbm3d_grid *g, int64_t steps)
{
    if (!g) return fail(LBM_EINVAL, "grid is NULL");
    if (steps < 0) return fail(LBM_EINVAL, "steps must be >= 0");
    const dim3 gr = grid3(g, 256);
    for (int64_t s = 0; s < steps; ++s) {
        if (g->esz == 8) step3d_kernel<double><<<gr, 256, 0, g->st>>>(args3<double>(g, g->cur));
        else step3d_kernel<float><<<gr, 256, 0, g->st>>>(args3<float>(g, g->cur));
        g->cur = 1 - g->cur;
    }
    count_launches(steps);
    L3_CUDA(cudaGetLastError());
    L3_CUDA(cudaStreamSynchronize(g->st));
    return LBM_OK;
}

lbm_status lbm3d_get_fields(lbm3d_grid *g, float *rho_dev, float *u_dev, float *v_dev, float *w_dev)
{
    if (!g) return fail(LBM_EINVAL, "grid is NULL");
    for (const float *q : {rho_dev, u_dev, v_dev, w_dev})
        if (q && !is_device_ptr(q)) return fail(LBM_EINVAL, "field outputs must be device pointers");
    if (g->esz == 8)
        fields3d_kernel<double><<<grid3(g, 128), 128, 0, g->st>>>(args3<double>(g, g->cur), rho_dev, u_dev, v_dev, w_dev, nullptr);
    else
        fields3d_kernel<float><<<grid3(g, 128), 128, 0, g->st>>>(args3<float>(g, g->cur), rho_dev, u_dev, v_dev, w_dev, nullptr);
    count_launches(1);
    L3_CUDA(cudaGetLastError());
    L3_CUDA(cudaStreamSynchronize(g->st));
    return LBM_OK;
}

lbm_status lbm3d_mean_velocity(lbm3d_grid *g, double out_mean_uvw[3])
{
    if (!g || !out_mean_uvw) return fail(LBM_EINVAL, "grid and out must not be NULL");
    if (g->esz == 8)
        fields3d_kernel<double><<<grid3(g, 128), 128, 0, g->st>>>(args3<double>(g, g->cur), nullptr, nullptr, nullptr, nullptr, g->partials);
    else
        fields3d_kernel<float><<<grid3(g, 128), 128, 0, g->st>>>(args3<float>(g, g->cur), nullptr, nullptr, nullptr, nullptr, g->partials);
    reduce3_kernel<<<1, 1024, 0, g->st>>>(g->partials, g->nblocks, 1.0 / (double)g->n, g->mean);
    count_launches(2);
    L3_CUDA(cudaGetLastError());
    L3_CUDA(cudaMemcpyAsync(out_mean_uvw, g->mean, sizeof(double) * 3, cudaMemcpyDeviceToHost, g->st));
    L3_CUDA(cudaStreamSynchronize(g->st));
    return LBM_OK;
}

}  // extern "C"
