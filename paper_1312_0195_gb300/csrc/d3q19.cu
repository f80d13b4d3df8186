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


#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <vector>

namespace lbm {

lbm_status fail(lbm_status s, const char *fmt, ...);
bool is_device_ptr(const void *p);
void count_launches(int64_t n);
double local_time_limit();

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

// Storage type T and compute type: FP16 storage (scaled deviations) computes in FP32.
template <typename T> struct Comp3 { using type = T; };
template <> struct Comp3<__half> { using type = float; };
__device__ __forceinline__ float to_comp(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_comp(float v) { return v; }
__device__ __forceinline__ double to_comp(double v) { return v; }
template <typename T, typename C> __device__ __forceinline__ T from_comp(C v) { return (T)v; }
template <> __device__ __forceinline__ __half from_comp<__half, float>(float v) { return __float2half_rn(v); }

template <typename T>
struct Step3Args {
    using C = typename Comp3<T>::type;
    const T *src;
    T *dst;
    const C *coef;          // e per cell, or the 9 planes E_ij of a tensor K* (E_ij at (3 i + j) plane)
    int nx, ny, nz;
    int64_t plane;          // elements per population (and coefficient) plane
    C omega, k_ru, k_j, hgx, hgy, hgz;   // 1/tau, 6 tau, 3 (1 - 2 tau), eps G / 2
    C rho0, inv_scale;      // the storage scale S: populations are S g, so rho = S + S drho
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

template <int A, typename T, typename C>
__device__ __forceinline__ void pull_one(const T *__restrict__ src, int64_t plane, const Nbr &nb, C (&g)[Q19])
{
    g[A] = to_comp(__ldg(src + A * plane + nb.template from<A>()));
}
template <typename T, typename C, int... As>
__device__ __forceinline__ void pull_all(const T *src, int64_t plane, const Nbr &nb, C (&g)[Q19])
{
    (pull_one<As>(src, plane, nb, g), ...);
}
template <typename T, typename C>
__device__ __forceinline__ void pull19(const T *src, int64_t plane, const Nbr &nb, C (&g)[Q19])
{
    pull_all<T, C, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18>(src, plane, nb, g);
}

// Moments through the nine opposite pairs (a, a + 1): s_p = g_a + g_{a+1} and
// d_p = g_a - g_{a+1}. The pairs point along x, y, z, (x, y), (x, -y), (x, z),
// (x, -z), (y, z) and (y, -z), which the asserts tie to the velocity table.
static_assert(cx(1) == 1 && cy(3) == 1 && cz(5) == 1, "face pairs");
static_assert(cx(7) == 1 && cy(7) == 1 && cx(9) == 1 && cy(9) == -1, "xy edge pairs");
static_assert(cx(11) == 1 && cz(11) == 1 && cx(13) == 1 && cz(13) == -1, "xz edge pairs");
static_assert(cy(15) == 1 && cz(15) == 1 && cy(17) == 1 && cz(17) == -1, "yz edge pairs");
static_assert(cx(2) == -1 && cy(4) == -1 && cz(6) == -1 && cx(8) == -1 && cy(8) == -1 && cx(10) == -1 &&
                  cy(10) == 1 && cx(12) == -1 && cz(12) == -1 && cx(14) == -1 && cz(14) == 1 && cy(16) == -1 &&
                  cz(16) == -1 && cy(18) == -1 && cz(18) == 1,
              "a + 1 is opposite to a");
static_assert(cz(1) == 0 && cz(7) == 0 && cz(9) == 0 && cy(11) == 0 && cy(13) == 0 && cx(15) == 0 && cx(17) == 0,
              "edge pairs lie in their planes");

// drho = sum_a g_a and j = sum_a e_a g_a
template <typename T> __device__ __forceinline__ void moments19(const T (&g)[Q19], T &drho, T &jx, T &jy, T &jz)
{
    T s[9], d[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        s[p] = g[2 * p + 1] + g[2 * p + 2];
        d[p] = g[2 * p + 1] - g[2 * p + 2];
    }
    drho = g[0] + ((((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]))) + s[8]);
    jx = d[0] + ((d[3] + d[4]) + (d[5] + d[6]));
    jy = d[1] + ((d[3] - d[4]) + (d[7] + d[8]));
    jz = d[2] + ((d[5] - d[6]) + (d[7] - d[8]));
}

// BGK (Eq. 13) in difference form for an opposite pair whose equilibria (Eq. 2) are
// w drho +/- w eu: g + om (w drho - g +/- w eu), with wd = w drho.
template <typename T> __device__ __forceinline__ void relax_pair(T &gp, T &gm, T wd, T w, T eu, T om)
{
    gp = fma(om, fma(w, eu, wd - gp), gp);
    gm = fma(om, fma(-w, eu, wd - gm), gm);
}
// FP32 pair in packed f32x2 instructions, lane by lane the operations of relax_pair:
// fma(g, -1, wd) is wd - g rounded once, then fma(+/-w, eu, .) and fma(om, ., g).
__device__ __forceinline__ void relax_pair2(float &gp, float &gm, float2 wd, float2 wpm, float eu, float2 om)
{
    const float2 g = make_float2(gp, gm);
    const float2 t = __ffma2_rn(g, make_float2(-1.0f, -1.0f), wd);
    const float2 r = __ffma2_rn(om, __ffma2_rn(wpm, make_float2(eu, eu), t), g);
    gp = r.x;
    gm = r.y;
}

// All 19 populations; ux, uy, uz are 3 rho u_eq (Eq. 16 times 3), so e_a . u is the eu above.
template <typename T> __device__ __forceinline__ void relax19(T (&g)[Q19], T drho, T ux, T uy, T uz, T om)
{
    const T w0 = T(1.0 / 3.0), w1 = T(1.0 / 18.0), w2 = T(1.0 / 36.0);
    const T d1 = w1 * drho, d2 = w2 * drho;
    g[0] = fma(om, fma(w0, drho, -g[0]), g[0]);
    if constexpr (sizeof(T) == 4) {
        const float2 o2 = make_float2(om, om), d12 = make_float2(d1, d1), d22 = make_float2(d2, d2);
        const float2 w12 = make_float2(w1, -w1), w22 = make_float2(w2, -w2);
        relax_pair2(g[1], g[2], d12, w12, ux, o2);
        relax_pair2(g[3], g[4], d12, w12, uy, o2);
        relax_pair2(g[5], g[6], d12, w12, uz, o2);
        relax_pair2(g[7], g[8], d22, w22, ux + uy, o2);
        relax_pair2(g[9], g[10], d22, w22, ux - uy, o2);
        relax_pair2(g[11], g[12], d22, w22, ux + uz, o2);
        relax_pair2(g[13], g[14], d22, w22, ux - uz, o2);
        relax_pair2(g[15], g[16], d22, w22, uy + uz, o2);
        relax_pair2(g[17], g[18], d22, w22, uy - uz, o2);
    } else {
        relax_pair(g[1], g[2], d1, w1, ux, om);
        relax_pair(g[3], g[4], d1, w1, uy, om);
        relax_pair(g[5], g[6], d1, w1, uz, om);
        relax_pair(g[7], g[8], d2, w2, ux + uy, om);
        relax_pair(g[9], g[10], d2, w2, ux - uy, om);
        relax_pair(g[11], g[12], d2, w2, ux + uz, om);
        relax_pair(g[13], g[14], d2, w2, ux - uz, om);
        relax_pair(g[15], g[16], d2, w2, uy + uz, om);
        relax_pair(g[17], g[18], d2, w2, uy - uz, om);
    }
}

// The whole collision of one cell: moments, r = j + (eps G / 2) rho, rho u = (1 - e) r
// (Eq. 6 times rho), 3 rho u_eq = 6 tau rho u + 3 (1 - 2 tau) j (Eq. 16 times 3), relax.
template <typename T>
__device__ __forceinline__ void collide19(T (&g)[Q19], T e, T hgx, T hgy, T hgz, T k_ru, T k_j, T om, T rho0 = T(1))
{
    T drho, jx, jy, jz;
    moments19(g, drho, jx, jy, jz);
    const T rho = rho0 + drho;
    const T rx = fma(hgx, rho, jx), ry = fma(hgy, rho, jy), rz = fma(hgz, rho, jz);
    const T rux = fma(-e, rx, rx), ruy = fma(-e, ry, ry), ruz = fma(-e, rz, rz);
    relax19(g, drho, fma(k_ru, rux, k_j * jx), fma(k_ru, ruy, k_j * jy), fma(k_ru, ruz, k_j * jz), om);
}

// Coarse cell with a tensor K* (Eq. 18 in Eq. 15): rho u = (I + c K*^-1)^-1 r = r - E r with
// E = c (K* + c I)^-1 and c = eps nu / 2 (for K* = kappa I, E = e I).
template <typename T>
__device__ __forceinline__ void drag_tensor(const T (&E)[9], T rx, T ry, T rz, T &rux, T &ruy, T &ruz)
{
    rux = rx - fma(E[0], rx, fma(E[1], ry, E[2] * rz));
    ruy = ry - fma(E[3], rx, fma(E[4], ry, E[5] * rz));
    ruz = rz - fma(E[6], rx, fma(E[7], ry, E[8] * rz));
}
template <typename T>
__device__ __forceinline__ void collide19_tensor(T (&g)[Q19], const T (&E)[9], T hgx, T hgy, T hgz, T k_ru, T k_j,
                                                 T om, T rho0 = T(1))
{
    T drho, jx, jy, jz, rux, ruy, ruz;
    moments19(g, drho, jx, jy, jz);
    const T rho = rho0 + drho;
    drag_tensor(E, fma(hgx, rho, jx), fma(hgy, rho, jy), fma(hgz, rho, jz), rux, ruy, ruz);
    relax19(g, drho, fma(k_ru, rux, k_j * jx), fma(k_ru, ruy, k_j * jy), fma(k_ru, ruz, k_j * jz), om);
}

template <typename T, bool TENSOR>
__global__ void __launch_bounds__(256) step3d_kernel(Step3Args<T> a)
{
    using C = typename Comp3<T>::type;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= a.nx) return;
    const T *__restrict__ src = a.src;
    T *__restrict__ dst = a.dst;
    const Nbr nb = neighbours(x, y, z, a.nx, a.ny, a.nz);
    C g[Q19];
    pull19(src, a.plane, nb, g);
    const int64_t c = nb.z[1] + nb.y[1] + x;
    if constexpr (TENSOR) {
        C E[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) E[k] = __ldg(a.coef + k * a.plane + c);
        collide19_tensor(g, E, a.hgx, a.hgy, a.hgz, a.k_ru, a.k_j, a.omega, a.rho0);
    } else {
        collide19(g, __ldg(a.coef + c), a.hgx, a.hgy, a.hgz, a.k_ru, a.k_j, a.omega, a.rho0);
    }
#pragma unroll
    for (int q = 0; q < Q19; ++q) dst[q * a.plane + c] = from_comp<T>(g[q]);
}

// Density and flow velocity (Eq. 15) of the streamed state, optional FP64 block sums of u.
template <typename T, bool TENSOR>
__global__ void __launch_bounds__(128) fields3d_kernel(Step3Args<T> a, float *rho_o, float *u_o, float *v_o,
                                                       float *w_o, double *partials)
{
    using C = typename Comp3<T>::type;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    double su = 0.0, sv = 0.0, sw = 0.0;
    if (x < a.nx) {
        const Nbr nb = neighbours(x, y, z, a.nx, a.ny, a.nz);
        C g[Q19];
        pull19(a.src, a.plane, nb, g);
        const int64_t c = nb.z[1] + nb.y[1] + x;
        C drho, jx, jy, jz;
        moments19(g, drho, jx, jy, jz);
        const C rho = a.rho0 + drho;        // scaled by S, which cancels in u = rho u / rho
        const C rx = fma(a.hgx, rho, jx), ry = fma(a.hgy, rho, jy), rz = fma(a.hgz, rho, jz);
        C rux, ruy, ruz;
        if constexpr (TENSOR) {
            C E[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) E[k] = a.coef[k * a.plane + c];
            drag_tensor(E, rx, ry, rz, rux, ruy, ruz);
        } else {
            const C e = a.coef[c];
            rux = fma(-e, rx, rx);
            ruy = fma(-e, ry, ry);
            ruz = fma(-e, rz, rz);
        }
        const C ux = rux / rho, uy = ruy / rho, uz = ruz / rho;
        if (rho_o) rho_o[c] = (float)fma(drho, a.inv_scale, C(1));
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
    unsigned bad = 0u, kmax = 0u;    // kmax: bits of the largest finite kappa (ordered like the floats, all >= 0)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float k = kappa[i];
        double e;
        if (!(k >= 0.0f)) { bad = 1u; e = 1.0; }
        else if (eps_nu == 0.0 || isinf(k)) e = 0.0;
        else if (k == 0.0f) e = 1.0;
        else e = eps_nu / (2.0 * (double)k + eps_nu);
        if (k >= 0.0f && !isinf(k)) kmax = max(kmax, __float_as_uint(k));
        coef[i] = (T)e;
    }
    if (bad) atomicOr(flags, 1u);
    if (kmax) atomicMax(flags + 1, kmax);
}

// E = c (K + c I)^-1 per coarse cell, K = scale keff (fine lattice units to coarse),
// c = eps nu / 2, by cofactors; flags bit 0: keff not finite, bit 1: K + c I singular.
template <typename T>
__global__ void __launch_bounds__(256) coef3d_tensor_kernel(const double *keff, double scale, T *coef, int64_t n,
                                                            int64_t plane, double c, unsigned *flags)
{
    unsigned bad = 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double m[9], E[9];
        bool finite = true;
        for (int k = 0; k < 9; ++k) {
            m[k] = scale * keff[9 * i + k] + (k % 4 == 0 ? c : 0.0);
            finite = finite && isfinite(m[k]);
        }
        for (int k = 0; k < 9; ++k) E[k] = 0.0;
        if (!finite) {
            bad |= 1u;
        } else if (c != 0.0) {
            const double c00 = m[4] * m[8] - m[5] * m[7], c01 = m[5] * m[6] - m[3] * m[8];
            const double c02 = m[3] * m[7] - m[4] * m[6];
            const double det = m[0] * c00 + m[1] * c01 + m[2] * c02;
            if (!(fabs(det) > 0.0)) {
                bad |= 2u;
            } else {
                const double f = c / det;     // E = c adj(m) / det(m); adj is the transposed cofactor matrix
                E[0] = f * c00;
                E[1] = f * (m[2] * m[7] - m[1] * m[8]);
                E[2] = f * (m[1] * m[5] - m[2] * m[4]);
                E[3] = f * c01;
                E[4] = f * (m[0] * m[8] - m[2] * m[6]);
                E[5] = f * (m[2] * m[3] - m[0] * m[5]);
                E[6] = f * c02;
                E[7] = f * (m[1] * m[6] - m[0] * m[7]);
                E[8] = f * (m[0] * m[4] - m[1] * m[3]);
            }
        }
        for (int k = 0; k < 9; ++k) coef[k * plane + i] = (T)E[k];
    }
    if (bad) atomicOr(flags, bad);
}

// Mean of a float [nz][ny][nx] field over block^3 cubes, FP64 in a fixed order.
__global__ void __launch_bounds__(256) block_average3_kernel(const float *in, int nx, int ny, int nz, int r,
                                                             float *out)
{
    const int cx = nx / r, cy = ny / r, cz = nz / r;
    const int64_t nb = (int64_t)cx * cy * cz;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
        const int I = (int)(b % cx), J = (int)((b / cx) % cy), K = (int)(b / ((int64_t)cx * cy));
        double s = 0.0;
        for (int z = K * r; z < (K + 1) * r; ++z)
            for (int y = J * r; y < (J + 1) * r; ++y) {
                const float *row = in + ((int64_t)z * ny + y) * nx + (int64_t)I * r;
                for (int x = 0; x < r; ++x) s += (double)row[x];
            }
        out[b] = (float)(s / ((double)r * r * r));
    }
}

// ------------------------------------------------------------------------
// Three-dimensional local problems (Section 3 on the D3Q19 lattice): job j is leaf
// j / 3 driven along axis j % 3, an s^3 periodic cube stored as the j-th block of s^3
// cells in every population plane. All jobs of one leaf size step together; a job
// that has met the stop rule is skipped.
template <typename T>
struct Local3Args {
    const T *src;
    T *dst;
    const T *coef;          // e per cell of every job
    const int *list;        // [blocks along y] the jobs still running
    int s, m;               // side of the simulated cube (leaf + 2 margin), margin
    int64_t s3, plane;
    T omega, k_ru, k_j, hg;      // 1/tau, 6 tau, 3 (1 - 2 tau); hg = eps G / 2 along the job's drive axis
};

// Neighbours within cube `job` (periodic on the cube): base offset folded into the z row.
__device__ __forceinline__ Nbr cube_neighbours(int x, int y, int z, int s, int64_t base)
{
    Nbr n;
    const int64_t pz = (int64_t)s * s;
    n.x[0] = x == 0 ? s - 1 : x - 1;
    n.x[1] = x;
    n.x[2] = x + 1 == s ? 0 : x + 1;
    n.y[0] = (int64_t)(y == 0 ? s - 1 : y - 1) * s;
    n.y[1] = (int64_t)y * s;
    n.y[2] = (int64_t)(y + 1 == s ? 0 : y + 1) * s;
    n.z[0] = base + (z == 0 ? s - 1 : z - 1) * pz;
    n.z[1] = base + z * pz;
    n.z[2] = base + (z + 1 == s ? 0 : z + 1) * pz;
    return n;
}

template <typename T>
__global__ void __launch_bounds__(256) local3d_step_kernel(Local3Args<T> a)
{
    const int job = a.list[blockIdx.y];
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.s3) return;
    const int s = a.s;
    const int x = (int)(c % s), yz = (int)(c / s), y = yz % s, z = yz / s;
    const int64_t base = (int64_t)job * a.s3;
    const T *__restrict__ src = a.src;
    T *__restrict__ dst = a.dst;
    const Nbr nb = cube_neighbours(x, y, z, s, base);
    T g[Q19];
    pull19(src, a.plane, nb, g);
    const T e = __ldg(a.coef + base + c);
    const int d = job % 3;
    collide19(g, e, d == 0 ? a.hg : T(0), d == 1 ? a.hg : T(0), d == 2 ? a.hg : T(0), a.k_ru, a.k_j, a.omega);
#pragma unroll
    for (int q = 0; q < Q19; ++q) dst[q * a.plane + base + c] = g[q];
}

struct Check3 {
    int t, k, regular;      // steps done, check interval, t is a multiple of k
    int64_t max_steps;
    double tol, nu_over_g;
    int *active;
    double *prev;           // [njobs] driven mean velocity at the previous regular check
    const int *job_leaf;    // [njobs] leaf index of the job
    double *keff;           // [n][9]
    int *status, *steps;    // [n], [n][3] or nullptr
    int *nactive;
};

// One block per job: mean flow velocity over the cube (pulled state, Eq. 15) in FP64 in a
// fixed order, then the stop rule on the driven component; a finished job writes column d of K*.
template <typename T>
__global__ void __launch_bounds__(256) local3d_check_kernel(Local3Args<T> a, Check3 ck)
{
    const int job = a.list[blockIdx.x];
    const int s = a.s, d = job % 3;
    const int64_t base = (int64_t)job * a.s3;
    double m0 = 0.0, m1 = 0.0, m2 = 0.0;
    const int lo = a.m, hi = s - a.m;       // the inner leaf of an oversampled cube
    for (int64_t c = threadIdx.x; c < a.s3; c += blockDim.x) {
        const int x = (int)(c % s), yz = (int)(c / s), y = yz % s, z = yz / s;
        if (x < lo || x >= hi || y < lo || y >= hi || z < lo || z >= hi) continue;
        const Nbr nb = cube_neighbours(x, y, z, s, base);
        T g[Q19];
        pull19(a.src, a.plane, nb, g);
        const T e = a.coef[base + c];
        T drho, jx, jy, jz;
        moments19(g, drho, jx, jy, jz);
        const T rho = T(1) + drho;
        const T rx = d == 0 ? fma(a.hg, rho, jx) : jx;
        const T ry = d == 1 ? fma(a.hg, rho, jy) : jy;
        const T rz = d == 2 ? fma(a.hg, rho, jz) : jz;
        m0 += (double)(fma(-e, rx, rx) / rho);
        m1 += (double)(fma(-e, ry, ry) / rho);
        m2 += (double)(fma(-e, rz, rz) / rho);
    }
    __shared__ double sh[3][256];
    sh[0][threadIdx.x] = m0;
    sh[1][threadIdx.x] = m1;
    sh[2][threadIdx.x] = m2;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    double m[3];
    const double sl = s - 2 * a.m;
    for (int q = 0; q < 3; ++q) m[q] = sh[q][0] / (sl * sl * sl);
    const double cur = m[d];
    int st = -1;
    if (ck.regular) {
        if (ck.tol > 0.0 && ck.t > ck.k && fabs(cur - ck.prev[job]) <= ck.tol * ck.k * fabs(cur)) st = LBM_OK;
        ck.prev[job] = cur;
    }
    if (st < 0 && ck.t >= ck.max_steps) st = ck.tol > 0.0 ? LBM_ENOTCONV : LBM_OK;
    if (st < 0) return;
    const int leaf = ck.job_leaf[job];
    for (int i = 0; i < 3; ++i) ck.keff[9 * (int64_t)leaf + 3 * i + d] = ck.nu_over_g * m[i];   // Eq. 17
    if (ck.steps) ck.steps[3 * (int64_t)leaf + d] = ck.t;
    if (st != LBM_OK) atomicMax(&ck.status[leaf], st);
    ck.active[job] = 0;
    atomicSub(ck.nactive, 1);
}

// Rebuilds the list of running jobs in job order: one block, each thread owns a contiguous
// run of jobs, a block-wide exclusive scan of the counts gives the write offsets.
__global__ void __launch_bounds__(1024) local3d_compact_kernel(const int *active, int njobs, int *list)
{
    __shared__ int cnt[1024];
    const int per = (njobs + 1023) / 1024;
    const int j0 = threadIdx.x * per, j1 = min(njobs, j0 + per);
    int n = 0;
    for (int j = j0; j < j1; ++j) n += active[j] != 0;
    cnt[threadIdx.x] = n;
    __syncthreads();
    for (int h = 1; h < 1024; h <<= 1) {      // Hillis-Steele inclusive scan
        const int v = threadIdx.x >= h ? cnt[threadIdx.x - h] : 0;
        __syncthreads();
        cnt[threadIdx.x] += v;
        __syncthreads();
    }
    int o = cnt[threadIdx.x] - n;
    for (int j = j0; j < j1; ++j)
        if (active[j]) list[o++] = j;
}

// ------------------------------------------------------------------------
// Cluster-resident local problems. One job per thread-block cluster of C CTAs: the
// s^3 cube is split along z into slabs of L = ceil(s / C) layers, CTA r holding
// layers [r L, r L + L) of all 19 populations and of e in shared memory, so a job
// never touches HBM after its first step. One copy of the populations is updated
// in place with the AA pattern: a step of even type reads cell x's own slots and
// writes each post-collision value to the opposite slot of x; a step of odd type
// reads slot opp(a) of x - e_a and writes slot a of x + e_a. Either way a thread
// touches only locations no other thread touches in that step, and after n steps
// the streamed state is what the next step reads. Neighbours on a slab boundary
// sit in a peer CTA and go through distributed shared memory; one cluster barrier
// ends every step. The checks every k steps sum the flow velocity in FP64 per
// thread, per warp by a fixed shuffle tree, per CTA in warp order and per
// cluster in rank order, so every CTA takes the same stop decision.
template <typename T>
struct Clu3Args {
    const float *kappa;
    int nx, ny, nz;
    const int4 *leaves;     // all leaves of the call
    const int *ids;         // [njobs / 3] leaf indices of this size
    int njobs, s, L;        // s: side of the simulated cube (leaf + 2 margin)
    int m;                  // oversampling margin: the mean is over the inner (s - 2 m)^3 leaf
    T omega, k_ru, k_j, hg;      // 1/tau, 6 tau, 3 (1 - 2 tau), eps G / 2
    double eps_nu, nu_over_g, tol;
    int k;
    int64_t max_steps;
    double *keff;
    int *status, *steps;
    unsigned long long *t_start;   // first globaltimer reading of the launch (0 before)
    int *abort_flag;
    unsigned long long time_limit_ns;
};

__device__ __forceinline__ unsigned long long globaltimer3()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr __host__ __device__ int opp19(int a) { return a == 0 ? 0 : ((a & 1) ? a + 1 : a - 1); }

// Distributed shared memory through 32-bit shared::cluster addresses
__device__ __forceinline__ uint32_t cluster_addr(const void *own_smem, uint32_t rank)
{
    uint32_t d;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(d) : "r"((uint32_t)__cvta_generic_to_shared(own_smem)), "r"(rank));
    return d;
}
__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_size()
{
    uint32_t n;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(n));
    return n;
}
template <typename T> __device__ __forceinline__ T ld_cluster(uint32_t a);
template <> __device__ __forceinline__ float ld_cluster<float>(uint32_t a)
{
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
template <> __device__ __forceinline__ double ld_cluster<double>(uint32_t a)
{
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void st_cluster(uint32_t a, float v)
{
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v));
}
__device__ __forceinline__ void st_cluster(uint32_t a, double v)
{
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v));
}

// Per-cell geometry: cluster addresses of layers z - 1, z, z + 1 (in whichever CTA
// holds them) and the wrapped x and y byte offsets within a layer.
template <typename T>
struct Cell3 {
    uint32_t lz[3];
    uint32_t xo[3], yo[3];
    int c;                 // index within this CTA's slab
    template <int A> __device__ __forceinline__ uint32_t from(uint32_t Pb) const   // slot opp(A) of x - e_A
    {
        return lz[1 - cz(A)] + opp19(A) * Pb + yo[1 - cy(A)] + xo[1 - cx(A)];
    }
    template <int A> __device__ __forceinline__ uint32_t to(uint32_t Pb) const     // slot A of x + e_A
    {
        return lz[1 + cz(A)] + A * Pb + yo[1 + cy(A)] + xo[1 + cx(A)];
    }
};

// PS is the slot stride in cells (compile time, so slot offsets are immediates)
template <bool ODD, int PS, int A, typename T>
__device__ __forceinline__ void aa_read_one(const Cell3<T> &q, const T *own, T (&g)[Q19])
{
    if (ODD) g[A] = ld_cluster<T>(q.template from<A>(PS * (uint32_t)sizeof(T)));
    else g[A] = own[A * PS + q.c];
}
template <bool ODD, int PS, int A, typename T>
__device__ __forceinline__ void aa_write_one(const Cell3<T> &q, T *own, const T (&g)[Q19])
{
    if (ODD) st_cluster(q.template to<A>(PS * (uint32_t)sizeof(T)), g[A]);
    else own[opp19(A) * PS + q.c] = g[A];
}
template <bool ODD, int PS, typename T, int... As>
__device__ __forceinline__ void aa_read(const Cell3<T> &q, const T *own, T (&g)[Q19])
{
    (aa_read_one<ODD, PS, As>(q, own, g), ...);
}
template <bool ODD, int PS, typename T, int... As>
__device__ __forceinline__ void aa_write(const Cell3<T> &q, T *own, const T (&g)[Q19])
{
    (aa_write_one<ODD, PS, As>(q, own, g), ...);
}
template <bool ODD, int PS, typename T>
__device__ __forceinline__ void aa_read19(const Cell3<T> &q, const T *own, T (&g)[Q19])
{
    aa_read<ODD, PS, T, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18>(q, own, g);
}

// moments of g plus the drag-reduced momentum (1 - e) r, r = j + hg rho along the drive axis d
template <typename T>
__device__ __forceinline__ void drag_momentum(const T (&g)[Q19], T e, T hg, int d, T &drho, T &jx, T &jy, T &jz,
                                              T &rux, T &ruy, T &ruz)
{
    moments19(g, drho, jx, jy, jz);
    const T rho = T(1) + drho;
    const T rx = d == 0 ? fma(hg, rho, jx) : jx;
    const T ry = d == 1 ? fma(hg, rho, jy) : jy;
    const T rz = d == 2 ? fma(hg, rho, jz) : jz;
    rux = fma(-e, rx, rx);
    ruy = fma(-e, ry, ry);
    ruz = fma(-e, rz, rz);
}

template <bool ODD, int PS, typename T>
__device__ __forceinline__ void aa_step_cell(const Cell3<T> &q, T *own, T e, const Clu3Args<T> &a, T hgx, T hgy, T hgz)
{
    T g[Q19];
    aa_read19<ODD, PS>(q, own, g);
    collide19(g, e, hgx, hgy, hgz, a.k_ru, a.k_j, a.omega);
    aa_write<ODD, PS, T, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18>(q, own, g);
}

template <bool ODD, int PS, typename T>
__device__ __forceinline__ void aa_velocity_cell(const Cell3<T> &q, const T *own, T e, T hg, int d,
                                                 double &m0, double &m1, double &m2)
{
    T g[Q19];
    aa_read19<ODD, PS>(q, own, g);
    T drho, jx, jy, jz, rux, ruy, ruz;
    drag_momentum(g, e, hg, d, drho, jx, jy, jz, rux, ruy, ruz);
    const T rho = T(1) + drho;
    m0 += (double)(rux / rho);
    m1 += (double)(ruy / rho);
    m2 += (double)(ruz / rho);
}

// cells per thread at most: a slab of P cells needs a block of at least P / CPT threads
template <typename T> __host__ __device__ constexpr int clu3_cpt() { return sizeof(T) == 4 ? 4 : 2; }
template <typename T> __host__ __device__ constexpr int clu3_threads() { return 512; }

// Packed cell: zl << 16 | y << 8 | x, plus CLU3_IN when the cell lies in the inner leaf of an
// oversampled cube (every cell without a margin)
constexpr int CLU3_IN = 1 << 30;

// Cell3 of a packed cell from the table of layer addresses
template <typename T>
__device__ __forceinline__ Cell3<T> cell3_of(int geo, int s, const uint32_t *zb, int z0)
{
    Cell3<T> q;
    const int x = geo & 255, y = (geo >> 8) & 255, zl = (geo >> 16) & 255, z = z0 + zl;
    const uint32_t E = sizeof(T);
    q.c = (zl * s + y) * s + x;
    q.xo[0] = (x == 0 ? s - 1 : x - 1) * E;
    q.xo[1] = x * E;
    q.xo[2] = (x + 1 == s ? 0 : x + 1) * E;
    q.yo[0] = (y == 0 ? s - 1 : y - 1) * s * E;
    q.yo[1] = y * s * E;
    q.yo[2] = (y + 1 == s ? 0 : y + 1) * s * E;
    q.lz[0] = zb[z == 0 ? s - 1 : z - 1];
    q.lz[1] = zb[z];
    q.lz[2] = zb[z + 1 == s ? 0 : z + 1];
    return q;
}

template <typename T, int PS>
__global__ void __launch_bounds__(clu3_threads<T>(), 1) local3d_cluster_kernel(Clu3Args<T> a)
{
    constexpr int CLU3_CPT = clu3_cpt<T>();
    const int C = (int)cluster_size();
    const int r = (int)cluster_rank();
    const int job = (int)(blockIdx.x / (unsigned)C);
    const int leaf = a.ids[job / 3], d = job % 3;
    const int s = a.s, s2 = s * s, L = a.L;
    static_assert(PS % 32 == 0, "slot stride");
    const int z0 = r * L, Lr = max(0, min(L, s - z0));      // this CTA's layers
    const int ncell = Lr * s2;
    const int tid = threadIdx.x, nt = blockDim.x;

    extern __shared__ __align__(16) unsigned char clu3_smem[];
    double *part = reinterpret_cast<double *>(clu3_smem);         // [4]: sums of u, abort
    double *wred = part + 4;                                       // [32][3]
    uint32_t *zb = reinterpret_cast<uint32_t *>(wred + 96);        // [32] layer z of the cube, any CTA
    T *own = reinterpret_cast<T *>(wred + 96 + 16);                // [19][PS] populations, L s^2 <= PS used

    for (int z = tid; z < s; z += nt) zb[z] = cluster_addr(own, z / L) + (uint32_t)((z % L) * s2 * sizeof(T));
    // this thread's cells; e from the leaf's cube of kappa
    const int4 Lf = a.leaves[leaf];
    int geo[CLU3_CPT];
    T ec[CLU3_CPT];
#pragma unroll
    for (int i = 0; i < CLU3_CPT; ++i) {
        const int c = tid + i * nt;
        geo[i] = -1;
        ec[i] = T(0);
        if (c >= ncell) continue;
        const int x = c % s, yz = c / s, y = yz % s, zl = yz / s, z = z0 + zl;
        const int sl = s - 2 * a.m;
        const bool in = x >= a.m && x < a.m + sl && y >= a.m && y < a.m + sl && z >= a.m && z < a.m + sl;
        geo[i] = (zl << 16) | (y << 8) | x | (in ? CLU3_IN : 0);
        // the grown cube starts margin cells before the leaf, wrapping at the field's edges
        int gx = Lf.x - a.m + x, gy = Lf.y - a.m + y, gz = Lf.z - a.m + z;
        gx = gx < 0 ? gx + a.nx : (gx >= a.nx ? gx - a.nx : gx);
        gy = gy < 0 ? gy + a.ny : (gy >= a.ny ? gy - a.ny : gy);
        gz = gz < 0 ? gz + a.nz : (gz >= a.nz ? gz - a.nz : gz);
        const float kv = a.kappa[((int64_t)gz * a.ny + gy) * a.nx + gx];
        double e;
        if (!(kv >= 0.0f)) e = 1.0;
        else if (a.eps_nu == 0.0 || isinf(kv)) e = 0.0;
        else if (kv == 0.0f) e = 1.0;
        else e = a.eps_nu / (2.0 * (double)kv + a.eps_nu);
        ec[i] = (T)e;
#pragma unroll
        for (int q = 0; q < Q19; ++q) own[q * PS + c] = T(0);      // rest: every deviation zero
    }
    unsigned long long t0 = 0;
    if (r == 0 && tid == 0) {
        const unsigned long long now = globaltimer3();
        const unsigned long long prev = atomicCAS(a.t_start, 0ull, now);
        t0 = prev == 0ull ? now : prev;
    }
    cluster_sync_all();

    const int lane = tid & 31, wid = tid >> 5;
    const T hgx = d == 0 ? a.hg : T(0), hgy = d == 1 ? a.hg : T(0), hgz = d == 2 ? a.hg : T(0);
    double prev_u = 0.0;
    int64_t t = 0;
    for (;;) {
        const int64_t nstep = min((int64_t)a.k, a.max_steps - t);
        for (int64_t i = 0; i < nstep; ++i) {
            const bool odd = ((t + i) & 1) != 0;
#pragma unroll
            for (int j = 0; j < CLU3_CPT; ++j) {
                if (geo[j] < 0) continue;
                int gj = geo[j];
                asm volatile("" : "+r"(gj));     // keeps the addresses out of registers between steps
                const Cell3<T> q = cell3_of<T>(gj, s, zb, z0);
                if (odd) aa_step_cell<true, PS>(q, own, ec[j], a, hgx, hgy, hgz);
                else aa_step_cell<false, PS>(q, own, ec[j], a, hgx, hgy, hgz);
            }
            cluster_sync_all();
        }
        t += nstep;

        // mean flow velocity of the streamed state (Eq. 15), FP64 in a fixed order
        double m0 = 0.0, m1 = 0.0, m2 = 0.0;
        const bool odd = (t & 1) != 0;
#pragma unroll
        for (int j = 0; j < CLU3_CPT; ++j) {
            if (geo[j] < 0 || !(geo[j] & CLU3_IN)) continue;
            int gj = geo[j];
            asm volatile("" : "+r"(gj));
            const Cell3<T> q = cell3_of<T>(gj, s, zb, z0);
            if (odd) aa_velocity_cell<true, PS>(q, own, ec[j], a.hg, d, m0, m1, m2);
            else aa_velocity_cell<false, PS>(q, own, ec[j], a.hg, d, m0, m1, m2);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            m0 += __shfl_down_sync(0xffffffffu, m0, o);
            m1 += __shfl_down_sync(0xffffffffu, m1, o);
            m2 += __shfl_down_sync(0xffffffffu, m2, o);
        }
        if (lane == 0) {
            wred[3 * wid] = m0;
            wred[3 * wid + 1] = m1;
            wred[3 * wid + 2] = m2;
        }
        __syncthreads();
        if (tid == 0) {
            double u0 = 0.0, u1 = 0.0, u2 = 0.0;
            for (int w = 0; w < (nt + 31) / 32; ++w) {
                u0 += wred[3 * w];
                u1 += wred[3 * w + 1];
                u2 += wred[3 * w + 2];
            }
            part[0] = u0;
            part[1] = u1;
            part[2] = u2;
            part[3] = 0.0;
            if (r == 0) {                 // rank 0 decides the wall-clock limit for the cluster
                if (*(volatile int *)a.abort_flag) part[3] = 1.0;
                else if (globaltimer3() - t0 > a.time_limit_ns) {
                    part[3] = 1.0;
                    atomicExch(a.abort_flag, 1);
                }
            }
        }
        cluster_sync_all();
        double m[3] = {0.0, 0.0, 0.0};
        for (int q = 0; q < C; ++q) {
            const uint32_t pq = cluster_addr(part, q);
            m[0] += ld_cluster<double>(pq);
            m[1] += ld_cluster<double>(pq + 8);
            m[2] += ld_cluster<double>(pq + 16);
        }
        const bool abort_now = ld_cluster<double>(cluster_addr(part, 0) + 24) != 0.0;
        const double sl = s - 2 * a.m, inv = 1.0 / (sl * sl * sl);
        for (int q = 0; q < 3; ++q) m[q] *= inv;
        const double cur = m[d];
        int st = -1;
        if (t % a.k == 0) {
            if (a.tol > 0.0 && t > a.k && fabs(cur - prev_u) <= a.tol * a.k * fabs(cur)) st = LBM_OK;
            prev_u = cur;
        }
        if (st < 0 && t >= a.max_steps) st = a.tol > 0.0 ? LBM_ENOTCONV : LBM_OK;
        if (st < 0 && abort_now) st = LBM_ETIMEOUT;
        if (st >= 0) {
            if (r == 0 && tid == 0) {
                for (int i = 0; i < 3; ++i) a.keff[9 * (int64_t)leaf + 3 * i + d] = a.nu_over_g * m[i];   // Eq. 17
                if (a.steps) a.steps[3 * (int64_t)leaf + d] = (int)t;
                if (st != LBM_OK) atomicMax(&a.status[leaf], st);
            }
            break;
        }
    }
    cluster_sync_all();     // no CTA leaves while a peer may still read its shared memory
}

// The compiled slot strides: FP32 up to 2048 cells per slab, FP64 up to 1024
template <typename T>
const void *clu3_kernel(int ps)
{
    switch (ps) {
    case 256: return reinterpret_cast<const void *>(&local3d_cluster_kernel<T, 256>);
    case 512: return reinterpret_cast<const void *>(&local3d_cluster_kernel<T, 512>);
    case 1024: return reinterpret_cast<const void *>(&local3d_cluster_kernel<T, 1024>);
    case 2048:
        if constexpr (sizeof(T) == 4) return reinterpret_cast<const void *>(&local3d_cluster_kernel<T, 2048>);
        return nullptr;
    default: return nullptr;
    }
}

// Shared memory of local3d_cluster_kernel at slot stride PS
inline size_t clu3_smem_bytes(int64_t PS, size_t esz)
{
    return sizeof(double) * (4 + 96 + 16) + (size_t)PS * Q19 * esz;
}

// e per cell of every job of a chunk: job j copies its leaf's cube of the field
__global__ void __launch_bounds__(256) local3d_coef_kernel(const float *kappa, int nx, int ny, int nz,
                                                           const int4 *leaves, const int *job_leaf, int s, int m,
                                                           int64_t s3, int njobs, double eps_nu, float *coef_f,
                                                           double *coef_d)
{
    const int64_t total = (int64_t)njobs * s3;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int job = (int)(i / s3);
        const int64_t c = i - (int64_t)job * s3;
        const int x = (int)(c % s), yz = (int)(c / s), y = yz % s, z = yz / s;
        const int4 L = leaves[job_leaf[job]];
        int gx = L.x - m + x, gy = L.y - m + y, gz = L.z - m + z;      // grown cube, periodic field
        gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
        gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
        gz = gz < 0 ? gz + nz : (gz >= nz ? gz - nz : gz);
        const float k = kappa[((int64_t)gz * ny + gy) * nx + gx];
        double e;
        if (!(k >= 0.0f)) e = 1.0;
        else if (eps_nu == 0.0 || isinf(k)) e = 0.0;
        else if (k == 0.0f) e = 1.0;
        else e = eps_nu / (2.0 * (double)k + eps_nu);
        if (coef_f) coef_f[i] = (float)e;
        else coef_d[i] = e;
    }
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
    int tensor = 0;         // coefficients are the 9 planes of E (coarse run with tensor K*)
    double S = 1.0;         // FP16 storage: populations are stored as S g
    int64_t n = 0, plane = 0, nblocks = 0;
    size_t esz = 4;
};

using namespace lbm;

namespace {

template <typename T>
Step3Args<T> args3(const lbm3d_grid *g, int src)
{
    using C = typename Comp3<T>::type;
    Step3Args<T> a;
    a.src = static_cast<const T *>(g->buf[src]);
    a.dst = static_cast<T *>(g->buf[1 - src]);
    a.coef = static_cast<const C *>(g->coef);
    a.nx = g->p.nx;
    a.ny = g->p.ny;
    a.nz = g->p.nz;
    a.plane = g->plane;
    a.omega = (C)(1.0 / g->p.tau);
    a.k_ru = (C)(6.0 * g->p.tau);
    a.k_j = (C)(3.0 * (1.0 - 2.0 * g->p.tau));
    a.hgx = (C)(0.5 * g->p.eps * g->p.gx);
    a.hgy = (C)(0.5 * g->p.eps * g->p.gy);
    a.hgz = (C)(0.5 * g->p.eps * g->p.gz);
    a.rho0 = (C)g->S;
    a.inv_scale = (C)(1.0 / g->S);
    return a;
}

dim3 grid3(const lbm3d_grid *g, int threads) { return dim3((g->p.nx + threads - 1) / threads, g->p.ny, g->p.nz); }

void launch_fields3(const lbm3d_grid *g, float *rho, float *u, float *v, float *w, double *partials)
{
    const dim3 gr = grid3(g, 128);
    if (g->esz == 2) {
        fields3d_kernel<__half, false><<<gr, 128, 0, g->st>>>(args3<__half>(g, g->cur), rho, u, v, w, partials);
    } else if (g->esz == 8) {
        if (g->tensor) fields3d_kernel<double, true><<<gr, 128, 0, g->st>>>(args3<double>(g, g->cur), rho, u, v, w, partials);
        else fields3d_kernel<double, false><<<gr, 128, 0, g->st>>>(args3<double>(g, g->cur), rho, u, v, w, partials);
    } else {
        if (g->tensor) fields3d_kernel<float, true><<<gr, 128, 0, g->st>>>(args3<float>(g, g->cur), rho, u, v, w, partials);
        else fields3d_kernel<float, false><<<gr, 128, 0, g->st>>>(args3<float>(g, g->cur), rho, u, v, w, partials);
    }
}

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

namespace {

// Runs every job of one leaf size on the cluster path. Returns LBM_EINVAL (nothing
// launched) when the cube does not fit the shared memory of a cluster of at most 16
// CTAs or the device cannot schedule such a cluster.
lbm_status run_cluster_size(const lbm3d_params *p, const float *kappa_dev, const int4 *d_l4,
                            const std::vector<int> &ids, int *d_ids, int sz, int m, double nu, double g_const,
                            double tol_rel, int64_t max_steps, int32_t check_every, int optin,
                            unsigned long long *d_clock, double *keff_dev, int32_t *status_dev, int32_t *steps_dev,
                            cudaStream_t st)
{
    const bool f64 = p->storage == LBM_F64;
    const size_t esz = f64 ? 8 : 4;
    const int NT = f64 ? clu3_threads<double>() : clu3_threads<float>();
    const int CPT = f64 ? clu3_cpt<double>() : clu3_cpt<float>();
    if (sz > 32) return LBM_EINVAL;
    // the fewest CTAs whose slab of L s^2 cells fits a compiled slot stride PS
    int C = 0, L = 0, PS = 0;
    for (int c = 1; c <= 16 && c <= sz && C == 0; c *= 2) {
        const int l = (sz + c - 1) / c;
        const int64_t P = (int64_t)l * sz * sz;
        for (int ps : {256, 512, 1024, 2048}) {
            if (P <= ps && P <= (int64_t)CPT * NT && clu3_smem_bytes(ps, esz) <= (size_t)optin &&
                (!f64 || ps <= 1024)) {
                C = c;
                L = l;
                PS = ps;
                break;
            }
        }
    }
    if (C == 0) return LBM_EINVAL;
    const int64_t P = (int64_t)L * sz * sz;
    const size_t smem = clu3_smem_bytes(PS, esz);
    // enough threads for CPT cells each, whole warps
    const int nt = (int)std::min<int64_t>(NT, ((P + CPT - 1) / CPT + 31) / 32 * 32);
    const void *fn = f64 ? clu3_kernel<double>(PS) : clu3_kernel<float>(PS);
    if (!fn) return LBM_EINVAL;
    // the opt-in maximum, not this launch's size: a concurrent call with a larger cube stays valid
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess ||
        (C > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
        cudaGetLastError();
        return LBM_EINVAL;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3((unsigned)nt);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3((unsigned)C);
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        return LBM_EINVAL;
    }
    const int n = (int)ids.size();
    if (cudaMemcpyAsync(d_ids, ids.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ECUDA, "copying the leaf list failed");
    }
    // launches of at most 2^31 - 1 CTAs, each a whole number of leaves
    const int64_t leaves_per = std::max<int64_t>(1, (((int64_t)1 << 31) - 1) / (3 * (int64_t)C));
    for (int64_t l0 = 0; l0 < n; l0 += leaves_per) {
        const int nl = (int)std::min<int64_t>(leaves_per, n - l0);
        cfg.gridDim = dim3((unsigned)(3 * (int64_t)nl * C));
        cudaError_t e;
        if (f64) {
            Clu3Args<double> a{kappa_dev, p->nx, p->ny, p->nz, d_l4, d_ids + l0, 3 * nl, sz, L, m, 1.0 / p->tau, 6.0 * p->tau,
                               3.0 * (1.0 - 2.0 * p->tau), 0.5 * p->eps * g_const, p->eps * nu, nu / g_const, tol_rel,
                               check_every, max_steps, keff_dev, status_dev, steps_dev, d_clock,
                               reinterpret_cast<int *>(d_clock + 1),
                               (unsigned long long)(local_time_limit() * 1e9)};
            void *args[] = {&a};
            e = cudaLaunchKernelExC(&cfg, fn, args);
        } else {
            Clu3Args<float> a{kappa_dev, p->nx, p->ny, p->nz, d_l4, d_ids + l0, 3 * nl, sz, L, m, (float)(1.0 / p->tau),
                              (float)(6.0 * p->tau), (float)(3.0 * (1.0 - 2.0 * p->tau)), (float)(0.5 * p->eps * g_const),
                              p->eps * nu, nu / g_const, tol_rel, check_every, max_steps, keff_dev, status_dev,
                              steps_dev, d_clock, reinterpret_cast<int *>(d_clock + 1),
                              (unsigned long long)(local_time_limit() * 1e9)};
            void *args[] = {&a};
            e = cudaLaunchKernelExC(&cfg, fn, args);
        }
        count_launches(1);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(LBM_ECUDA, "cluster launch failed: %s", cudaGetErrorString(e));
        }
    }
    unsigned long long clk[2] = {0, 0};
    if (cudaMemcpyAsync(clk, d_clock, sizeof(clk), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ECUDA, "local problems failed on the device");
    }
    if (reinterpret_cast<const int *>(&clk[1])[0])
        return fail(LBM_ETIMEOUT, "local problems exceeded the time limit; unfinished leaves carry LBM_ETIMEOUT");
    return LBM_OK;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

// A 3-D grid with per-cell scalar kappa (kappa_dev) or, for a coarse run, per-cell
// tensor K* = kscale keff (keff_dev [n][9], row-major).
lbm_status grid3_create_impl(const lbm3d_params *p, const float *kappa_dev, const double *keff_dev, double kscale,
                             void *cuda_stream, lbm3d_grid **out)
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
    if (p->storage != LBM_F32 && p->storage != LBM_F64 && !(p->storage == LBM_F16 && !keff_dev))
        return fail(LBM_EINVAL, "storage must be LBM_F32, LBM_F16 (scalar kappa only) or LBM_F64");
    if (keff_dev ? !is_device_ptr(keff_dev) : !is_device_ptr(kappa_dev))
        return fail(LBM_EINVAL, keff_dev ? "keff_dev must be a device pointer" : "kappa_dev must be a device pointer");
    lbm3d_grid *g = new lbm3d_grid;
    g->p = *p;
    g->tensor = keff_dev ? 1 : 0;
    cudaGetDevice(&g->dev);
    g->st = static_cast<cudaStream_t>(cuda_stream);
    g->n = (int64_t)p->nx * p->ny * p->nz;
    g->plane = (g->n + 63) / 64 * 64;
    g->esz = p->storage == LBM_F64 ? 8 : (p->storage == LBM_F16 ? 2 : 4);
    const size_t csz = g->esz == 8 ? 8 : 4;        // coefficients in the compute type
    const dim3 gr = grid3(g, 128);
    g->nblocks = (int64_t)gr.x * gr.y * gr.z;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaMalloc(&g->buf[k], Q19 * g->plane * g->esz);
    if (e == cudaSuccess) e = cudaMalloc(&g->coef, (g->tensor ? 9 * g->plane : g->n) * csz);
    if (e == cudaSuccess) e = cudaMalloc(&g->partials, sizeof(double) * 3 * g->nblocks);
    if (e == cudaSuccess) e = cudaMalloc(&g->mean, sizeof(double) * 3);
    if (e == cudaSuccess) e = cudaMalloc(&g->flags, 2 * sizeof(unsigned));
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaMemsetAsync(g->buf[k], 0, Q19 * g->plane * g->esz, g->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->flags, 0, 2 * sizeof(unsigned), g->st);
    if (e != cudaSuccess) {
        free3(g);
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "3-D grid allocation: %s",
                    cudaGetErrorString(e));
    }
    const double nu = p->nu < 0.0 ? (p->tau - 0.5) / 3.0 : p->nu;
    const int nb = (int)std::min<int64_t>((g->n + 255) / 256, 8192);
    if (g->tensor) {
        if (g->esz == 8)
            coef3d_tensor_kernel<double><<<nb, 256, 0, g->st>>>(keff_dev, kscale, static_cast<double *>(g->coef), g->n,
                                                                g->plane, 0.5 * p->eps * nu, g->flags);
        else
            coef3d_tensor_kernel<float><<<nb, 256, 0, g->st>>>(keff_dev, kscale, static_cast<float *>(g->coef), g->n,
                                                               g->plane, 0.5 * p->eps * nu, g->flags);
    } else {
        if (g->esz == 8)
            coef3d_kernel<double><<<nb, 256, 0, g->st>>>(kappa_dev, static_cast<double *>(g->coef), g->n, p->eps * nu,
                                                         g->flags);
        else
            coef3d_kernel<float><<<nb, 256, 0, g->st>>>(kappa_dev, static_cast<float *>(g->coef), g->n, p->eps * nu,
                                                        g->flags);
    }
    count_launches(1);
    unsigned hflags[2] = {0u, 0u};
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hflags, g->flags, sizeof hflags, cudaMemcpyDeviceToHost, g->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
    if (e != cudaSuccess) {
        free3(g);
        return fail(LBM_ECUDA, "3-D coefficient pass: %s", cudaGetErrorString(e));
    }
    const unsigned flags = hflags[0];
    if (flags) {
        free3(g);
        if (!keff_dev) return fail(LBM_EINVAL, "kappa holds NaN or negative values");
        return fail(LBM_EINVAL, (flags & 1u) ? "keff holds non-finite values" : "K* + (eps nu / 2) I is singular");
    }
    if (g->esz == 2) {
        // FP16 keeps 11 bits: store S g with S = 2^k placing the largest expected deviation,
        // ~ 3 w u_max with u_max ~ kappa_max |G| / nu, near 2^12 (headroom below the FP16 maximum)
        float kmax;
        std::memcpy(&kmax, &hflags[1], sizeof kmax);
        const double gmag = std::fabs(p->gx) + std::fabs(p->gy) + std::fabs(p->gz);
        double umax = (nu > 0.0 && kmax > 0.0f) ? (double)kmax * gmag / nu : gmag * 1e3;
        if (!(umax > 0.0)) umax = 1e-3;
        if (umax > 0.1) umax = 0.1;
        const int e2 = std::max(0, std::min(60, (int)std::floor(std::log2(4096.0 / umax))));
        g->S = std::ldexp(1.0, e2);
    }
    *out = g;
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm3d_grid_create(const lbm3d_params *p, const float *kappa_dev, void *cuda_stream, lbm3d_grid **out)
{
    return grid3_create_impl(p, kappa_dev, nullptr, 1.0, cuda_stream, out);
}

int64_t lbm3d_grid_state_bytes(const lbm3d_grid *g)
{
    return g ? CKPT_HEADER_BYTES + (int64_t)Q19 * g->plane * (int64_t)g->esz : -1;
}

}  // extern "C"

namespace {

// The header a checkpoint of 3-D grid g carries (and a loaded one must match).
CkptHeader grid3_header(const lbm3d_grid *g)
{
    CkptHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, "LBM3CKPT", 8);
    h.version = 1;
    h.storage = g->p.storage;
    h.nx = g->p.nx;
    h.ny = g->p.ny;
    h.nz = g->p.nz;
    h.scale = g->S;
    const double d[6] = {g->p.tau, g->p.nu, g->p.eps, g->p.gx, g->p.gy, g->p.gz};
    const int32_t t = g->tensor;
    h.params_hash = fnv1a(&t, sizeof t, fnv1a(d, sizeof d));
    h.steps = 0;
    return h;
}

}  // namespace

extern "C" {

lbm_status lbm3d_grid_save_state(lbm3d_grid *g, void *state_dev, int64_t nbytes)
{
    if (!g) return fail(LBM_EINVAL, "grid is NULL");
    if (nbytes != lbm3d_grid_state_bytes(g))
        return fail(LBM_EINVAL, "state buffer holds %lld bytes, the grid's state is %lld", (long long)nbytes,
                    (long long)lbm3d_grid_state_bytes(g));
    if (!is_device_ptr(state_dev)) return fail(LBM_EINVAL, "state_dev must be a device pointer");
    const CkptHeader h = grid3_header(g);
    char *dst = static_cast<char *>(state_dev);
    L3_CUDA(cudaMemcpyAsync(dst, &h, sizeof h, cudaMemcpyHostToDevice, g->st));
    L3_CUDA(cudaMemcpyAsync(dst + CKPT_HEADER_BYTES, g->buf[g->cur], (size_t)(nbytes - CKPT_HEADER_BYTES),
                            cudaMemcpyDeviceToDevice, g->st));
    L3_CUDA(cudaStreamSynchronize(g->st));
    return LBM_OK;
}

lbm_status lbm3d_grid_load_state(lbm3d_grid *g, const void *state_dev, int64_t nbytes)
{
    if (!g) return fail(LBM_EINVAL, "grid is NULL");
    if (nbytes != lbm3d_grid_state_bytes(g))
        return fail(LBM_EINVAL, "state buffer holds %lld bytes, the grid's state is %lld", (long long)nbytes,
                    (long long)lbm3d_grid_state_bytes(g));
    if (!is_device_ptr(state_dev)) return fail(LBM_EINVAL, "state_dev must be a device pointer");
    CkptHeader saved;
    L3_CUDA(cudaMemcpyAsync(&saved, state_dev, sizeof saved, cudaMemcpyDeviceToHost, g->st));
    L3_CUDA(cudaStreamSynchronize(g->st));
    const CkptHeader mine = grid3_header(g);
    if (std::memcmp(saved.magic, mine.magic, 8) || saved.version != mine.version || saved.storage != mine.storage ||
        saved.nx != mine.nx || saved.ny != mine.ny || saved.nz != mine.nz || saved.scale != mine.scale ||
        saved.params_hash != mine.params_hash)
        return fail(LBM_EINVAL, "the state was saved by a grid of another size, storage, scale or parameter set");
    const char *src = static_cast<const char *>(state_dev);
    L3_CUDA(cudaMemcpyAsync(g->buf[g->cur], src + CKPT_HEADER_BYTES, (size_t)(nbytes - CKPT_HEADER_BYTES),
                            cudaMemcpyDeviceToDevice, g->st));
    L3_CUDA(cudaStreamSynchronize(g->st));
    return LBM_OK;
}

lbm_status lbm3d_coarse_params(const lbm3d_params *fine_p, int32_t block, lbm3d_params *coarse_out)
{
    if (!fine_p || !coarse_out) return fail(LBM_EINVAL, "params and out must not be NULL");
    if (block < 1 || fine_p->nx % block || fine_p->ny % block || fine_p->nz % block)
        return fail(LBM_EINVAL, "nx, ny, nz must be multiples of block %d", block);
    if (!std::isfinite(fine_p->tau) || fine_p->tau < 0.5) return fail(LBM_EINVAL, "tau must be finite and >= 0.5");
    const double r = block;
    lbm3d_params c = *fine_p;
    c.nx = fine_p->nx / block;
    c.ny = fine_p->ny / block;
    c.nz = fine_p->nz / block;
    c.tau = 0.5 + (fine_p->tau - 0.5) / r;
    c.nu = (fine_p->nu < 0.0 ? (fine_p->tau - 0.5) / 3.0 : fine_p->nu) / r;
    c.gx = fine_p->gx * r;
    c.gy = fine_p->gy * r;
    c.gz = fine_p->gz * r;
    *coarse_out = c;
    return LBM_OK;
}

lbm_status lbm3d_coarse_grid_create(const lbm3d_params *fine_p, int32_t block, const double *keff_coarse_dev,
                                    void *cuda_stream, lbm3d_grid **out)
{
    if (out) *out = nullptr;
    lbm3d_params c;
    lbm_status s = lbm3d_coarse_params(fine_p, block, &c);
    if (s != LBM_OK) return s;
    if (!keff_coarse_dev) return fail(LBM_EINVAL, "keff_coarse_dev is NULL");
    return grid3_create_impl(&c, nullptr, keff_coarse_dev, 1.0 / ((double)block * block), cuda_stream, out);
}

lbm_status lbm3d_block_average(const float *in_dev, int32_t nx, int32_t ny, int32_t nz, int32_t block,
                               float *out_dev, void *cuda_stream)
{
    if (nx < 1 || ny < 1 || nz < 1 || block < 1 || nx % block || ny % block || nz % block)
        return fail(LBM_EINVAL, "nx, ny, nz must be positive multiples of block");
    if (!is_device_ptr(in_dev) || !is_device_ptr(out_dev)) return fail(LBM_EINVAL, "in/out must be device pointers");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int64_t nb = (int64_t)(nx / block) * (ny / block) * (nz / block);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((nb + 255) / 256, 4096));
    block_average3_kernel<<<blocks, 256, 0, st>>>(in_dev, nx, ny, nz, block, out_dev);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(LBM_ECUDA, "3-D block average: %s", cudaGetErrorString(e));
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
        if (g->esz == 2) {
            step3d_kernel<__half, false><<<gr, 256, 0, g->st>>>(args3<__half>(g, g->cur));
        } else if (g->esz == 8) {
            if (g->tensor) step3d_kernel<double, true><<<gr, 256, 0, g->st>>>(args3<double>(g, g->cur));
            else step3d_kernel<double, false><<<gr, 256, 0, g->st>>>(args3<double>(g, g->cur));
        } else {
            if (g->tensor) step3d_kernel<float, true><<<gr, 256, 0, g->st>>>(args3<float>(g, g->cur));
            else step3d_kernel<float, false><<<gr, 256, 0, g->st>>>(args3<float>(g, g->cur));
        }
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
    launch_fields3(g, rho_dev, u_dev, v_dev, w_dev, nullptr);
    count_launches(1);
    L3_CUDA(cudaGetLastError());
    L3_CUDA(cudaStreamSynchronize(g->st));
    return LBM_OK;
}

lbm_status lbm3d_mean_velocity(lbm3d_grid *g, double out_mean_uvw[3])
{
    if (!g || !out_mean_uvw) return fail(LBM_EINVAL, "grid and out must not be NULL");
    launch_fields3(g, nullptr, nullptr, nullptr, nullptr, g->partials);
    reduce3_kernel<<<1, 1024, 0, g->st>>>(g->partials, g->nblocks, 1.0 / (double)g->n, g->mean);
    count_launches(2);
    L3_CUDA(cudaGetLastError());
    L3_CUDA(cudaMemcpyAsync(out_mean_uvw, g->mean, sizeof(double) * 3, cudaMemcpyDeviceToHost, g->st));
    L3_CUDA(cudaStreamSynchronize(g->st));
    return LBM_OK;
}

lbm_status lbm3d_local_keff_batch(const lbm3d_params *p, const float *kappa_dev, const lbm3d_leaf *leaves_dev,
                                  int32_t n_leaves, double g_const, double tol_rel, int64_t max_steps,
                                  int32_t check_every, double *keff_dev, int32_t *status_dev, int32_t *steps_dev,
                                  void *cuda_stream)
{
    if (!p) return fail(LBM_EINVAL, "params is NULL");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return fail(LBM_EINVAL, "nx, ny, nz must be >= 1");
    if (!std::isfinite(p->tau) || p->tau < 0.5) return fail(LBM_EINVAL, "tau must be finite and >= 0.5");
    if (!std::isfinite(p->nu) || !std::isfinite(p->eps) || p->eps < 0.0)
        return fail(LBM_EINVAL, "nu must be finite and eps finite and >= 0");
    if (p->storage != LBM_F32 && p->storage != LBM_F64) return fail(LBM_EINVAL, "storage must be LBM_F32 or LBM_F64");
    if (n_leaves < 0) return fail(LBM_EINVAL, "n_leaves must be >= 0");
    if (!std::isfinite(g_const) || g_const == 0.0) return fail(LBM_EINVAL, "g_const must be finite and non-zero");
    if (!std::isfinite(tol_rel) || tol_rel < 0.0) return fail(LBM_EINVAL, "tol_rel must be finite and >= 0");
    if (max_steps < 1 || max_steps >= ((int64_t)1 << 31)) return fail(LBM_EINVAL, "max_steps must be in [1, 2^31 - 1]");
    if (check_every < 1) return fail(LBM_EINVAL, "check_every must be >= 1");
    if (n_leaves == 0) return LBM_OK;
    if (!is_device_ptr(kappa_dev) || !is_device_ptr(leaves_dev) || !is_device_ptr(keff_dev) ||
        !is_device_ptr(status_dev) || (steps_dev && !is_device_ptr(steps_dev)))
        return fail(LBM_EINVAL, "kappa, leaves, keff, status (and steps) must be device pointers");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    std::vector<lbm3d_leaf> lv(n_leaves);
    L3_CUDA(cudaMemcpyAsync(lv.data(), leaves_dev, sizeof(lbm3d_leaf) * n_leaves, cudaMemcpyDeviceToHost, st));
    L3_CUDA(cudaStreamSynchronize(st));
    const int m = p->margin;
    if (m < 0 || m > 32 || m > p->nx || m > p->ny || m > p->nz)
        return fail(LBM_EINVAL, "margin %d must be in [0, 32] and at most nx, ny, nz", m);
    std::map<int, std::vector<int>> by_size;       // by the side of the simulated cube, size + 2 margin
    for (int i = 0; i < n_leaves; ++i) {
        const lbm3d_leaf &L = lv[i];
        if (L.size < 1 || L.size > 256) return fail(LBM_EINVAL, "leaf %d: size %d outside [1, 256]", i, L.size);
        if (L.x0 < 0 || L.y0 < 0 || L.z0 < 0 || (int64_t)L.x0 + L.size > p->nx || (int64_t)L.y0 + L.size > p->ny ||
            (int64_t)L.z0 + L.size > p->nz)
            return fail(LBM_EINVAL, "leaf %d (%d, %d, %d, %d) lies outside the field", i, L.x0, L.y0, L.z0, L.size);
        if (L.size + 2 * m > 256) return fail(LBM_EINVAL, "leaf %d: size + 2 margin exceeds 256", i);
        by_size[L.size + 2 * m].push_back(i);
    }
    L3_CUDA(cudaMemsetAsync(status_dev, 0, sizeof(int32_t) * n_leaves, st));
    if (steps_dev) L3_CUDA(cudaMemsetAsync(steps_dev, 0, sizeof(int32_t) * 3 * n_leaves, st));
    const double nu = p->nu < 0.0 ? (p->tau - 0.5) / 3.0 : p->nu;
    const bool f64 = p->storage == LBM_F64;
    const size_t esz = f64 ? 8 : 4;
    std::vector<int4> l4(n_leaves);
    for (int i = 0; i < n_leaves; ++i) l4[i] = make_int4(lv[i].x0, lv[i].y0, lv[i].z0, lv[i].size);

    // device scratch, sized for the largest chunk and freed on every exit
    int4 *d_l4 = nullptr;
    void *buf[2] = {nullptr, nullptr};
    void *coef = nullptr;
    int *d_active = nullptr, *d_list = nullptr, *d_jl = nullptr, *d_nact = nullptr, *d_ids = nullptr;
    double *d_prev = nullptr;
    unsigned long long *d_clock = nullptr;    // [0] launch start (globaltimer), [1] abort flag
    auto release = [&]() {
        cudaFree(d_l4); cudaFree(buf[0]); cudaFree(buf[1]); cudaFree(coef);
        cudaFree(d_active); cudaFree(d_list); cudaFree(d_jl); cudaFree(d_nact); cudaFree(d_prev);
        cudaFree(d_ids); cudaFree(d_clock);
        cudaGetLastError();
    };
#define L3_CUDA2(call)                                                                           \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            cudaGetLastError();                                                                  \
            release();                                                                           \
            return fail(e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s failed: %s", \
                        #call, cudaGetErrorString(e_));                                          \
        }                                                                                        \
    } while (0)
    L3_CUDA2(cudaMalloc(&d_l4, sizeof(int4) * n_leaves));
    L3_CUDA2(cudaMemcpyAsync(d_l4, l4.data(), sizeof(int4) * n_leaves, cudaMemcpyHostToDevice, st));
    L3_CUDA2(cudaMalloc(&d_nact, sizeof(int)));
    L3_CUDA2(cudaMalloc(&d_ids, sizeof(int) * n_leaves));
    L3_CUDA2(cudaMalloc(&d_clock, 2 * sizeof(unsigned long long)));
    L3_CUDA2(cudaMemsetAsync(d_clock, 0, 2 * sizeof(unsigned long long), st));
    int dev = 0, optin = 0;
    L3_CUDA2(cudaGetDevice(&dev));
    L3_CUDA2(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const char *force_global = std::getenv("LBM_LOCAL3_GLOBAL");
    const bool cluster_ok = !(force_global && force_global[0] == '1');
    constexpr int64_t CELL_BUDGET = (int64_t)1 << 26;     // cells per chunk (10 GB of FP32 state)
    int64_t cap_cells = 0, cap_jobs = 0;
    for (const auto &kv : by_size) {
        const int sz = kv.first;
        const int64_t s3 = (int64_t)sz * sz * sz;
        if (cluster_ok) {
            const lbm_status cs = run_cluster_size(p, kappa_dev, d_l4, kv.second, d_ids, sz, m, nu, g_const, tol_rel,
                                                   max_steps, check_every, optin, d_clock, keff_dev, status_dev,
                                                   steps_dev, st);
            // LBM_ETIMEOUT is in the leaves' status already; LBM_EINVAL: the cube does not fit, take the global path
            if (cs == LBM_OK || cs == LBM_ETIMEOUT) continue;
            if (cs != LBM_EINVAL) {
                release();
                return cs;
            }
        }
        // jobs per chunk: a multiple of 3, so that a job's drive axis is its chunk index modulo 3
        const int64_t per = std::max<int64_t>(3, std::min<int64_t>(65535, CELL_BUDGET / s3) / 3 * 3);
        const std::vector<int> &ids = kv.second;
        const int64_t njobs_all = 3 * (int64_t)ids.size();
        for (int64_t j0 = 0; j0 < njobs_all; j0 += per) {
            const int njobs = (int)std::min<int64_t>(per, njobs_all - j0);
            const int64_t cells = (int64_t)njobs * s3, plane = (cells + 63) / 64 * 64;
            if (plane > cap_cells || njobs > cap_jobs) {   // grow the scratch
                cudaFree(buf[0]); cudaFree(buf[1]); cudaFree(coef); cudaFree(d_active); cudaFree(d_list);
                cudaFree(d_jl); cudaFree(d_prev);
                buf[0] = buf[1] = coef = nullptr;
                d_active = d_list = d_jl = nullptr;
                d_prev = nullptr;
                cap_cells = std::max(cap_cells, plane);
                cap_jobs = std::max<int64_t>(cap_jobs, njobs);
                L3_CUDA2(cudaMalloc(&buf[0], Q19 * cap_cells * esz));
                L3_CUDA2(cudaMalloc(&buf[1], Q19 * cap_cells * esz));
                L3_CUDA2(cudaMalloc(&coef, cap_cells * esz));
                L3_CUDA2(cudaMalloc(&d_active, sizeof(int) * cap_jobs));
                L3_CUDA2(cudaMalloc(&d_list, sizeof(int) * cap_jobs));
                L3_CUDA2(cudaMalloc(&d_jl, sizeof(int) * cap_jobs));
                L3_CUDA2(cudaMalloc(&d_prev, sizeof(double) * cap_jobs));
            }
            std::vector<int> jl(njobs), act(njobs, 1), list(njobs);
            for (int j = 0; j < njobs; ++j) {
                jl[j] = ids[(size_t)((j0 + j) / 3)];
                list[j] = j;
            }
            L3_CUDA2(cudaMemcpyAsync(d_list, list.data(), sizeof(int) * njobs, cudaMemcpyHostToDevice, st));
            L3_CUDA2(cudaMemcpyAsync(d_jl, jl.data(), sizeof(int) * njobs, cudaMemcpyHostToDevice, st));
            L3_CUDA2(cudaMemcpyAsync(d_active, act.data(), sizeof(int) * njobs, cudaMemcpyHostToDevice, st));
            L3_CUDA2(cudaMemsetAsync(d_prev, 0, sizeof(double) * njobs, st));
            L3_CUDA2(cudaMemsetAsync(buf[0], 0, Q19 * plane * esz, st));
            L3_CUDA2(cudaMemsetAsync(buf[1], 0, Q19 * plane * esz, st));
            int nact = njobs;
            L3_CUDA2(cudaMemcpyAsync(d_nact, &nact, sizeof(int), cudaMemcpyHostToDevice, st));
            const int nb = (int)std::min<int64_t>((cells + 255) / 256, 8192);
            local3d_coef_kernel<<<nb, 256, 0, st>>>(kappa_dev, p->nx, p->ny, p->nz, d_l4, d_jl, sz, m, s3, njobs, p->eps * nu,
                                                    f64 ? nullptr : static_cast<float *>(coef),
                                                    f64 ? static_cast<double *>(coef) : nullptr);
            count_launches(1);
            int cur = 0, nlist = njobs;    // blocks go to the nlist jobs of d_list only
            int64_t t = 0;
            while (t < max_steps && nact > 0) {
                const int64_t nstep = std::min<int64_t>(check_every, max_steps - t);
                const dim3 sgrid((unsigned)((s3 + 255) / 256), (unsigned)nlist);
                for (int64_t i = 0; i < nstep; ++i) {
                    if (f64) {
                        Local3Args<double> a{static_cast<const double *>(buf[cur]), static_cast<double *>(buf[1 - cur]),
                                             static_cast<const double *>(coef), d_list, sz, m, s3, plane,
                                             1.0 / p->tau, 6.0 * p->tau, 3.0 * (1.0 - 2.0 * p->tau), 0.5 * p->eps * g_const};
                        local3d_step_kernel<double><<<sgrid, 256, 0, st>>>(a);
                    } else {
                        Local3Args<float> a{static_cast<const float *>(buf[cur]), static_cast<float *>(buf[1 - cur]),
                                            static_cast<const float *>(coef), d_list, sz, m, s3, plane,
                                            (float)(1.0 / p->tau), (float)(6.0 * p->tau), (float)(3.0 * (1.0 - 2.0 * p->tau)),
                                            (float)(0.5 * p->eps * g_const)};
                        local3d_step_kernel<float><<<sgrid, 256, 0, st>>>(a);
                    }
                    cur = 1 - cur;
                }
                t += nstep;
                Check3 ck{(int)t, check_every, t % check_every == 0 ? 1 : 0, max_steps, tol_rel, nu / g_const,
                          d_active, d_prev, d_jl, keff_dev, status_dev, steps_dev, d_nact};
                if (f64) {
                    Local3Args<double> a{static_cast<const double *>(buf[cur]), nullptr, static_cast<const double *>(coef),
                                         d_list, sz, m, s3, plane, 1.0 / p->tau, 6.0 * p->tau, 3.0 * (1.0 - 2.0 * p->tau),
                                         0.5 * p->eps * g_const};
                    local3d_check_kernel<double><<<nlist, 256, 0, st>>>(a, ck);
                } else {
                    Local3Args<float> a{static_cast<const float *>(buf[cur]), nullptr, static_cast<const float *>(coef),
                                        d_list, sz, m, s3, plane, (float)(1.0 / p->tau), (float)(6.0 * p->tau),
                                        (float)(3.0 * (1.0 - 2.0 * p->tau)), (float)(0.5 * p->eps * g_const)};
                    local3d_check_kernel<float><<<nlist, 256, 0, st>>>(a, ck);
                }
                count_launches(nstep + 1);
                L3_CUDA2(cudaGetLastError());
                L3_CUDA2(cudaMemcpyAsync(&nact, d_nact, sizeof(int), cudaMemcpyDeviceToHost, st));
                L3_CUDA2(cudaStreamSynchronize(st));
                if (nact > 0 && nact < nlist) {    // drop the finished jobs from the launch grid
                    local3d_compact_kernel<<<1, 1024, 0, st>>>(d_active, njobs, d_list);
                    count_launches(1);
                    L3_CUDA2(cudaGetLastError());
                    nlist = nact;
                }
            }
        }
    }
    std::vector<int32_t> stat(n_leaves);
    L3_CUDA2(cudaMemcpyAsync(stat.data(), status_dev, sizeof(int32_t) * n_leaves, cudaMemcpyDeviceToHost, st));
    L3_CUDA2(cudaStreamSynchronize(st));
    release();
    int worst = LBM_OK;
    for (int v : stat) worst = std::max(worst, v);
    return (lbm_status)worst;
}

lbm_status lbm3d_upscale(const lbm3d_params *p, const float *kappa_dev, int32_t block, double g_const,
                         double tol_rel, int64_t max_steps, double *keff_coarse_dev, int32_t *n_notconv,
                         void *cuda_stream)
{
    if (n_notconv) *n_notconv = 0;
    if (!p) return fail(LBM_EINVAL, "params is NULL");
    if (block < 1 || p->nx < 1 || p->ny < 1 || p->nz < 1 || p->nx % block || p->ny % block || p->nz % block)
        return fail(LBM_EINVAL, "nx, ny, nz must be positive multiples of block %d", block);
    if (block > 256) return fail(LBM_EINVAL, "block must be at most 256");
    if (!keff_coarse_dev || !is_device_ptr(keff_coarse_dev)) return fail(LBM_EINVAL, "keff_coarse_dev must be a device pointer");
    const int bx = p->nx / block, by = p->ny / block, bz = p->nz / block;
    const int64_t n = (int64_t)bx * by * bz;
    if (n > INT32_MAX) return fail(LBM_EINVAL, "too many blocks");
    // one cubic leaf per coarse cell, in the coarse grid's [z][y][x] order, so keff lands in place
    std::vector<lbm3d_leaf> lv((size_t)n);
    for (int z = 0, i = 0; z < bz; ++z)
        for (int y = 0; y < by; ++y)
            for (int x = 0; x < bx; ++x, ++i) lv[i] = lbm3d_leaf{x * block, y * block, z * block, block};
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    lbm3d_leaf *d_leaves = nullptr;
    int32_t *d_status = nullptr;
    cudaError_t e = cudaMalloc(&d_leaves, sizeof(lbm3d_leaf) * n);
    if (e == cudaSuccess) e = cudaMalloc(&d_status, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_leaves, lv.data(), sizeof(lbm3d_leaf) * n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_leaves);
        cudaFree(d_status);
        return fail(e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "3-D upscale set-up: %s",
                    cudaGetErrorString(e));
    }
    lbm_status s = lbm3d_local_keff_batch(p, kappa_dev, d_leaves, (int32_t)n, g_const, tol_rel, max_steps, 64,
                                          keff_coarse_dev, d_status, nullptr, cuda_stream);
    if (n_notconv && (s == LBM_OK || s == LBM_ENOTCONV || s == LBM_ETIMEOUT)) {
        std::vector<int32_t> stat((size_t)n);
        if (cudaMemcpyAsync(stat.data(), d_status, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
            cudaStreamSynchronize(st) == cudaSuccess) {
            for (int32_t v : stat) *n_notconv += v != LBM_OK;
        } else {
            cudaGetLastError();
        }
    }
    cudaFree(d_leaves);
    cudaFree(d_status);
    return s;
}

}  // extern "C"
