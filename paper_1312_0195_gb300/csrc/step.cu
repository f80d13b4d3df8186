// step.cu -- fused pull-stream + collide of the simplified Shan-Chen LBM
// (Section 2.2: Eqs. 2, 6, 13, 15, 16), the moment/residual pass, and the
// per-cell coefficient set-up.
//
// Storage. Distributions live as deviations g_a = f_a - w_a rho0 in nine SoA
// planes [9][plane], x fastest. Every quantity of the step is linear in f (the
// force enters as rho G and rho is a sum of f), so in deviation form
//   drho = sum_a g_a,  j = sum_a e_a g_a,  rho = rho0 + drho
//   rho u    = (1 - e) r,  r = j + eps rho G / 2       (Eq. 6 times rho)
//   rho u_eq = 2 tau (rho u) + (1 - 2 tau) j            (Eq. 16 times rho)
//   g_eq     = w (drho + 3 e . rho u_eq)                (Eq. 2 minus w rho0)
//   g*       = g + (g_eq - g) / tau                     (Eq. 13)
// with the drag fraction e = 1 - 1/(1 + eps nu / (2 kappa)) precomputed per cell. No division by
// rho happens inside the step. Scaling every g by S (FP16 storage) is exact if
// rho0 is replaced by S in the force term, which is what `rho0` carries.
//
// Pull scheme: the buffer holds the post-collision state of step n-1; step n
// reads g*_a(x - e_a) (that is streaming, Eq. 13 left-hand side), collides and
// writes g*_a(x) to the other buffer. Each thread owns VEC consecutive cells of
// one row and moves them with 128-bit loads and stores; the one-cell shift of
// populations with e_x = +-1 is taken from the neighbouring lane with a warp
// shuffle, and only lanes at a row edge (or warp edge) load that cell directly.
// Rows (e_y = +-1) are whole-row offsets, so every load stays aligned.
#include "lbm_internal.h"

#include <math.h>

namespace lbm {
namespace {

template <typename T> struct Comp { using type = float; };
template <> struct Comp<double> { using type = double; };

__device__ __forceinline__ float to_c(float v) { return v; }
__device__ __forceinline__ float to_c(__half v) { return __half2float(v); }
__device__ __forceinline__ double to_c(double v) { return v; }
template <typename T> __device__ __forceinline__ T from_c(float v);
template <> __device__ __forceinline__ float from_c<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_c<__half>(float v) { return __float2half_rn(v); }
template <typename T> __device__ __forceinline__ T from_c(double v);
template <> __device__ __forceinline__ double from_c<double>(double v) { return v; }

template <typename T, int VEC>
struct alignas(sizeof(T) * VEC) Pack { T v[VEC]; };

template <typename C> __device__ __forceinline__ C wgt(int a)
{
    return a == 0 ? C(4.0 / 9.0) : (a <= 4 ? C(1.0 / 9.0) : C(1.0 / 36.0));
}

template <typename T>
__device__ __forceinline__ T shfl_up1(T v) { return __shfl_up_sync(0xffffffffu, v, 1); }
template <typename T>
__device__ __forceinline__ T shfl_down1(T v) { return __shfl_down_sync(0xffffffffu, v, 1); }
template <>
__device__ __forceinline__ __half shfl_up1<__half>(__half v)
{
    return __ushort_as_half((unsigned short)__shfl_up_sync(0xffffffffu, (unsigned)__half_as_ushort(v), 1));
}
template <>
__device__ __forceinline__ __half shfl_down1<__half>(__half v)
{
    return __ushort_as_half((unsigned short)__shfl_down_sync(0xffffffffu, (unsigned)__half_as_ushort(v), 1));
}

// Loads VEC consecutive coefficient values starting at index i (i multiple of VEC).
template <typename CT, int VEC>
__device__ __forceinline__ void load_vec(const CT *p, int64_t i, CT out[VEC])
{
    if constexpr (VEC * sizeof(CT) >= 16) {
        constexpr int PER = 16 / sizeof(CT);
#pragma unroll
        for (int k = 0; k < VEC / PER; ++k) {
            Pack<CT, PER> pk = *reinterpret_cast<const Pack<CT, PER> *>(p + i + k * PER);
#pragma unroll
            for (int m = 0; m < PER; ++m) out[k * PER + m] = pk.v[m];
        }
    } else {
        Pack<CT, VEC> pk = *reinterpret_cast<const Pack<CT, VEC> *>(p + i);
#pragma unroll
        for (int m = 0; m < VEC; ++m) out[m] = pk.v[m];
    }
}

// The collision of one cell given its streamed deviations gq[9] (in place).
// Guo scheme (guo != 0): u_eq = u and g* += w_a 3 (1 - 1/(2 tau)) e_a . (rho f_m) with
// rho f_m = 2 (rho u - j) (Eq. 3 with u_eq = u), i.e. the forcing term of Eq. 4.
template <typename C, int COEF>
__device__ __forceinline__ void collide_cell(C (&gq)[Q], C rho0, C half_eps, C Gx, C Gy,
                                             C c0, C c1, C c2, C c3,
                                             C omega, C two_tau, C omt, int guo = 0, C guo_c = C(0))
{
    C drho = 0, jx = 0, jy = 0;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        drho += gq[a];
        if (ex(a) == 1) jx += gq[a];
        if (ex(a) == -1) jx -= gq[a];
        if (ey(a) == 1) jy += gq[a];
        if (ey(a) == -1) jy -= gq[a];
    }
    const C rho = rho0 + drho;
    const C rx = jx + half_eps * rho * Gx;
    const C ry = jy + half_eps * rho * Gy;
    C rux, ruy;
    if constexpr (COEF == COEF_SCALAR) {          // rho u = (1 - e) r, written so that e << 1 keeps its digits
        rux = rx - c0 * rx;
        ruy = ry - c0 * ry;
    } else {                                      // rho u = (I - E) r
        rux = rx - (c0 * rx + c1 * ry);
        ruy = ry - (c2 * rx + c3 * ry);
    }
    if (guo) {
        const C fx = guo_c * (rux - jx), fy = guo_c * (ruy - jy);
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            C eu = C(0), ef = C(0);
            if (ex(a) == 1) { eu += rux; ef += fx; }
            if (ex(a) == -1) { eu -= rux; ef -= fx; }
            if (ey(a) == 1) { eu += ruy; ef += fy; }
            if (ey(a) == -1) { eu -= ruy; ef -= fy; }
            const C geq = wgt<C>(a) * (drho + C(3) * eu);
            gq[a] = gq[a] + omega * (geq - gq[a]) + wgt<C>(a) * ef;
        }
        return;
    }
    const C uex = two_tau * rux + omt * jx;   // rho u_eq, Eq. 16
    const C uey = two_tau * ruy + omt * jy;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        C eu = C(0);
        if (ex(a) == 1) eu += uex;
        if (ex(a) == -1) eu -= uex;
        if (ey(a) == 1) eu += uey;
        if (ey(a) == -1) eu -= uey;
        const C geq = wgt<C>(a) * (drho + C(3) * eu);
        gq[a] = gq[a] + omega * (geq - gq[a]);
    }
}

// Streamed (pre-collision) deviations of the VEC cells (y, x0 .. x0+VEC-1):
// g[q][i] = src_q(x - e_q) with periodic wrap, or the opposite population of the
// same cell for links that cross a bounce-back wall. Every lane of the warp must
// call this (the one-cell x shifts use warp shuffles).
template <typename T, int VEC, bool WALLS>
__device__ __forceinline__ void pull_chunk(const T *__restrict__ src, int64_t plane, int nx, int ny, int y, int xc,
                                           int cpr, int lane, typename Comp<T>::type (&g)[Q][VEC])
{
    using P = Pack<T, VEC>;
    const int x0 = xc * VEC;
    const bool left_in_warp = lane > 0 && xc > 0;         // lane-1 holds (y, x0 - VEC)
    const bool right_in_warp = lane < 31 && xc < cpr - 1; // lane+1 holds (y, x0 + VEC)
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int dy = ey(q), dx = ex(q);
        bool bb = false;
        int ys = y - dy;
        if (WALLS) bb = (dy == 1 && y == 0) || (dy == -1 && y == ny - 1);
        if (ys < 0) ys += ny;
        if (ys >= ny) ys -= ny;
        const T *pl = src + (int64_t)q * plane;
        if (WALLS && bb) ys = y;
        const T *plb = WALLS && bb ? src + (int64_t)opp(q) * plane : pl;
        const P pk = *reinterpret_cast<const P *>(plb + (int64_t)ys * nx + x0);
        if (dx == 0) {
#pragma unroll
            for (int i = 0; i < VEC; ++i) g[q][i] = to_c(pk.v[i]);
        } else if (dx == 1) {
            T left = shfl_up1(pk.v[VEC - 1]);
            if (!(WALLS && bb)) {
                if (!left_in_warp) left = pl[(int64_t)ys * nx + (x0 == 0 ? nx - 1 : x0 - 1)];
                g[q][0] = to_c(left);
#pragma unroll
                for (int i = 1; i < VEC; ++i) g[q][i] = to_c(pk.v[i - 1]);
            } else {
#pragma unroll
                for (int i = 0; i < VEC; ++i) g[q][i] = to_c(pk.v[i]);
            }
        } else {
            T right = shfl_down1(pk.v[0]);
            if (!(WALLS && bb)) {
                if (!right_in_warp) right = pl[(int64_t)ys * nx + (x0 + VEC == nx ? 0 : x0 + VEC)];
#pragma unroll
                for (int i = 0; i < VEC - 1; ++i) g[q][i] = to_c(pk.v[i + 1]);
                g[q][VEC - 1] = to_c(right);
            } else {
#pragma unroll
                for (int i = 0; i < VEC; ++i) g[q][i] = to_c(pk.v[i]);
            }
        }
    }
}

// Per-cell drag coefficients and body force of the VEC cells starting at cell0.
template <typename T, typename C, int VEC, int COEF, bool GF>
__device__ __forceinline__ void cell_params(const StepArgs<T, C> &a, int64_t cell0, C (&c0)[VEC], C (&c1)[VEC],
                                            C (&c2)[VEC], C (&c3)[VEC], C (&gxv)[VEC], C (&gyv)[VEC])
{
    load_vec<C, VEC>(a.coef, cell0, c0);
    if constexpr (COEF == COEF_TENSOR) {
        load_vec<C, VEC>(a.coef + a.plane, cell0, c1);
        load_vec<C, VEC>(a.coef + 2 * a.plane, cell0, c2);
        load_vec<C, VEC>(a.coef + 3 * a.plane, cell0, c3);
    } else {
#pragma unroll
        for (int i = 0; i < VEC; ++i) c1[i] = c2[i] = c3[i] = C(0);
    }
    if constexpr (GF) {
        load_vec<C, VEC>(a.gfield, cell0, gxv);
        load_vec<C, VEC>(a.gfield + a.plane, cell0, gyv);
    } else {
#pragma unroll
        for (int i = 0; i < VEC; ++i) { gxv[i] = a.gx; gyv[i] = a.gy; }
    }
}

template <typename T, int VEC, int COEF, bool GF, bool WALLS>
__global__ void __launch_bounds__(512) step_kernel(StepArgs<T, typename Comp<T>::type> a)
{
    using C = typename Comp<T>::type;
    using P = Pack<T, VEC>;
    const int lane = threadIdx.x & 31;
    const int nx = a.nx, ny = a.ny;
    const int cpr = nx / VEC;                              // chunks per row
    const int64_t nchunk = (int64_t)cpr * ny;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;

    for (int64_t base = warp0 * 32; base < nchunk; base += wstride * 32) {
        const int64_t c = base + lane;
        const bool active = c < nchunk;
        const int64_t ce = active ? c : nchunk - 1;
        const int y = (int)(ce / cpr);
        const int xc = (int)(ce - (int64_t)y * cpr);
        const int x0 = xc * VEC;

        C g[Q][VEC];
        pull_chunk<T, VEC, WALLS>(a.src, a.plane, nx, ny, y, xc, cpr, lane, g);

        const int64_t cell0 = (int64_t)y * nx + x0;
        C c0[VEC], c1[VEC], c2[VEC], c3[VEC], gxv[VEC], gyv[VEC];
        cell_params<T, C, VEC, COEF, GF>(a, cell0, c0, c1, c2, c3, gxv, gyv);

#pragma unroll
        for (int i = 0; i < VEC; ++i) {
            C gq[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) gq[q] = g[q][i];
            collide_cell<C, COEF>(gq, a.rho0, a.half_eps, gxv[i], gyv[i], c0[i], c1[i], c2[i], c3[i],
                                  a.omega, a.two_tau, a.one_m_two_tau, a.guo, a.guo_c);
#pragma unroll
            for (int q = 0; q < Q; ++q) g[q][i] = gq[q];
        }

        if (active) {
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                P out;
#pragma unroll
                for (int i = 0; i < VEC; ++i) out.v[i] = from_c<T>(g[q][i]);
                *reinterpret_cast<P *>(a.dst + (int64_t)q * a.plane + cell0) = out;
            }
        }
    }
}

// Density deviation (storage units) and flow velocity of one streamed cell:
// Eq. 15 with Eq. 6 (scalar d) or Eq. 18 (coefficient matrix), in the compute
// type. The storage scale cancels in u = (rho u) / rho.
template <typename C, int COEF>
__device__ __forceinline__ void cell_uv(const C (&g)[Q], C rho0, C half_eps, C Gx, C Gy, C c0, C c1, C c2, C c3,
                                        C &drho_o, C &u, C &v)
{
    C drho = 0, jx = 0, jy = 0;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        drho += g[a];
        if (ex(a) == 1) jx += g[a];
        if (ex(a) == -1) jx -= g[a];
        if (ey(a) == 1) jy += g[a];
        if (ey(a) == -1) jy -= g[a];
    }
    const C r = rho0 + drho;
    const C rx = jx + half_eps * r * Gx, ry = jy + half_eps * r * Gy;
    C rux, ruy;
    if constexpr (COEF == COEF_SCALAR) {
        rux = rx - c0 * rx;
        ruy = ry - c0 * ry;
    } else {
        rux = rx - (c0 * rx + c1 * ry);
        ruy = ry - (c2 * rx + c3 * ry);
    }
    drho_o = drho;
    u = rux / r;
    v = ruy / r;
}

// Moment / residual pass (same vectorised pulls as the step): flow velocity of
// the current state and, when m.prev is set, of the previous one; optional
// rho/u/v fields; per-block max|du|, max|u| and FP64 sums of u and v.
template <typename T, int VEC, int COEF, bool GF, bool WALLS>
__global__ void __launch_bounds__(256) moments_kernel(MomArgs<T, typename Comp<T>::type> m)
{
    using C = typename Comp<T>::type;
    const StepArgs<T, C> &a = m.s;
    const int lane = threadIdx.x & 31;
    const int nx = a.nx, ny = a.ny;
    const int cpr = nx / VEC;
    const int64_t nchunk = (int64_t)cpr * ny;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double dmax = 0.0, umax = 0.0, su = 0.0, sv = 0.0;
    for (int64_t base = warp0 * 32; base < nchunk; base += wstride * 32) {
        const int64_t c = base + lane;
        const bool active = c < nchunk;
        const int64_t ce = active ? c : nchunk - 1;
        const int y = (int)(ce / cpr);
        const int xc = (int)(ce - (int64_t)y * cpr);
        const int64_t cell0 = (int64_t)y * nx + xc * VEC;
        C c0[VEC], c1[VEC], c2[VEC], c3[VEC], gxv[VEC], gyv[VEC];
        cell_params<T, C, VEC, COEF, GF>(a, cell0, c0, c1, c2, c3, gxv, gyv);
        C g[Q][VEC];
        pull_chunk<T, VEC, WALLS>(a.src, a.plane, nx, ny, y, xc, cpr, lane, g);
        C uu[VEC], vv[VEC];
        C csu = 0, csv = 0, cmax = 0;
#pragma unroll
        for (int i = 0; i < VEC; ++i) {
            C gq[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) gq[q] = g[q][i];
            C dr;
            cell_uv<C, COEF>(gq, a.rho0, a.half_eps, gxv[i], gyv[i], c0[i], c1[i], c2[i], c3[i], dr, uu[i], vv[i]);
            if (active) {
                if (m.rho) m.rho[cell0 + i] = (float)(1.0 + (double)dr * (double)m.inv_scale);
                if (m.u) m.u[cell0 + i] = (float)uu[i];
                if (m.v) m.v[cell0 + i] = (float)vv[i];
            }
            csu += uu[i];
            csv += vv[i];
            cmax = fmax(cmax, fmax(fabs(uu[i]), fabs(vv[i])));
        }
        if (m.prev) {
            pull_chunk<T, VEC, WALLS>(m.prev, a.plane, nx, ny, y, xc, cpr, lane, g);
            C cd = 0;
#pragma unroll
            for (int i = 0; i < VEC; ++i) {
                C gq[Q];
#pragma unroll
                for (int q = 0; q < Q; ++q) gq[q] = g[q][i];
                C dr, up, vp;
                cell_uv<C, COEF>(gq, a.rho0, a.half_eps, gxv[i], gyv[i], c0[i], c1[i], c2[i], c3[i], dr, up, vp);
                cd = fmax(cd, fmax(fabs(uu[i] - up), fabs(vv[i] - vp)));
            }
            if (active) dmax = fmax(dmax, (double)cd);
        }
        if (active) {
            su += (double)csu;
            sv += (double)csv;
            umax = fmax(umax, (double)cmax);
        }
    }
    // block reduction in a fixed order: warp shuffles, then warp 0 over the warps
    __shared__ double sh[4][32];
    const int wid = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        dmax = fmax(dmax, __shfl_down_sync(0xffffffffu, dmax, off));
        umax = fmax(umax, __shfl_down_sync(0xffffffffu, umax, off));
        su += __shfl_down_sync(0xffffffffu, su, off);
        sv += __shfl_down_sync(0xffffffffu, sv, off);
    }
    if (lane == 0) { sh[0][wid] = dmax; sh[1][wid] = umax; sh[2][wid] = su; sh[3][wid] = sv; }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        dmax = lane < nw ? sh[0][lane] : 0.0;
        umax = lane < nw ? sh[1][lane] : 0.0;
        su = lane < nw ? sh[2][lane] : 0.0;
        sv = lane < nw ? sh[3][lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            dmax = fmax(dmax, __shfl_down_sync(0xffffffffu, dmax, off));
            umax = fmax(umax, __shfl_down_sync(0xffffffffu, umax, off));
            su += __shfl_down_sync(0xffffffffu, su, off);
            sv += __shfl_down_sync(0xffffffffu, sv, off);
        }
        if (lane == 0 && m.partials) {
            double *p = m.partials + 4 * (int64_t)blockIdx.x;
            p[0] = dmax; p[1] = umax; p[2] = su; p[3] = sv;
        }
    }
}

// One block folds the per-block partials in a fixed order.
__global__ void __launch_bounds__(256) reduce_partials_kernel(const double *partials, int n, double *out)
{
    double dmax = 0.0, umax = 0.0, su = 0.0, sv = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double *p = partials + 4 * (int64_t)i;
        dmax = fmax(dmax, p[0]);
        umax = fmax(umax, p[1]);
        su += p[2];
        sv += p[3];
    }
    __shared__ double sh[4][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        dmax = fmax(dmax, __shfl_down_sync(0xffffffffu, dmax, off));
        umax = fmax(umax, __shfl_down_sync(0xffffffffu, umax, off));
        su += __shfl_down_sync(0xffffffffu, su, off);
        sv += __shfl_down_sync(0xffffffffu, sv, off);
    }
    if (lane == 0) { sh[0][wid] = dmax; sh[1][wid] = umax; sh[2][wid] = su; sh[3][wid] = sv; }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        dmax = lane < nw ? sh[0][lane] : 0.0;
        umax = lane < nw ? sh[1][lane] : 0.0;
        su = lane < nw ? sh[2][lane] : 0.0;
        sv = lane < nw ? sh[3][lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            dmax = fmax(dmax, __shfl_down_sync(0xffffffffu, dmax, off));
            umax = fmax(umax, __shfl_down_sync(0xffffffffu, umax, off));
            su += __shfl_down_sync(0xffffffffu, su, off);
            sv += __shfl_down_sync(0xffffffffu, sv, off);
        }
        if (lane == 0) { out[0] = dmax; out[1] = umax; out[2] = su; out[3] = sv; }
    }
}

// Drag fraction e = 1 - d with d = 1 / (1 + eps nu / (2 kappa)) of Eq. 6, i.e.
// e = eps nu / (2 kappa + eps nu), evaluated in double; kappa = +inf (or
// eps nu = 0) gives 0, kappa = 0 gives 1. The step forms rho u = r - e r: storing
// e rather than d keeps full relative precision when the drag is weak (d -> 1),
// where FP32 d alone would leave 1 - d with only a few digits. flags bit 0 is set
// for a negative or NaN kappa. kmax_bits collects the largest finite
// kappa (the bit pattern of a non-negative float orders like an unsigned int).
template <typename CT>
__global__ void __launch_bounds__(256) coef_scalar_kernel(const float *kappa, CT *d, int64_t n, double eps_nu,
                                                          unsigned *flags, unsigned *kmax_bits)
{
    unsigned local_max = 0u;
    unsigned bad = 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float k = kappa[i];
        double dd;
        if (!(k >= 0.0f)) { bad = 1u; dd = 1.0; }
        else if (eps_nu == 0.0 || isinf(k)) dd = 0.0;
        else if (k == 0.0f) dd = 1.0;
        else dd = eps_nu / (2.0 * (double)k + eps_nu);
        d[i] = (CT)dd;
        if (k >= 0.0f && !isinf(k)) local_max = max(local_max, __float_as_uint(k));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        local_max = max(local_max, __shfl_down_sync(0xffffffffu, local_max, off));
        bad |= __shfl_down_sync(0xffffffffu, bad, off);
    }
    if ((threadIdx.x & 31) == 0) {
        if (local_max) atomicMax(kmax_bits, local_max);
        if (bad) atomicOr(flags, 1u);
    }
}

// Coarse-grid coefficient for a tensor K* (Eq. 18 in Eq. 15):
// rho u = (I + c K*^-1)^-1 r = (K* + c I)^-1 K* r = (I - E) r with E = c (K* + c I)^-1,
// c = eps nu / 2, r = j + eps rho G / 2. E (the drag part, like e of the scalar
// case) is stored as 4 planes; kstar is [n][4] (xx, xy, yx, yy).
template <typename CT>
__global__ void __launch_bounds__(256) coef_tensor_kernel(const double *kstar, CT *m, int64_t n, int64_t plane,
                                                          double c, unsigned *flags)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double kxx = kstar[4 * i], kxy = kstar[4 * i + 1], kyx = kstar[4 * i + 2], kyy = kstar[4 * i + 3];
        double mxx = 0.0, mxy = 0.0, myx = 0.0, myy = 0.0;
        if (!(isfinite(kxx) && isfinite(kxy) && isfinite(kyx) && isfinite(kyy))) {
            atomicOr(flags, 1u);
        } else if (c != 0.0) {
            const double axx = kxx + c, axy = kxy, ayx = kyx, ayy = kyy + c;
            const double det = axx * ayy - axy * ayx;
            if (!(fabs(det) > 0.0)) {
                atomicOr(flags, 2u);
            } else {
                mxx = c * ayy / det;
                mxy = -c * axy / det;
                myx = -c * ayx / det;
                myy = c * axx / det;
            }
        }
        m[i] = (CT)mxx;
        m[plane + i] = (CT)mxy;
        m[2 * plane + i] = (CT)myx;
        m[3 * plane + i] = (CT)myy;
    }
}

template <typename CT>
__global__ void __launch_bounds__(256) copy_force_kernel(const float *g, CT *dst, int64_t n, int64_t plane)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        dst[i] = (CT)g[i];
        dst[plane + i] = (CT)g[n + i];
    }
}

template <typename T, int VEC>
int occupancy_t(int coef_mode, bool gf, bool walls, int threads)
{
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
#define LBM_OCC_CASE(CM, GFv, WLv)                                                                   \
    if (coef_mode == CM && gf == GFv && walls == WLv)                                                \
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, step_kernel<T, VEC, CM, GFv, WLv>, threads, 0);
    LBM_OCC_CASE(COEF_SCALAR, false, false)
    LBM_OCC_CASE(COEF_SCALAR, false, true)
    LBM_OCC_CASE(COEF_SCALAR, true, false)
    LBM_OCC_CASE(COEF_SCALAR, true, true)
    LBM_OCC_CASE(COEF_TENSOR, false, false)
    LBM_OCC_CASE(COEF_TENSOR, false, true)
    LBM_OCC_CASE(COEF_TENSOR, true, false)
    LBM_OCC_CASE(COEF_TENSOR, true, true)
#undef LBM_OCC_CASE
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb < 1 ? 1 : nb;
}

template <typename T, int VEC>
cudaError_t launch_step_t(int coef_mode, bool gf, bool walls, const void *args, const GridLaunch &L, cudaStream_t st)
{
    using C = typename Comp<T>::type;
    const StepArgs<T, C> &a = *static_cast<const StepArgs<T, C> *>(args);
    dim3 grid(L.step_blocks), block(L.step_threads);
#define LBM_STEP_CASE(CM, GFv, WLv)                                                     \
    if (coef_mode == CM && gf == GFv && walls == WLv) {                                 \
        step_kernel<T, VEC, CM, GFv, WLv><<<grid, block, 0, st>>>(a);                   \
        return cudaGetLastError();                                                      \
    }
    LBM_STEP_CASE(COEF_SCALAR, false, false)
    LBM_STEP_CASE(COEF_SCALAR, false, true)
    LBM_STEP_CASE(COEF_SCALAR, true, false)
    LBM_STEP_CASE(COEF_SCALAR, true, true)
    LBM_STEP_CASE(COEF_TENSOR, false, false)
    LBM_STEP_CASE(COEF_TENSOR, false, true)
    LBM_STEP_CASE(COEF_TENSOR, true, false)
    LBM_STEP_CASE(COEF_TENSOR, true, true)
#undef LBM_STEP_CASE
    return cudaErrorInvalidValue;
}

template <typename T, int VEC>
cudaError_t launch_moments_t(int coef_mode, bool gf, bool walls, const void *args, const GridLaunch &L, cudaStream_t st)
{
    using C = typename Comp<T>::type;
    const MomArgs<T, C> &m = *static_cast<const MomArgs<T, C> *>(args);
    dim3 grid(L.mom_blocks), block(L.mom_threads);
#define LBM_MOM_CASE(CM, GFv, WLv)                                                      \
    if (coef_mode == CM && gf == GFv && walls == WLv) {                                 \
        moments_kernel<T, VEC, CM, GFv, WLv><<<grid, block, 0, st>>>(m);                \
        return cudaGetLastError();                                                      \
    }
    LBM_MOM_CASE(COEF_SCALAR, false, false)
    LBM_MOM_CASE(COEF_SCALAR, false, true)
    LBM_MOM_CASE(COEF_SCALAR, true, false)
    LBM_MOM_CASE(COEF_SCALAR, true, true)
    LBM_MOM_CASE(COEF_TENSOR, false, false)
    LBM_MOM_CASE(COEF_TENSOR, false, true)
    LBM_MOM_CASE(COEF_TENSOR, true, false)
    LBM_MOM_CASE(COEF_TENSOR, true, true)
#undef LBM_MOM_CASE
    return cudaErrorInvalidValue;
}

int elementwise_blocks(int64_t n)
{
    int64_t b = (n + 255) / 256;
    return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

}  // namespace

int step_vec(int storage, int nx)
{
    switch (storage) {
    case LBM_F32: return nx % 4 == 0 ? 4 : 1;
    case LBM_F16: return nx % 8 == 0 ? 8 : (nx % 2 == 0 ? 2 : 1);
    case LBM_F64: return nx % 2 == 0 ? 2 : 1;
    }
    return 1;
}

bool step_vec_ok(int storage, int nx, int vec)
{
    if (vec <= 0 || nx % vec) return false;
    switch (storage) {
    case LBM_F32: return vec == 1 || vec == 4 || vec == 8;
    case LBM_F16: return vec == 1 || vec == 2 || vec == 4 || vec == 8;
    case LBM_F64: return vec == 1 || vec == 2;
    }
    return false;
}

int step_blocks_per_sm(int storage, int coef_mode, bool gfield, bool walls, int nx, int threads, int vec)
{
    const int v = vec > 0 ? vec : step_vec(storage, nx);
    switch (storage) {
    case LBM_F32:
        return v == 8 ? occupancy_t<float, 8>(coef_mode, gfield, walls, threads)
                      : (v == 4 ? occupancy_t<float, 4>(coef_mode, gfield, walls, threads)
                                : occupancy_t<float, 1>(coef_mode, gfield, walls, threads));
    case LBM_F16:
        return v == 8 ? occupancy_t<__half, 8>(coef_mode, gfield, walls, threads)
                      : (v == 4 ? occupancy_t<__half, 4>(coef_mode, gfield, walls, threads)
                      : (v == 2 ? occupancy_t<__half, 2>(coef_mode, gfield, walls, threads)
                                : occupancy_t<__half, 1>(coef_mode, gfield, walls, threads)));
    case LBM_F64:
        return v == 2 ? occupancy_t<double, 2>(coef_mode, gfield, walls, threads)
                      : occupancy_t<double, 1>(coef_mode, gfield, walls, threads);
    }
    return 1;
}

cudaError_t launch_step(int storage, int coef_mode, bool gfield, bool walls, const void *args,
                        const GridLaunch &L, cudaStream_t st)
{
    int nx = 0;
    switch (storage) {
    case LBM_F32: {
        nx = static_cast<const StepArgs<float, float> *>(args)->nx;
        const int v = step_vec_ok(storage, nx, L.step_vec) ? L.step_vec : step_vec(storage, nx);
        return v == 8 ? launch_step_t<float, 8>(coef_mode, gfield, walls, args, L, st)
                      : (v == 4 ? launch_step_t<float, 4>(coef_mode, gfield, walls, args, L, st)
                                : launch_step_t<float, 1>(coef_mode, gfield, walls, args, L, st));
    }
    case LBM_F16: {
        nx = static_cast<const StepArgs<__half, float> *>(args)->nx;
        const int v = step_vec_ok(storage, nx, L.step_vec) ? L.step_vec : step_vec(storage, nx);
        return v == 8 ? launch_step_t<__half, 8>(coef_mode, gfield, walls, args, L, st)
                      : (v == 4 ? launch_step_t<__half, 4>(coef_mode, gfield, walls, args, L, st)
                      : (v == 2 ? launch_step_t<__half, 2>(coef_mode, gfield, walls, args, L, st)
                                : launch_step_t<__half, 1>(coef_mode, gfield, walls, args, L, st)));
    }
    case LBM_F64: {
        nx = static_cast<const StepArgs<double, double> *>(args)->nx;
        const int v = step_vec_ok(storage, nx, L.step_vec) ? L.step_vec : step_vec(storage, nx);
        return v == 2 ? launch_step_t<double, 2>(coef_mode, gfield, walls, args, L, st)
                      : launch_step_t<double, 1>(coef_mode, gfield, walls, args, L, st);
    }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_moments(int storage, int coef_mode, bool gfield, bool walls, const void *args,
                           const GridLaunch &L, cudaStream_t st)
{
    switch (storage) {
    case LBM_F32: {
        const int nx = static_cast<const MomArgs<float, float> *>(args)->s.nx;
        return step_vec(storage, nx) == 4 ? launch_moments_t<float, 4>(coef_mode, gfield, walls, args, L, st)
                                          : launch_moments_t<float, 1>(coef_mode, gfield, walls, args, L, st);
    }
    case LBM_F16: {
        const int nx = static_cast<const MomArgs<__half, float> *>(args)->s.nx;
        const int v = step_vec(storage, nx);
        return v == 8 ? launch_moments_t<__half, 8>(coef_mode, gfield, walls, args, L, st)
                      : (v == 2 ? launch_moments_t<__half, 2>(coef_mode, gfield, walls, args, L, st)
                                : launch_moments_t<__half, 1>(coef_mode, gfield, walls, args, L, st));
    }
    case LBM_F64: {
        const int nx = static_cast<const MomArgs<double, double> *>(args)->s.nx;
        return step_vec(storage, nx) == 2 ? launch_moments_t<double, 2>(coef_mode, gfield, walls, args, L, st)
                                          : launch_moments_t<double, 1>(coef_mode, gfield, walls, args, L, st);
    }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_reduce_partials(const double *partials, int n, double *out4, cudaStream_t st)
{
    reduce_partials_kernel<<<1, 256, 0, st>>>(partials, n, out4);
    return cudaGetLastError();
}

cudaError_t launch_coef_scalar(int storage, const float *kappa, void *coef, int64_t n, int64_t plane,
                               double eps_nu, unsigned *flags, unsigned *kmax_bits, cudaStream_t st)
{
    (void)plane;
    const int nb = elementwise_blocks(n);
    if (storage == LBM_F64)
        coef_scalar_kernel<double><<<nb, 256, 0, st>>>(kappa, static_cast<double *>(coef), n, eps_nu, flags, kmax_bits);
    else
        coef_scalar_kernel<float><<<nb, 256, 0, st>>>(kappa, static_cast<float *>(coef), n, eps_nu, flags, kmax_bits);
    return cudaGetLastError();
}

cudaError_t launch_coef_tensor(int storage, const double *kstar, void *coef, int64_t n, int64_t plane,
                               double c, unsigned *flags, cudaStream_t st)
{
    const int nb = elementwise_blocks(n);
    if (storage == LBM_F64)
        coef_tensor_kernel<double><<<nb, 256, 0, st>>>(kstar, static_cast<double *>(coef), n, plane, c, flags);
    else
        coef_tensor_kernel<float><<<nb, 256, 0, st>>>(kstar, static_cast<float *>(coef), n, plane, c, flags);
    return cudaGetLastError();
}

cudaError_t launch_copy_force(int storage, const float *g, void *dst, int64_t n, int64_t plane,
                              double, cudaStream_t st)
{
    const int nb = elementwise_blocks(n);
    if (storage == LBM_F64)
        copy_force_kernel<double><<<nb, 256, 0, st>>>(g, static_cast<double *>(dst), n, plane);
    else
        copy_force_kernel<float><<<nb, 256, 0, st>>>(g, static_cast<float *>(dst), n, plane);
    return cudaGetLastError();
}

}  // namespace lbm
