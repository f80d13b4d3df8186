// surrogate.cu -- the learned K* surrogate: patches, forward, backward, Adam,
// training loop, ensemble inference and the gate that sends doubtful patches
// back to local LBM. (An addition to the paper's method, which computes every
// K* by local LBM, Section 3; local LBM here stays the fallback and the arbiter.)
#include "lbm_internal.h"
#include "surrogate_kernels.cuh"

#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace lbm {

lbm_status fail(lbm_status s, const char *fmt, ...);
bool is_device_ptr(const void *p);
void count_launches(int64_t n);
int sm_count(int dev);
lbm_status local_keff_impl(const lbm_params *p, const float *kappa_dev, const lbm_leaf *leaves_dev, int32_t n_leaves,
                           double g_const, double tol_rel, int64_t max_steps, int32_t check_every,
                           int32_t persistent, double *keff_dev, int32_t *status_dev, int32_t *steps_dev,
                           void *cuda_stream, double time_limit_s);
double local_time_limit();

namespace sur {

// ------------------------------------------------------------ parameter layout
// Per model, FP32 master parameters laid out as
//   for l in 0..5: W_l [cout][cin][3][3], b_l [cout];  then W_h [2][64], b_h [2].
struct Layout {
    int64_t w[NLAYER], b[NLAYER], wh, bh, total;
    Layout()
    {
        int64_t o = 0;
        for (int l = 0; l < NLAYER; ++l) {
            w[l] = o;
            o += (int64_t)cout_of(l) * cin_real(l) * 9;
            b[l] = o;
            o += cout_of(l);
        }
        wh = o;
        o += 2 * 64;
        bh = o;
        o += 2;
        total = o;
    }
};
static const Layout LAYOUT;

// ------------------------------------------------------------------ kernels

// Is s a leaf size the input planes are defined for: a divisor of 32, or a multiple of 64 up to 1024.
__host__ __device__ inline bool patch_size_ok(int s)
{
    return (s >= 1 && s <= IMG && IMG % s == 0) || (s >= 64 && s <= 1024 && s % 64 == 0);
}

// Leaf -> the nine input planes [n][9][32][32] and (mean, std, gradient energy) of its 32 x 32
// log-K patch. The leaf's log K is first put on a 64 x 64 plane (each cell repeated 64 / s times
// per axis for s <= 32, the leaf itself for s = 64, means of log K over (s / 64)^2 blocks above);
// phase plane 2 a + b holds that plane's cell (2 i + a, 2 j + b) at (i, j). Plane 4 is the
// constant log2(s) / 6. The 32 x 32 patch the statistics describe is the mean of the four phase
// planes (the leaf itself for s <= 32, its 2 x 2 block means for s = 64). Planes 5-8 are its
// context: the harmonic and arithmetic means of K along each row of that patch, then along each
// column, in log K, repeated across the row or down the column. One CTA per leaf; an invalid leaf
// (size, or not inside the field) gets zero planes and sets *bad (may be NULL).
__global__ void __launch_bounds__(256) patch_kernel(const float *kappa, int nx, int ny, const int *leaves,
                                                   float *x, float *stats, int *bad)
{
    const int i = blockIdx.x;
    const int x0 = leaves[3 * i], y0 = leaves[3 * i + 1], s = leaves[3 * i + 2];
    float *xi = x + (int64_t)i * IN_PLANES * PIX;
    const bool valid = patch_size_ok(s) && x0 >= 0 && y0 >= 0 && (int64_t)x0 + s <= nx && (int64_t)y0 + s <= ny;
    if (!valid) {
        for (int q = threadIdx.x; q < IN_PLANES * PIX; q += blockDim.x) xi[q] = 0.0f;
        if (threadIdx.x < 3) stats[3 * i + threadIdx.x] = 0.0f;
        if (threadIdx.x == 0 && bad) atomicExch(bad, 1);
        return;
    }
    __shared__ float p[PIX];
    __shared__ double red[3][8];
    const float size_plane = log2f((float)s) / 6.0f;
    for (int q = threadIdx.x; q < PIX; q += blockDim.x) {
        const int py = q >> 5, px = q & 31;
        float v[4];
        if (s <= IMG) {                        // all four phases are the same cell
            const int r = IMG / s;
            v[0] = v[1] = v[2] = v[3] = logf(kappa[(int64_t)(y0 + py / r) * nx + x0 + px / r]);
        } else {
            const int r = s / 64;
#pragma unroll
            for (int ph = 0; ph < 4; ++ph) {
                const int Y = 2 * py + (ph >> 1), X = 2 * px + (ph & 1);
                if (r == 1) {
                    v[ph] = logf(kappa[(int64_t)(y0 + Y) * nx + x0 + X]);
                } else {
                    double acc = 0.0;
                    for (int a = 0; a < r; ++a)
                        for (int b = 0; b < r; ++b)
                            acc += (double)logf(kappa[(int64_t)(y0 + Y * r + a) * nx + x0 + X * r + b]);
                    v[ph] = (float)(acc / (r * r));
                }
            }
        }
#pragma unroll
        for (int ph = 0; ph < 4; ++ph) xi[ph * PIX + q] = v[ph];
        xi[4 * PIX + q] = size_plane;
        p[q] = 0.25f * ((v[0] + v[1]) + (v[2] + v[3]));
    }
    __syncthreads();
    // context planes: harmonic and arithmetic means of K = exp(p) along each row and each column
    __shared__ double rk[IMG], ri[IMG], ck[IMG], ci[IMG];
    if (threadIdx.x < IMG) {
        const int r = threadIdx.x;
        double a = 0.0, b = 0.0;
        for (int c = 0; c < IMG; ++c) { a += exp((double)p[r * IMG + c]); b += exp(-(double)p[r * IMG + c]); }
        rk[r] = a;
        ri[r] = b;
    } else if (threadIdx.x < 2 * IMG) {
        const int c = threadIdx.x - IMG;
        double a = 0.0, b = 0.0;
        for (int r = 0; r < IMG; ++r) { a += exp((double)p[r * IMG + c]); b += exp(-(double)p[r * IMG + c]); }
        ck[c] = a;
        ci[c] = b;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < PIX; q += blockDim.x) {
        const int py = q >> 5, px = q & 31;
        xi[5 * PIX + q] = (float)(-log(ri[py] / IMG));
        xi[6 * PIX + q] = (float)log(rk[py] / IMG);
        xi[7 * PIX + q] = (float)(-log(ci[px] / IMG));
        xi[8 * PIX + q] = (float)log(ck[px] / IMG);
    }
    double sm = 0.0, sq = 0.0, ge = 0.0;
    for (int q = threadIdx.x; q < PIX; q += blockDim.x) {
        const int py = q >> 5, px = q & 31;
        const double v = p[q];
        sm += v;
        sq += v * v;
        if (px < 31) { const double d = p[q + 1] - v; ge += d * d; }
        if (py < 31) { const double d = p[q + 32] - v; ge += d * d; }
    }
    for (int off = 16; off > 0; off >>= 1) {
        sm += __shfl_down_sync(0xffffffffu, sm, off);
        sq += __shfl_down_sync(0xffffffffu, sq, off);
        ge += __shfl_down_sync(0xffffffffu, ge, off);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[0][w] = sm; red[1][w] = sq; red[2][w] = ge; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, c = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { a += red[0][k]; b += red[1][k]; c += red[2][k]; }
        const double mean = a / PIX;
        const double var = b / PIX - mean * mean;
        stats[3 * i] = (float)mean;
        stats[3 * i + 1] = (float)sqrt(var > 0.0 ? var : 0.0);
        stats[3 * i + 2] = (float)(0.5 * c / (IMG * (IMG - 1)));
    }
}

// FP32 input planes [n][9][32][32] (rows idx[b]) -> BF16 16-channel activation (act_at layout):
// channels 0-3 and 5-8 (log-K planes) as (x - shift) / scale, channel 4 (size) as is, 9-15 zero.
__global__ void __launch_bounds__(256) input_kernel(const float *x, const int *idx, int B, float shift, float scale,
                                                   __nv_bfloat16 *out)
{
    const int64_t total = (int64_t)B * PIX;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / PIX), q = (int)(t - (int64_t)b * PIX);
        const int64_t src = (int64_t)(idx ? idx[b] : b) * IN_PLANES * PIX;
        uint4 o[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
        __nv_bfloat16 *ob = reinterpret_cast<__nv_bfloat16 *>(o);
#pragma unroll
        for (int c = 0; c < IN_PLANES; ++c) {
            const float v = x[src + c * PIX + q];
            ob[c] = __float2bfloat16_rn(c == 4 ? v : (v - shift) / scale);
        }
        *reinterpret_cast<uint4 *>(out + act_at(b, q, 0, CIN0)) = o[0];
        *reinterpret_cast<uint4 *>(out + act_at(b, q, 8, CIN0)) = o[1];
    }
}

// B operand of the forward conv: row n = c_out, k = tap * CIN_P + c_in.
__global__ void pack_fwd_kernel(const float *w, int cin, int cin_p, int cout, __nv_bfloat16 *out)
{
    const int K = 9 * cin_p;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cout * K; t += gridDim.x * blockDim.x) {
        const int n = t / K, k = t - n * K, tap = k / cin_p, ci = k - tap * cin_p;
        const float v = ci < cin ? w[((int64_t)n * cin + ci) * 9 + tap] : 0.0f;
        out[umma::core_offset(n, k, K) / 2] = __float2bfloat16_rn(v);
    }
}

// B operand of the input-gradient conv: row n = c_in, k = tap' * COUT + c_out, value
// W[c_out][c_in][8 - tap'] (the transposed, spatially flipped kernel).
__global__ void pack_bwd_kernel(const float *w, int cin, int cout, __nv_bfloat16 *out)
{
    const int K = 9 * cout;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cin * K; t += gridDim.x * blockDim.x) {
        const int n = t / K, k = t - n * K, tp = k / cout, co = k - tp * cout;
        out[umma::core_offset(n, k, K) / 2] = __float2bfloat16_rn(w[((int64_t)co * cin + n) * 9 + (8 - tp)]);
    }
}

// Global average pooling of the last activation and the linear head. One CTA per image;
// thread t reads elements t, t + 256, ... of each 8-channel plane (always channel t % 8), and
// the 32 partial sums of a channel are folded in a fixed order.
__global__ void __launch_bounds__(256) gap_head_kernel(const __nv_bfloat16 *act, const float *wh, const float *bh,
                                                      float *pooled, float *y)
{
    const int b = blockIdx.x, t = threadIdx.x;
    __shared__ float part[32][64];
    __shared__ float pool[64];
    for (int g = 0; g < 8; ++g) {
        const __nv_bfloat16 *plane = act + act_at(b, 0, 8 * g, 64);
        float s = 0.0f;
        for (int e = t; e < PIX * 8; e += 256) s += __bfloat162float(plane[e]);
        part[t >> 3][8 * g + (t & 7)] = s;
    }
    __syncthreads();
    if (t < 64) {
        float v = 0.0f;
        for (int k = 0; k < 32; ++k) v += part[k][t];
        v /= PIX;
        pool[t] = v;
        pooled[(int64_t)b * 64 + t] = v;
    }
    __syncthreads();
    if (t < 2) {
        float acc = bh[t];
        for (int k = 0; k < 64; ++k) acc += wh[t * 64 + k] * pool[k];
        y[(int64_t)b * 2 + t] = acc;
    }
}

// Loss L = mean((y - t)^2) over B x 2 entries (targets already standardised), the head's
// gradients and dL/dpool. One CTA; every sum runs in a fixed order.
__global__ void __launch_bounds__(256) loss_head_backward_kernel(const float *y, const float *t, const float *pooled,
                                                                const float *wh, int B, float *dpool, float *gwh,
                                                                float *gbh, float *loss)
{
    __shared__ float dy[2][1024];
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        dy[0][b] = 2.0f * (y[2 * b] - t[2 * b]) / (2.0f * B);
        dy[1][b] = 2.0f * (y[2 * b + 1] - t[2 * b + 1]) / (2.0f * B);
    }
    __syncthreads();
    if (threadIdx.x < 128) {
        const int o = threadIdx.x >> 6, c = threadIdx.x & 63;
        float acc = 0.0f;
        for (int b = 0; b < B; ++b) acc += dy[o][b] * pooled[(int64_t)b * 64 + c];
        gwh[o * 64 + c] = acc;
    } else if (threadIdx.x < 130) {
        const int o = threadIdx.x - 128;
        float acc = 0.0f;
        for (int b = 0; b < B; ++b) acc += dy[o][b];
        gbh[o] = acc;
    } else if (threadIdx.x == 130) {
        double acc = 0.0;
        for (int b = 0; b < B; ++b) {
            const double e0 = (double)y[2 * b] - t[2 * b], e1 = (double)y[2 * b + 1] - t[2 * b + 1];
            acc += e0 * e0 + e1 * e1;
        }
        *loss = (float)(acc / (2.0 * B));
    }
    for (int q = threadIdx.x; q < B * 64; q += blockDim.x) {
        const int b = q >> 6, c = q & 63;
        dpool[q] = dy[0][b] * wh[c] + dy[1][b] * wh[64 + c];
    }
}

// dL/d(last activation), ReLU mask applied: dpool / 1024 where the activation is positive.
__global__ void __launch_bounds__(256) gap_backward_kernel(const float *dpool, const __nv_bfloat16 *act, int B,
                                                          __nv_bfloat16 *dact)
{
    const int64_t total = (int64_t)B * PIX * 64;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t / (PIX * 64);
        const int c = (int)((t / (PIX * 8)) & 7) * 8 + (int)(t & 7);      // act_at layout
        const float g = __bfloat162float(act[t]) > 0.0f ? dpool[b * 64 + c] / PIX : 0.0f;
        dact[t] = __float2bfloat16_rn(g);
    }
}

// Bias gradient partials: bpart[g][co] = sum over images g, g + G, ... and all their pixels of
// dout[img][p][co] (dout holds the ReLU-masked gradient of the layer's output). Thread t sums
// channel t % COUT over pixels p = t / COUT (mod 256 / COUT); the phases are folded in order.
template <int COUT>
__global__ void __launch_bounds__(256) bias_grad_kernel(const __nv_bfloat16 *dout, int B, float *bpart)
{
    constexpr int NPH = 256 / COUT;
    const int t = threadIdx.x, co = t % COUT, ph = t / COUT;
    float acc = 0.0f;
    for (int img = blockIdx.x; img < B; img += gridDim.x)
        for (int p = ph; p < PIX; p += NPH) acc += __bfloat162float(dout[act_at(img, p, co, COUT)]);
    __shared__ float red[256];
    red[t] = acc;
    __syncthreads();
    if (t < COUT) {
        float v = 0.0f;
        for (int k = 0; k < NPH; ++k) v += red[k * COUT + t];
        bpart[(int64_t)blockIdx.x * COUT + t] = v;
    }
}

// Folds the per-CTA partials of wgrad_tc_kernel (CTA b holds input-channel part b % P; its rows h
// are separate partials) into W's gradient [co][ci][3][3] and the bias partials into b's, in a
// fixed order (deterministic).
__global__ void __launch_bounds__(256) wgrad_tc_reduce_kernel(const float *part, int grid, int P, int HM, int cout,
                                                             int cip, int cin, const float *bpart, int nb, float *gw,
                                                             float *gb)
{
    const int nw = cout * cin * 9;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nw + cout; t += gridDim.x * blockDim.x) {
        if (t < nw) {
            const int co = t / (cin * 9), rem = t - co * cin * 9, ci = rem / 9, tap = rem - ci * 9;
            const int pp = ci / cip, c = ci - pp * cip;
            float acc = 0.0f;
            for (int b = pp; b < grid; b += P)
                for (int h = 0; h < HM; ++h)
                    acc += part[((((int64_t)b * HM + h) * 9 + tap) * cout + co) * cip + c];
            gw[t] = acc;
        } else {
            const int co = t - nw;
            float acc = 0.0f;
            for (int b = 0; b < nb; ++b) acc += bpart[(int64_t)b * cout + co];
            gb[co] = acc;
        }
    }
}

// Adam (Kingma & Ba) on the FP32 master parameters.
__global__ void __launch_bounds__(256) adam_kernel(float *p, const float *g, float *m, float *v, int64_t n, float lr,
                                                  float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Sum and sum of squares of the log-K phase planes of x [n][9][32][32], per block (fixed order).
__global__ void __launch_bounds__(256) input_moments_kernel(const float *x, int n, double *part)
{
    double s = 0.0, q = 0.0;
    const int64_t per = 4 * PIX;
    const int64_t total = (int64_t)n * per;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / per, pq = t - i * per;
        const double v = x[i * IN_PLANES * PIX + pq];
        s += v;
        q += v * v;
    }
    __shared__ double sh[2][256];
    sh[0][threadIdx.x] = s;
    sh[1][threadIdx.x] = q;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < 256; ++k) { a += sh[0][k]; b += sh[1][k]; }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

// Per-leaf target base for the two components, cw[i] = (c_xx, w_xx, c_yy, w_yy): the network learns
// (log K* - c) / w. It is computed on the 64 x 64 log-K plane the four phase planes form (the
// leaf itself for 64 cells, the leaf repeated for smaller ones). Mode 0: c = mean log K, w = 1.
// Modes 1 and 2 centre on the layered-medium bounds (for flow along x, rows as parallel series
// tubes give A_y(H_x K) below and columns as series parallel slabs give H_x(A_y K) above; the same
// with x and y swapped for K*_yy): c = the midpoint of the log bounds, and w = 1 (mode 1) or half
// the log width, at least 0.05 (mode 2). One block per leaf, FP64 sums in a fixed order.
__global__ void __launch_bounds__(256) patch_base_kernel(const float *x, int n, int mode, float4 *cw)
{
    constexpr int F = 64;                      // side of the full plane
    __shared__ double K[F][F + 1];
    __shared__ double rowK[F], rowI[F], colK[F], colI[F];
    __shared__ double lsum;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const float *xi = x + (int64_t)i * IN_PLANES * PIX;
        for (int q = threadIdx.x; q < F * F; q += 256) {
            const int Y = q / F, X = q % F;
            K[Y][X] = (double)xi[((Y & 1) * 2 + (X & 1)) * PIX + (Y >> 1) * IMG + (X >> 1)];   // log K for now
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0;
            for (int r = 0; r < F; ++r)
                for (int c = 0; c < F; ++c) a += K[r][c];
            lsum = a;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < F * F; q += 256) K[q / F][q % F] = exp(K[q / F][q % F]);
        __syncthreads();
        if (threadIdx.x < F) {
            const int r = threadIdx.x;
            double sk = 0.0, si = 0.0;
            for (int c = 0; c < F; ++c) { sk += K[r][c]; si += 1.0 / K[r][c]; }
            rowK[r] = sk;
            rowI[r] = si;
        } else if (threadIdx.x < 2 * F) {
            const int c = threadIdx.x - F;
            double sk = 0.0, si = 0.0;
            for (int r = 0; r < F; ++r) { sk += K[r][c]; si += 1.0 / K[r][c]; }
            colK[c] = sk;
            colI[c] = si;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float4 o;
            if (mode == 0) {
                const float m = (float)(lsum / (F * F));
                o = make_float4(m, 1.0f, m, 1.0f);
            } else {
                double ahx = 0.0, hax = 0.0, ahy = 0.0, hay = 0.0;
                for (int k = 0; k < F; ++k) {
                    ahx += F / rowI[k];            // H_x of row k
                    hax += F / colK[k];            // 1 / A_y of column k
                    ahy += F / colI[k];            // H_y of column k
                    hay += F / rowK[k];            // 1 / A_x of row k
                }
                const double lox = log(ahx / F), hix = log(F / hax);
                const double loy = log(ahy / F), hiy = log(F / hay);
                const float wx = mode == 2 ? (float)fmax(0.5 * (hix - lox), 0.05) : 1.0f;
                const float wy = mode == 2 ? (float)fmax(0.5 * (hiy - loy), 0.05) : 1.0f;
                o = make_float4((float)(0.5 * (lox + hix)), wx, (float)(0.5 * (loy + hiy)), wy);
            }
            cw[i] = o;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ Darcy base (target mode 3)
// The Darcy K* of each leaf by finite volumes: the flux across the face between two neighbouring
// cells is k_f (p_i - p_j + G . (x_j - x_i)) with k_f the harmonic mean of the two cells, every cell
// conserves mass, the leaf is periodic, and a unit force drives the flow along x, then along y.
// K* along the drive is the mean face flux. The pressure system is solved by conjugate gradients
// with the diagonal as preconditioner, in FP32 with the cross-thread sums in FP64, to a relative
// residual of 1e-5 (K* then agrees with an FP64 direct solve to a few 1e-6). The leaf's log K is
// read back from the input planes (phase plane 0 sampled every 32 / s pixels for s <= 32, the four
// phase planes for 64 cells; above 64 cells the 64 x 64 plane stands for the leaf).
// Leaves of up to 32 cells are solved by one warp each (darcy_small_kernel), larger ones by a
// CTA each (darcy_big_kernel); each kernel passes over the leaves of the other kind.
constexpr int DB_N = 64;
constexpr int DB_CELLS = DB_N * DB_N;
constexpr int DB_MAXIT = 4000;
constexpr int DBS_WARPS = 8;                                 // warps per CTA of the small-leaf kernel
constexpr int DBS_CELLS = IMG * IMG;                         // cells per warp (leaves up to 32)
constexpr size_t DBS_SMEM = (size_t)DBS_WARPS * 6 * DBS_CELLS * sizeof(float);
constexpr int DBB_THREADS = 256;
constexpr size_t DBB_SMEM = (size_t)6 * DB_CELLS * sizeof(float);

__device__ __forceinline__ int darcy_size(const float *xi)
{
    const int s = (int)lrintf(exp2f(6.0f * xi[4 * PIX]));   // the size plane holds log2(s) / 6
    return s < 1 ? 1 : (s > DB_N ? DB_N : s);
}

__device__ __forceinline__ float harmonic2f(double a, double b)
{
    if (isinf(a)) return (float)(isinf(b) ? a : 2.0 * b);
    if (isinf(b)) return (float)(2.0 * a);
    return a + b > 0.0 ? (float)(2.0 * a * b / (a + b)) : 0.0f;
}

// A group of NT threads solving one leaf: one warp (NT = 32) or the whole CTA.
template <int NT> struct DarcyGroup {
    __device__ static int rank() { return threadIdx.x % NT; }
    __device__ static void sync()
    {
        if constexpr (NT == 32) __syncwarp(); else __syncthreads();
    }
    // (a, b) summed over the group in a fixed order; every thread gets the sums
    __device__ static void sum2(double &a, double &b, double (*red)[2])
    {
        for (int off = 16; off > 0; off >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, off);
            b += __shfl_xor_sync(0xffffffffu, b, off);
        }
        if constexpr (NT > 32) {
            if ((threadIdx.x & 31) == 0) {
                red[threadIdx.x >> 5][0] = a;
                red[threadIdx.x >> 5][1] = b;
            }
            __syncthreads();
            double x = 0.0, y = 0.0;
            for (int k = 0; k < NT / 32; ++k) { x += red[k][0]; y += red[k][1]; }
            __syncthreads();
            a = x;
            b = y;
        }
    }
};

// K*_xx and K*_yy of the leaf whose input planes start at xi; the group's work arrays hold cap cells.
template <int NT>
__device__ void darcy_leaf(const float *xi, int s, float *KX, float *KY, float *P, float *R, float *Dv, float *AD,
                          double (*red)[2], double (&kd)[2])
{
    using G = DarcyGroup<NT>;
    const int nc = s * s, r0 = G::rank();
    for (int c = r0; c < nc; c += NT) {
        const int y = c / s, xx = c - y * s;
        float v;
        if (s <= IMG) {
            const int r = IMG / s;
            v = xi[(y * r) * IMG + xx * r];
        } else {
            v = xi[((y & 1) * 2 + (xx & 1)) * PIX + (y >> 1) * IMG + (xx >> 1)];
        }
        P[c] = v;                                          // log K, for now
    }
    G::sync();
    for (int c = r0; c < nc; c += NT) {
        const int y = c / s, xx = c - y * s;
        const double k = exp((double)P[c]);
        KX[c] = harmonic2f(k, exp((double)P[y * s + (xx + 1 == s ? 0 : xx + 1)]));
        KY[c] = harmonic2f(k, exp((double)P[(y + 1 == s ? 0 : y + 1) * s + xx]));
    }
    G::sync();
    for (int drive = 0; drive < 2; ++drive) {
        // A p = b with (A p)_c = sum over the faces of c of k_f (p_c - p_neighbour) and
        // b_c = k_f(behind c) - k_f(ahead of c) along the drive
        float prr = 0.0f, prz = 0.0f;
        for (int c = r0; c < nc; c += NT) {
            const int y = c / s, xx = c - y * s;
            const int cl = y * s + (xx == 0 ? s - 1 : xx - 1), cd = (y == 0 ? s - 1 : y - 1) * s + xx;
            const float b = drive == 0 ? KX[cl] - KX[c] : KY[cd] - KY[c];
            const float dg = KX[c] + KX[cl] + KY[c] + KY[cd];
            const float z = dg > 0.0f ? b / dg : 0.0f;
            P[c] = 0.0f;
            R[c] = b;
            Dv[c] = z;
            prr = fmaf(b, b, prr);
            prz = fmaf(b, z, prz);
        }
        double rr = prr, rz = prz;
        G::sum2(rr, rz, red);
        const double stop = 1e-10 * rr;                    // (1e-5 relative residual)^2
        for (int it = 0; it < DB_MAXIT && rr > stop; ++it) {
            float pdad = 0.0f;
            for (int c = r0; c < nc; c += NT) {
                const int y = c / s, xx = c - y * s;
                const int cl = y * s + (xx == 0 ? s - 1 : xx - 1), cr = y * s + (xx + 1 == s ? 0 : xx + 1);
                const int cd = (y == 0 ? s - 1 : y - 1) * s + xx, cu = (y + 1 == s ? 0 : y + 1) * s + xx;
                const float dc = Dv[c];
                const float ad = KX[c] * (dc - Dv[cr]) + KX[cl] * (dc - Dv[cl]) + KY[c] * (dc - Dv[cu]) +
                                 KY[cd] * (dc - Dv[cd]);
                AD[c] = ad;
                pdad = fmaf(dc, ad, pdad);
            }
            double dad = pdad, unused = 0.0;
            G::sum2(dad, unused, red);
            if (!(dad > 0.0)) break;                          // a direction in the null space
            const float alpha = (float)(rz / dad);
            float prr2 = 0.0f, prz2 = 0.0f;
            for (int c = r0; c < nc; c += NT) {
                const int y = c / s, xx = c - y * s;
                const int cl = y * s + (xx == 0 ? s - 1 : xx - 1), cd = (y == 0 ? s - 1 : y - 1) * s + xx;
                P[c] = fmaf(alpha, Dv[c], P[c]);
                const float r = fmaf(-alpha, AD[c], R[c]);
                R[c] = r;
                const float dg = KX[c] + KX[cl] + KY[c] + KY[cd];
                prr2 = fmaf(r, r, prr2);
                prz2 = dg > 0.0f ? fmaf(r, r / dg, prz2) : prz2;
            }
            double rr2 = prr2, rz2 = prz2;
            G::sum2(rr2, rz2, red);
            const float beta = (float)(rz2 / rz);
            rz = rz2;
            rr = rr2;
            for (int c = r0; c < nc; c += NT) {
                const int y = c / s, xx = c - y * s;
                const int cl = y * s + (xx == 0 ? s - 1 : xx - 1), cd = (y == 0 ? s - 1 : y - 1) * s + xx;
                const float dg = KX[c] + KX[cl] + KY[c] + KY[cd];
                Dv[c] = fmaf(beta, Dv[c], dg > 0.0f ? R[c] / dg : 0.0f);
            }
            G::sync();
        }
        // mean face flux along the drive
        float pq = 0.0f;
        for (int c = r0; c < nc; c += NT) {
            const int y = c / s, xx = c - y * s;
            pq += drive == 0 ? KX[c] * (P[c] - P[y * s + (xx + 1 == s ? 0 : xx + 1)] + 1.0f)
                             : KY[c] * (P[c] - P[(y + 1 == s ? 0 : y + 1) * s + xx] + 1.0f);
        }
        double q = pq, unused = 0.0;
        G::sum2(q, unused, red);
        kd[drive] = q / nc;
        G::sync();
    }
}

// Leaves of up to 32 cells: one warp per leaf, eight warps per CTA, each with its own work arrays.
__global__ void __launch_bounds__(DBS_WARPS * 32) darcy_small_kernel(const float *x, int n, float4 *cw)
{
    extern __shared__ __align__(16) unsigned char dsm_raw[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *base = reinterpret_cast<float *>(dsm_raw) + (size_t)w * 6 * DBS_CELLS;
    float *KX = base, *KY = KX + DBS_CELLS, *P = KY + DBS_CELLS, *R = P + DBS_CELLS, *Dv = R + DBS_CELLS,
          *AD = Dv + DBS_CELLS;
    for (int i = blockIdx.x * DBS_WARPS + w; i < n; i += gridDim.x * DBS_WARPS) {
        const float *xi = x + (int64_t)i * IN_PLANES * PIX;
        const int s = darcy_size(xi);
        if (s > IMG) continue;                              // the CTA kernel's leaf
        double kd[2];
        darcy_leaf<32>(xi, s, KX, KY, P, R, Dv, AD, nullptr, kd);
        if (lane == 0) cw[i] = make_float4((float)log(kd[0]), 1.0f, (float)log(kd[1]), 1.0f);
        __syncwarp();
    }
}

// Leaves of 64 cells and more: one CTA per leaf.
__global__ void __launch_bounds__(DBB_THREADS) darcy_big_kernel(const float *x, int n, float4 *cw)
{
    extern __shared__ __align__(16) unsigned char dsm_raw[];
    float *KX = reinterpret_cast<float *>(dsm_raw);
    float *KY = KX + DB_CELLS, *P = KY + DB_CELLS, *R = P + DB_CELLS, *Dv = R + DB_CELLS, *AD = Dv + DB_CELLS;
    __shared__ double red[DBB_THREADS / 32][2];
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const float *xi = x + (int64_t)i * IN_PLANES * PIX;
        const int s = darcy_size(xi);
        if (s <= IMG) continue;                             // the warp kernel's leaf
        double kd[2];
        darcy_leaf<DBB_THREADS>(xi, s, KX, KY, P, R, Dv, AD, red, kd);
        if (threadIdx.x == 0) cw[i] = make_float4((float)log(kd[0]), 1.0f, (float)log(kd[1]), 1.0f);
        __syncthreads();
    }
}

// Targets of a mini-batch: t[b] = ty[idx[b]] (two components).
__global__ void gather_targets_kernel(const float *ty, const int *idx, int B, float *t)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
        t[2 * b] = ty[2 * (int64_t)idx[b]];
        t[2 * b + 1] = ty[2 * (int64_t)idx[b] + 1];
    }
}

// Standardised network outputs -> log K*: c + w (y * std + mean) per component, [model][n][2].
__global__ void destandardise_kernel(float *y, int n, int nmodels, const float4 *cw, float m0, float s0, float m1,
                                     float s1)
{
    const int64_t n2 = (int64_t)nmodels * n * 2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 b = cw[(i >> 1) % n];
        y[i] = (i & 1) ? b.z + b.w * (y[i] * s1 + m1) : b.x + b.y * (y[i] * s0 + m0);
    }
}

// ---------------------------------------------------------------- launchers

int nblk(int64_t n) { int64_t b = (n + 255) / 256; return (int)(b < 1 ? 1 : (b > 8192 ? 8192 : b)); }

// Per-leaf target base of the given mode: patch_base_kernel (modes 0-2) or the batched Darcy
// solve (mode 3: a warp per leaf up to 32 cells, a CTA per larger leaf).
cudaError_t launch_base(const float *x, int n, int mode, float4 *cw, cudaStream_t st)
{
    if (mode == 3) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(darcy_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DBS_SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(darcy_big_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DBB_SMEM);
        if (e != cudaSuccess) return e;
        const int sms = sm_count(dev);
        const int gs = (n + DBS_WARPS - 1) / DBS_WARPS;
        darcy_small_kernel<<<gs < sms ? gs : sms, DBS_WARPS * 32, DBS_SMEM, st>>>(x, n, cw);
        darcy_big_kernel<<<n < 2 * sms ? n : 2 * sms, DBB_THREADS, DBB_SMEM, st>>>(x, n, cw);
        count_launches(1);
    } else {
        patch_base_kernel<<<n < 65535 ? n : 65535, 256, 0, st>>>(x, n, mode, cw);
    }
    count_launches(1);
    return cudaGetLastError();
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link-time libcuda dependency)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Tensor map over BF16 activations in channel-group planes [nimg][cin_p/8][32][32][8], seen as 4-D
// (8 channels, 32 columns, 32 rows, nimg * cin_p / 8 planes): boxes of 8 channels x 34 columns x 18 rows
// of one plane (a half-image tile with its one-pixel halo); out-of-range pixels read as zero.
static cudaError_t encode_halo_map(CUtensorMap *map, const __nv_bfloat16 *act, int cin_p, int nimg)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[4] = {8, IMG, IMG, (cuuint64_t)nimg * (cin_p / 8)};
    const cuuint64_t strides[3] = {8 * 2, (cuuint64_t)IMG * 8 * 2, (cuuint64_t)PIX * 8 * 2};
    const cuuint32_t box[4] = {8, HALO_W, HALO_H, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16 *>(act), dims, strides,
                           box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int CIN_P, int COUT, int EPI>
cudaError_t launch_conv(const ConvArgs &a, cudaStream_t st)
{
    using S = ConvShape<CIN_P, COUT>;
    static int resident = 0;     // CTAs per SM for this instantiation (persistent grid)
    static int sms = 0;
    if (!resident) {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return e;
        if ((int)S::SMEM > optin) return cudaErrorInvalidConfiguration;
        e = cudaFuncSetAttribute(conv3x3_tc_kernel<CIN_P, COUT, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)S::SMEM);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, conv3x3_tc_kernel<CIN_P, COUT, EPI>, CONV_THREADS,
                                                          S::SMEM);
        if (e != cudaSuccess) return e;
        // co-resident CTAs share the SM's 512 TMEM columns
        const int tmem_fit = 512 / (int)S::TMEM_COLS;
        sms = sm_count(dev);
        resident = std::max(1, std::min(nb, tmem_fit));
    }
    CUtensorMap map;
    cudaError_t e = encode_halo_map(&map, a.in, CIN_P, a.nimg);
    if (e != cudaSuccess) return e;
    const int64_t nitems = (int64_t)a.nimg * 2;
    const int64_t cap = (int64_t)sms * resident;
    conv3x3_tc_kernel<CIN_P, COUT, EPI><<<(int)(nitems < cap ? nitems : cap), CONV_THREADS, S::SMEM, st>>>(map, a);
    return cudaGetLastError();
}

cudaError_t conv_forward(int l, const ConvArgs &a, cudaStream_t st)
{
    switch (l) {
    case 0: return launch_conv<16, 32, EPI_BIAS_RELU>(a, st);
    case 1: return launch_conv<32, 32, EPI_BIAS_RELU>(a, st);
    case 2: return launch_conv<32, 64, EPI_BIAS_RELU>(a, st);
    default: return launch_conv<64, 64, EPI_BIAS_RELU>(a, st);
    }
}

// input gradient of layer l (l >= 1): CIN_P' = cout(l), COUT' = cin(l)
cudaError_t conv_dgrad(int l, const ConvArgs &a, cudaStream_t st)
{
    switch (l) {
    case 1: return launch_conv<32, 32, EPI_MASK>(a, st);
    case 2: return launch_conv<64, 32, EPI_MASK>(a, st);
    default: return launch_conv<64, 64, EPI_MASK>(a, st);
    }
}

// Tensor map over BF16 activations [nimg][C/8][32][32][8] seen as 5-D (8 channels, 32 columns,
// C/8 channel groups, 32 rows, nimg), so that a box lands in shared memory row by row:
// [rows][groups][columns][8]. Out-of-range pixels read as zero.
static cudaError_t encode_rows_map(CUtensorMap *map, const __nv_bfloat16 *act, int c, int nimg, int box_w,
                                   int box_groups, int box_h)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[5] = {8, IMG, (cuuint64_t)(c / 8), IMG, (cuuint64_t)nimg};
    const cuuint64_t strides[4] = {8 * 2, (cuuint64_t)PIX * 8 * 2, (cuuint64_t)IMG * 8 * 2,
                                   (cuuint64_t)(c / 8) * PIX * 8 * 2};
    const cuuint32_t box[5] = {8, (cuuint32_t)box_w, (cuuint32_t)box_groups, (cuuint32_t)box_h, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16 *>(act), dims, strides,
                           box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Tensor map over BF16 activations [nimg][C/8][32][32][8] seen as 4-D (a row of 32 pixels x 8 channels,
// C/8 channel groups, 32 rows, nimg): a box of whole rows lands in shared memory as
// [rows][groups][32 pixels][8], with 512-byte rows for the copy engine (no halo needed).
static cudaError_t encode_fullrow_map(CUtensorMap *map, const __nv_bfloat16 *act, int c, int nimg, int box_groups,
                                      int box_h)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[4] = {(cuuint64_t)IMG * 8, (cuuint64_t)(c / 8), IMG, (cuuint64_t)nimg};
    const cuuint64_t strides[3] = {(cuuint64_t)PIX * 8 * 2, (cuuint64_t)IMG * 8 * 2, (cuuint64_t)(c / 8) * PIX * 8 * 2};
    const cuuint32_t box[4] = {(cuuint32_t)IMG * 8, (cuuint32_t)box_groups, (cuuint32_t)box_h, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16 *>(act), dims, strides,
                           box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Weight and bias gradient of one layer: wgrad_tc_kernel, bias partials, and the fixed-order fold
// into gw [cout][cin][3][3] and gb [cout].
template <int COUT, int CIN_P, int CIP>
static cudaError_t launch_wgrad_tc(const __nv_bfloat16 *in, const __nv_bfloat16 *dout, float *part, float *bpart,
                                   int B, int cin, int *err, float *gw, float *gb, cudaStream_t st)
{
    using W = WgtShape<COUT, CIN_P, CIP>;
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        const cudaError_t e = cudaFuncSetAttribute(wgrad_tc_kernel<COUT, CIN_P, CIP>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)W::SMEM);
        if (e != cudaSuccess) return e;
        sms = sm_count(dev);
    }
    CUtensorMap tin, tout;
    cudaError_t e = encode_rows_map(&tin, in, CIN_P, B, HALO_W, CIP / 8, W::ROWS + 2);
    if (e == cudaSuccess) e = encode_fullrow_map(&tout, dout, COUT, B, COUT / 8, W::ROWS);
    if (e != cudaSuccess) return e;
    const int units = W::ITEMS * B * W::P;
    int grid = units < sms ? units : sms;
    grid -= grid % W::P;
    WgtArgs a{part, B, err};
    wgrad_tc_kernel<COUT, CIN_P, CIP><<<grid, CONV_THREADS, W::SMEM, st>>>(tin, tout, a);
    const int nb = B < 128 ? B : 128;
    bias_grad_kernel<COUT><<<nb, 256, 0, st>>>(dout, B, bpart);
    wgrad_tc_reduce_kernel<<<nblk((int64_t)COUT * cin * 9 + COUT), 256, 0, st>>>(part, grid, W::P, W::HM, COUT, CIP,
                                                                                cin, bpart, nb, gw, gb);
    count_launches(3);
    return cudaGetLastError();
}

// Weight and bias gradient of layer l into gw, gb (the layer's slots of the gradient vector).
cudaError_t wgrad(int l, const __nv_bfloat16 *in, const __nv_bfloat16 *dout, float *part, float *bpart, int B,
                  int *err, float *gw, float *gb, cudaStream_t st)
{
    switch (l) {
    case 0: return launch_wgrad_tc<32, 16, 16>(in, dout, part, bpart, B, IN_PLANES, err, gw, gb, st);
    case 1: return launch_wgrad_tc<32, 32, 16>(in, dout, part, bpart, B, 32, err, gw, gb, st);
    case 2: return launch_wgrad_tc<64, 32, 32>(in, dout, part, bpart, B, 32, err, gw, gb, st);
    default: return launch_wgrad_tc<64, 64, 32>(in, dout, part, bpart, B, 64, err, gw, gb, st);
    }
}


// splitmix64 (Steele, Lea, Flood 2014) for the library's own initialisation and shuffles
struct SplitMix {
    uint64_t s;
    uint64_t next()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return (next() >> 11) * (1.0 / 9007199254740992.0); }
    double normal()
    {
        const double u1 = uniform() + 1e-300, u2 = uniform();
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    }
};

}  // namespace sur
}  // namespace lbm

using namespace lbm;
using namespace lbm::sur;

// ------------------------------------------------------------- the ensemble

struct lbm_surrogate {
    int nmodels = 0;
    int dev = 0;
    float *params = nullptr;      // device [nmodels][P] FP32 master
    float *adam_m = nullptr, *adam_v = nullptr;
    int64_t adam_t = 0;
    __nv_bfloat16 *wf[NLAYER] = {};   // packed forward weights (current model)
    __nv_bfloat16 *wb[NLAYER] = {};   // packed input-gradient weights (current model)
    // normalisation: input plane 0 and targets; stats range for the gate
    float in_shift = 0.0f, in_scale = 1.0f;
    float y_mean[2] = {0.0f, 0.0f}, y_std[2] = {1.0f, 1.0f};
    float stat_lo[3] = {-1e30f, -1e30f, -1e30f}, stat_hi[3] = {1e30f, 1e30f, 1e30f};
    int target_mode = 2;          // 0 mean log K, 1 bound midpoint, 2 midpoint and width, 3 Darcy K*
    float gate_spread[7] = {0.03f, 0.03f, 0.03f, 0.03f, 0.03f, 0.03f, 0.03f};   // per log2 leaf size 0..6
    // buffers of lbm_surrogate_keff: one chunk of leaves, the job list and the queue table
    int kcap = 0;
    float *kx = nullptr, *kstats = nullptr, *ky = nullptr;
    float4 *kcw = nullptr;
    int64_t jcap = 0;
    int *jobs = nullptr, *fb = nullptr, *stt = nullptr, *table = nullptr;
    lbm_leaf *ul = nullptr;       // uniform leaves of lbm_upscale
    int64_t ulcap = 0;
    // work buffers sized for `cap` images
    int cap = 0;
    __nv_bfloat16 *act[NLAYER + 1] = {};
    __nv_bfloat16 *dact[2] = {};
    float *pooled = nullptr, *y = nullptr, *t = nullptr, *dpool = nullptr, *grad = nullptr, *loss = nullptr;
    float *part = nullptr, *bpart = nullptr;
    int *idx = nullptr, *err = nullptr;
};

namespace lbm {
namespace sur {

static void free_work(lbm_surrogate *s)
{
    for (auto &p : s->act) { cudaFree(p); p = nullptr; }
    for (auto &p : s->dact) { cudaFree(p); p = nullptr; }
    cudaFree(s->pooled); cudaFree(s->y); cudaFree(s->t); cudaFree(s->dpool); cudaFree(s->grad);
    cudaFree(s->loss); cudaFree(s->part); cudaFree(s->bpart); cudaFree(s->idx);
    s->pooled = s->y = s->t = s->dpool = s->grad = s->loss = s->part = s->bpart = nullptr;
    s->idx = nullptr;
    s->cap = 0;
    cudaGetLastError();
}

static lbm_status ensure_work(lbm_surrogate *s, int B)
{
    if (B <= s->cap) return LBM_OK;
    free_work(s);
    cudaError_t e = cudaSuccess;
    for (int l = 0; l <= NLAYER && e == cudaSuccess; ++l) {
        const int c = l == 0 ? CIN0 : cout_of(l - 1);
        e = cudaMalloc(&s->act[l], sizeof(__nv_bfloat16) * (size_t)B * PIX * c);
    }
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaMalloc(&s->dact[k], sizeof(__nv_bfloat16) * (size_t)B * PIX * 64);
    if (e == cudaSuccess) e = cudaMalloc(&s->pooled, sizeof(float) * (size_t)B * 64);
    if (e == cudaSuccess) e = cudaMalloc(&s->y, sizeof(float) * (size_t)B * 2);
    if (e == cudaSuccess) e = cudaMalloc(&s->t, sizeof(float) * (size_t)B * 2);
    if (e == cudaSuccess) e = cudaMalloc(&s->dpool, sizeof(float) * (size_t)B * 64);
    if (e == cudaSuccess) e = cudaMalloc(&s->grad, sizeof(float) * (size_t)LAYOUT.total);
    if (e == cudaSuccess) e = cudaMalloc(&s->loss, sizeof(float) * 4);
    // weight-gradient partials: one [HM][9][COUT][CIP] block (128 x 9 x 32 floats at most) per CTA
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) == cudaSuccess) sms = sm_count(dev);
    if (e == cudaSuccess) e = cudaMalloc(&s->part, sizeof(float) * (size_t)sms * 128 * 9 * 32);
    if (e == cudaSuccess) e = cudaMalloc(&s->bpart, sizeof(float) * (size_t)B * 64);
    if (e == cudaSuccess) e = cudaMalloc(&s->idx, sizeof(int) * (size_t)B);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_work(s);
        return fail(LBM_ENOMEM, "surrogate work buffers for %d images: %s", B, cudaGetErrorString(e));
    }
    s->cap = B;
    return LBM_OK;
}

// packs model m's weights for the tensor-core convolutions
static cudaError_t pack_model(lbm_surrogate *s, int m, cudaStream_t st)
{
    const float *P = s->params + (int64_t)m * LAYOUT.total;
    for (int l = 0; l < NLAYER; ++l) {
        const int ci = cin_real(l), cp = cin_p(l), co = cout_of(l);
        pack_fwd_kernel<<<nblk((int64_t)co * 9 * cp), 256, 0, st>>>(P + LAYOUT.w[l], ci, cp, co, s->wf[l]);
        if (l >= 1) pack_bwd_kernel<<<nblk((int64_t)ci * 9 * co), 256, 0, st>>>(P + LAYOUT.w[l], ci, co, s->wb[l]);
    }
    count_launches(2 * NLAYER - 1);
    return cudaGetLastError();
}

// forward of model m on act[0] (B images): fills act[1..6], pooled, y (standardised units)
static cudaError_t forward(lbm_surrogate *s, int m, int B, cudaStream_t st)
{
    const float *P = s->params + (int64_t)m * LAYOUT.total;
    for (int l = 0; l < NLAYER; ++l) {
        ConvArgs a{s->act[l], s->wf[l], P + LAYOUT.b[l], nullptr, s->act[l + 1], B, s->err};
        cudaError_t e = conv_forward(l, a, st);
        if (e != cudaSuccess) return e;
    }
    gap_head_kernel<<<B, 256, 0, st>>>(s->act[NLAYER], P + LAYOUT.wh, P + LAYOUT.bh, s->pooled, s->y);
    count_launches(NLAYER + 1);
    return cudaGetLastError();
}

// backward of model m after forward(): gradient of mean((y - t)^2) into s->grad, loss into s->loss[0]
static cudaError_t backward(lbm_surrogate *s, int m, int B, cudaStream_t st)
{
    const float *P = s->params + (int64_t)m * LAYOUT.total;
    float *G = s->grad;
    loss_head_backward_kernel<<<1, 256, 0, st>>>(s->y, s->t, s->pooled, P + LAYOUT.wh, B, s->dpool, G + LAYOUT.wh,
                                                 G + LAYOUT.bh, s->loss);
    gap_backward_kernel<<<nblk((int64_t)B * PIX * 64), 256, 0, st>>>(s->dpool, s->act[NLAYER], B, s->dact[0]);
    count_launches(2);
    int cur = 0;
    for (int l = NLAYER - 1; l >= 0; --l) {
        cudaError_t e = wgrad(l, s->act[l], s->dact[cur], s->part, s->bpart, B, s->err, G + LAYOUT.w[l],
                              G + LAYOUT.b[l], st);
        if (e != cudaSuccess) return e;
        if (l >= 1) {
            // dL/d(act_l) masked by act_l > 0: the masked gradient of layer l-1's output
            ConvArgs a{s->dact[cur], s->wb[l], nullptr, s->act[l], s->dact[1 - cur], B, s->err};
            e = conv_dgrad(l, a, st);
            if (e != cudaSuccess) return e;
            count_launches(1);
            cur = 1 - cur;
        }
    }
    return cudaGetLastError();
}

static lbm_status check_err(lbm_surrogate *s, cudaStream_t st)
{
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, s->err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ECUDA, "surrogate: %s", cudaGetErrorString(e));
    }
    if (h) return fail(LBM_ETIMEOUT, "surrogate: a tensor-core wait gave up (results not valid)");
    return LBM_OK;
}

}  // namespace sur
}  // namespace lbm

#define SUR_CUDA(call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            cudaGetLastError();                                                                \
            return fail(e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s failed: %s", #call, \
                        cudaGetErrorString(e_));                                               \
        }                                                                                      \
    } while (0)

extern "C" {

int64_t lbm_surrogate_param_count(void) { return LAYOUT.total; }

lbm_status lbm_surrogate_create(int32_t n_models, uint64_t seed, lbm_surrogate **out)
{
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_models < 1 || n_models > 16) return fail(LBM_EINVAL, "n_models must be in [1, 16]");
    lbm_surrogate *s = new lbm_surrogate();
    s->nmodels = n_models;
    cudaGetDevice(&s->dev);
    const int64_t P = LAYOUT.total;
    auto bail = [&](lbm_status st) { lbm_surrogate_destroy(s); return st; };
    cudaError_t e = cudaMalloc(&s->params, sizeof(float) * P * n_models);
    if (e == cudaSuccess) e = cudaMalloc(&s->adam_m, sizeof(float) * P * n_models);
    if (e == cudaSuccess) e = cudaMalloc(&s->adam_v, sizeof(float) * P * n_models);
    if (e == cudaSuccess) e = cudaMalloc(&s->err, sizeof(int));
    for (int l = 0; l < NLAYER && e == cudaSuccess; ++l) {
        e = cudaMalloc(&s->wf[l], 2 * (size_t)cout_of(l) * 9 * cin_p(l));
        if (e == cudaSuccess) e = cudaMalloc(&s->wb[l], 2 * (size_t)cin_p(l) * 9 * cout_of(l));
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(LBM_ENOMEM, "surrogate parameters: %s", cudaGetErrorString(e)));
    }
    // He-normal conv weights, zero biases, head ~ N(0, 1/64); splitmix64 per model
    std::vector<float> h((size_t)P);
    for (int m = 0; m < n_models; ++m) {
        SplitMix rng{seed * 0x100000001B3ull + (uint64_t)m * 0x9E3779B97F4A7C15ull + 1};
        std::fill(h.begin(), h.end(), 0.0f);
        for (int l = 0; l < NLAYER; ++l) {
            const double sd = std::sqrt(2.0 / (9.0 * cin_real(l)));
            for (int64_t i = 0; i < (int64_t)cout_of(l) * cin_real(l) * 9; ++i) h[LAYOUT.w[l] + i] = (float)(sd * rng.normal());
        }
        for (int i = 0; i < 128; ++i) h[LAYOUT.wh + i] = (float)(rng.normal() / 8.0);
        e = cudaMemcpy(s->params + (int64_t)m * P, h.data(), sizeof(float) * P, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = cudaMemset(s->adam_m, 0, sizeof(float) * P * n_models);
    if (e == cudaSuccess) e = cudaMemset(s->adam_v, 0, sizeof(float) * P * n_models);
    if (e == cudaSuccess) e = cudaMemset(s->err, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(LBM_ECUDA, "surrogate initialisation: %s", cudaGetErrorString(e)));
    }
    *out = s;
    return LBM_OK;
}

lbm_status lbm_surrogate_destroy(lbm_surrogate *s)
{
    if (!s) return LBM_OK;
    free_work(s);
    cudaFree(s->params); cudaFree(s->adam_m); cudaFree(s->adam_v); cudaFree(s->err);
    cudaFree(s->kx); cudaFree(s->kstats); cudaFree(s->ky); cudaFree(s->kcw);
    cudaFree(s->jobs); cudaFree(s->fb); cudaFree(s->stt); cudaFree(s->table); cudaFree(s->ul);
    for (int l = 0; l < NLAYER; ++l) { cudaFree(s->wf[l]); cudaFree(s->wb[l]); }
    cudaGetLastError();
    delete s;
    return LBM_OK;
}

lbm_status lbm_surrogate_get_params(const lbm_surrogate *s, int32_t model, float *host_out)
{
    if (!s || !host_out || model < 0 || model >= s->nmodels) return fail(LBM_EINVAL, "bad surrogate, model or output");
    SUR_CUDA(cudaMemcpy(host_out, s->params + (int64_t)model * LAYOUT.total, sizeof(float) * LAYOUT.total,
                        cudaMemcpyDeviceToHost));
    return LBM_OK;
}

lbm_status lbm_surrogate_set_params(lbm_surrogate *s, int32_t model, const float *host_in)
{
    if (!s || !host_in || model < 0 || model >= s->nmodels) return fail(LBM_EINVAL, "bad surrogate, model or input");
    SUR_CUDA(cudaMemcpy(s->params + (int64_t)model * LAYOUT.total, host_in, sizeof(float) * LAYOUT.total,
                        cudaMemcpyHostToDevice));
    return LBM_OK;
}

lbm_status lbm_surrogate_set_normalization(lbm_surrogate *s, const float norm[13])
{
    if (!s || !norm) return fail(LBM_EINVAL, "bad surrogate or norm");
    if (!(norm[1] > 0.0f) || !(norm[3] > 0.0f) || !(norm[5] > 0.0f)) return fail(LBM_EINVAL, "scales must be > 0");
    s->in_shift = norm[0]; s->in_scale = norm[1];
    s->y_mean[0] = norm[2]; s->y_std[0] = norm[3]; s->y_mean[1] = norm[4]; s->y_std[1] = norm[5];
    const int mode = (int)norm[12];
    if (!(norm[12] == (float)mode) || mode < 0 || mode > 3) return fail(LBM_EINVAL, "target mode must be 0, 1, 2 or 3");
    for (int k = 0; k < 3; ++k) { s->stat_lo[k] = norm[6 + 2 * k]; s->stat_hi[k] = norm[7 + 2 * k]; }
    s->target_mode = mode;
    return LBM_OK;
}

lbm_status lbm_surrogate_get_normalization(const lbm_surrogate *s, float norm[13])
{
    if (!s || !norm) return fail(LBM_EINVAL, "bad surrogate or norm");
    norm[0] = s->in_shift; norm[1] = s->in_scale;
    norm[2] = s->y_mean[0]; norm[3] = s->y_std[0]; norm[4] = s->y_mean[1]; norm[5] = s->y_std[1];
    for (int k = 0; k < 3; ++k) { norm[6 + 2 * k] = s->stat_lo[k]; norm[7 + 2 * k] = s->stat_hi[k]; }
    norm[12] = (float)s->target_mode;
    return LBM_OK;
}

lbm_status lbm_patches(const float *kappa_dev, int32_t nx, int32_t ny, const lbm_leaf *leaves_dev, int32_t n,
                       float *x_dev, float *stats_dev, void *cuda_stream)
{
    if (nx < 1 || ny < 1 || n < 0) return fail(LBM_EINVAL, "bad sizes");
    if (n == 0) return LBM_OK;
    if (!is_device_ptr(kappa_dev) || !is_device_ptr(leaves_dev) || !is_device_ptr(x_dev) || !is_device_ptr(stats_dev))
        return fail(LBM_EINVAL, "kappa, leaves, x and stats must be device pointers");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    std::vector<lbm_leaf> lv(n);
    SUR_CUDA(cudaMemcpyAsync(lv.data(), leaves_dev, sizeof(lbm_leaf) * n, cudaMemcpyDeviceToHost, st));
    SUR_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < n; ++i) {
        const int s = lv[i].size;
        if (!patch_size_ok(s) || lv[i].x0 < 0 || lv[i].y0 < 0 || (int64_t)lv[i].x0 + s > nx || (int64_t)lv[i].y0 + s > ny)
            return fail(LBM_EINVAL, "leaf %d: size %d must divide 32 or be a multiple of 64 up to 1024, inside the field",
                        i, s);
    }
    patch_kernel<<<n, 256, 0, st>>>(kappa_dev, nx, ny, reinterpret_cast<const int *>(leaves_dev), x_dev, stats_dev,
                                    nullptr);
    SUR_CUDA(cudaGetLastError());
    count_launches(1);
    SUR_CUDA(cudaStreamSynchronize(st));
    return LBM_OK;
}

// One forward + backward of `model` on n inputs (standardised targets t_dev [n][2]);
// gradient of mean((y - t)^2) to grad_host [P], loss to *loss_host; predictions
// (standardised units) to y_host [n][2] if not NULL. For gradient checks.
lbm_status lbm_surrogate_grad(lbm_surrogate *s, int32_t model, const float *x_dev, const float *t_dev, int32_t n,
                              float *grad_host, float *loss_host, float *y_host, void *cuda_stream)
{
    if (!s || model < 0 || model >= s->nmodels || n < 1 || n > 1024) return fail(LBM_EINVAL, "bad arguments");
    if (!is_device_ptr(x_dev) || !is_device_ptr(t_dev)) return fail(LBM_EINVAL, "x and t must be device pointers");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    lbm_status r = ensure_work(s, n);
    if (r != LBM_OK) return r;
    SUR_CUDA(pack_model(s, model, st));
    input_kernel<<<nblk((int64_t)n * PIX), 256, 0, st>>>(x_dev, nullptr, n, s->in_shift, s->in_scale, s->act[0]);
    count_launches(1);
    SUR_CUDA(cudaMemcpyAsync(s->t, t_dev, sizeof(float) * 2 * n, cudaMemcpyDeviceToDevice, st));
    SUR_CUDA(forward(s, model, n, st));
    SUR_CUDA(backward(s, model, n, st));
    r = check_err(s, st);
    if (r != LBM_OK) return r;
    if (grad_host) SUR_CUDA(cudaMemcpy(grad_host, s->grad, sizeof(float) * LAYOUT.total, cudaMemcpyDeviceToHost));
    if (loss_host) SUR_CUDA(cudaMemcpy(loss_host, s->loss, sizeof(float), cudaMemcpyDeviceToHost));
    if (y_host) SUR_CUDA(cudaMemcpy(y_host, s->y, sizeof(float) * 2 * n, cudaMemcpyDeviceToHost));
    return LBM_OK;
}

// Predictions of every model: y_dev [n_models][n][2] = log K*_xx, log K*_yy.
lbm_status lbm_surrogate_predict(lbm_surrogate *s, const float *x_dev, int32_t n, float *y_dev, void *cuda_stream)
{
    if (!s || n < 0) return fail(LBM_EINVAL, "bad arguments");
    if (n == 0) return LBM_OK;
    if (!is_device_ptr(x_dev) || !is_device_ptr(y_dev)) return fail(LBM_EINVAL, "x and y must be device pointers");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int B = n < 2048 ? n : 2048;
    lbm_status r = ensure_work(s, B);
    if (r != LBM_OK) return r;
    for (int m = 0; m < s->nmodels; ++m) {
        SUR_CUDA(pack_model(s, m, st));
        for (int b0 = 0; b0 < n; b0 += B) {
            const int nb = n - b0 < B ? n - b0 : B;
            input_kernel<<<nblk((int64_t)nb * PIX), 256, 0, st>>>(x_dev + (int64_t)b0 * IN_PLANES * PIX, nullptr, nb,
                                                                 s->in_shift, s->in_scale, s->act[0]);
            count_launches(1);
            SUR_CUDA(forward(s, m, nb, st));
            SUR_CUDA(cudaMemcpyAsync(y_dev + ((int64_t)m * n + b0) * 2, s->y, sizeof(float) * 2 * nb,
                                     cudaMemcpyDeviceToDevice, st));
        }
    }
    float4 *d_cw = nullptr;
    SUR_CUDA(cudaMalloc(&d_cw, sizeof(float4) * n));
    cudaError_t eb = launch_base(x_dev, n, s->target_mode, d_cw, st);
    if (eb != cudaSuccess) {
        cudaFree(d_cw);
        cudaGetLastError();
        return fail(LBM_ECUDA, "target base: %s", cudaGetErrorString(eb));
    }
    destandardise_kernel<<<nblk((int64_t)s->nmodels * n * 2), 256, 0, st>>>(y_dev, n, s->nmodels, d_cw, s->y_mean[0],
                                                                          s->y_std[0], s->y_mean[1], s->y_std[1]);
    count_launches(1);
    r = check_err(s, st);
    cudaFree(d_cw);
    return r;
}

// Trains every model of the ensemble on n samples: inputs x_dev [n][9][32][32]
// (lbm_patches), targets y_dev [n][2] = log K*_xx, log K*_yy. The networks learn
// (log K* - c) / w, standardised, with the per-patch base (c, w) of the target
// mode (patch_base_kernel; mode 2 unless set before training). Sets the input and target
// normalisation from the data and the patch-statistics range of the gate from
// stats_dev [n][3] (lbm_patches). Adam (0.9, 0.999, 1e-8), learning rate lr
// with cosine decay to lr / 10, mini-batches of `batch` drawn by a seeded
// shuffle each epoch. loss_host (may be NULL): [n_models][epochs] mean loss.
lbm_status lbm_surrogate_train(lbm_surrogate *s, const float *x_dev, const float *y_dev, const float *stats_dev,
                               int32_t n, int32_t epochs, int32_t batch, double lr, uint64_t seed, float *loss_host,
                               void *cuda_stream)
{
    if (!s || n < 2 || epochs < 1 || batch < 1 || batch > 1024 || !(lr > 0.0)) return fail(LBM_EINVAL, "bad arguments");
    if (!is_device_ptr(x_dev) || !is_device_ptr(y_dev) || !is_device_ptr(stats_dev))
        return fail(LBM_EINVAL, "x, y and stats must be device pointers");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // normalisation from the data (host, once)
    std::vector<float> hy((size_t)2 * n), hs((size_t)3 * n), hx0;
    SUR_CUDA(cudaMemcpy(hy.data(), y_dev, sizeof(float) * 2 * n, cudaMemcpyDeviceToHost));
    SUR_CUDA(cudaMemcpy(hs.data(), stats_dev, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost));
    // targets are learned relative to a per-patch base (c, w) (patch_base_kernel, target_mode)
    std::vector<float> cw((size_t)4 * n);
    {
        float4 *d_cw = nullptr;
        SUR_CUDA(cudaMalloc(&d_cw, sizeof(float4) * n));
        cudaError_t e1 = launch_base(x_dev, n, s->target_mode, d_cw, st);
        if (e1 == cudaSuccess) e1 = cudaMemcpy(cw.data(), d_cw, sizeof(float4) * n, cudaMemcpyDeviceToHost);
        cudaFree(d_cw);
        if (e1 != cudaSuccess) { cudaGetLastError(); return fail(LBM_ECUDA, "patch bases: %s", cudaGetErrorString(e1)); }
    }
    auto resid = [&](int i, int k) {   // (log K* - c) / w
        return ((double)hy[2 * i + k] - cw[4 * i + 2 * k]) / cw[4 * i + 2 * k + 1];
    };
    double my[2] = {0, 0}, sy[2] = {0, 0}, mx = 0, sx = 0;
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 2; ++k) {
            const double rr = resid(i, k);
            my[k] += rr;
            sy[k] += rr * rr;
        }
    for (int k = 0; k < 2; ++k) {
        my[k] /= n;
        sy[k] = std::sqrt(std::max(sy[k] / n - my[k] * my[k], 1e-12));
        s->y_mean[k] = (float)my[k];
        s->y_std[k] = (float)sy[k];
    }
    {   // mean and standard deviation of the log-K planes over every training pixel
        constexpr int NB = 256;
        double *d_part = nullptr;
        SUR_CUDA(cudaMalloc(&d_part, sizeof(double) * 2 * NB));
        input_moments_kernel<<<NB, 256, 0, cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : nullptr>>>(
            x_dev, n, d_part);
        count_launches(1);
        double hp[2 * NB];
        cudaError_t e2 = cudaMemcpy(hp, d_part, sizeof hp, cudaMemcpyDeviceToHost);
        cudaFree(d_part);
        if (e2 != cudaSuccess) { cudaGetLastError(); return fail(LBM_ECUDA, "input moments: %s", cudaGetErrorString(e2)); }
        for (int k = 0; k < NB; ++k) { mx += hp[2 * k]; sx += hp[2 * k + 1]; }
        const double cnt = (double)n * 4 * PIX;     // the four phase planes of every sample
        mx /= cnt;
        sx = std::sqrt(std::max(sx / cnt - mx * mx, 1e-12));
    }
    s->in_shift = (float)mx;
    s->in_scale = (float)sx;
    for (int k = 0; k < 3; ++k) {
        std::vector<float> col(n);
        for (int i = 0; i < n; ++i) col[i] = hs[3 * i + k];
        std::sort(col.begin(), col.end());
        s->stat_lo[k] = col[(size_t)(0.005 * (n - 1))];
        s->stat_hi[k] = col[(size_t)(0.995 * (n - 1))];
    }
    // standardised residual targets
    std::vector<float> ty((size_t)2 * n);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 2; ++k) ty[2 * i + k] = (float)((resid(i, k) - my[k]) / sy[k]);
    float *d_ty = nullptr;
    SUR_CUDA(cudaMalloc(&d_ty, sizeof(float) * 2 * n));
    cudaError_t e = cudaMemcpy(d_ty, ty.data(), sizeof(float) * 2 * n, cudaMemcpyHostToDevice);
    lbm_status r = e == cudaSuccess ? ensure_work(s, batch) : fail(LBM_ECUDA, "target upload failed");
    if (r != LBM_OK) { cudaFree(d_ty); return r; }
    const int steps_per_epoch = n / batch > 0 ? n / batch : 1;
    const int64_t total_steps = (int64_t)steps_per_epoch * epochs;
    std::vector<int> order(n);
    std::vector<float> step_loss(steps_per_epoch);
    int *d_order = nullptr;
    float *d_losses = nullptr;
    e = cudaMalloc(&d_order, sizeof(int) * n);
    if (e == cudaSuccess) e = cudaMalloc(&d_losses, sizeof(float) * steps_per_epoch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_ty); cudaFree(d_order); cudaFree(d_losses);
        return fail(LBM_ENOMEM, "training buffers: %s", cudaGetErrorString(e));
    }
    // every step is enqueued without waiting; the host reads the losses once per epoch
    for (int m = 0; m < s->nmodels && r == LBM_OK; ++m) {
        SplitMix rng{seed * 0x2545F4914F6CDD1Dull + (uint64_t)m + 7};
        int64_t step = 0;
        for (int ep = 0; ep < epochs && r == LBM_OK; ++ep) {
            for (int i = 0; i < n; ++i) order[i] = i;
            for (int i = n - 1; i > 0; --i) std::swap(order[i], order[rng.next() % (uint64_t)(i + 1)]);
            e = cudaMemcpyAsync(d_order, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st);
            for (int sb = 0; sb < steps_per_epoch && e == cudaSuccess; ++sb, ++step) {
                const int B = std::min(batch, n - sb * batch);
                const int *idx = d_order + (int64_t)sb * batch;
                e = pack_model(s, m, st);
                if (e == cudaSuccess) {
                    input_kernel<<<nblk((int64_t)B * PIX), 256, 0, st>>>(x_dev, idx, B, s->in_shift, s->in_scale,
                                                                        s->act[0]);
                    gather_targets_kernel<<<nblk(B), 256, 0, st>>>(d_ty, idx, B, s->t);
                    count_launches(2);
                    e = forward(s, m, B, st);
                }
                if (e == cudaSuccess) e = backward(s, m, B, st);
                if (e == cudaSuccess) {
                    const double frac = total_steps > 1 ? (double)step / (total_steps - 1) : 0.0;
                    const double lr_t = lr * (0.1 + 0.9 * 0.5 * (1.0 + std::cos(3.141592653589793 * frac)));
                    const int64_t t = step + 1;
                    const float c1 = (float)(1.0 - std::pow(0.9, (double)t));
                    const float c2 = (float)(1.0 - std::pow(0.999, (double)t));
                    const int64_t P = LAYOUT.total;
                    adam_kernel<<<nblk(P), 256, 0, st>>>(s->params + m * P, s->grad, s->adam_m + m * P,
                                                         s->adam_v + m * P, P, (float)lr_t, 0.9f, 0.999f, 1e-8f, c1, c2);
                    count_launches(1);
                    e = cudaGetLastError();
                }
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(d_losses + sb, s->loss, sizeof(float), cudaMemcpyDeviceToDevice, st);
            }
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(step_loss.data(), d_losses, sizeof(float) * steps_per_epoch, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) {
                cudaGetLastError();
                r = fail(LBM_ECUDA, "surrogate training: %s", cudaGetErrorString(e));
                break;
            }
            double ep_loss = 0.0;
            for (float l : step_loss) ep_loss += l;
            if (loss_host) loss_host[(int64_t)m * epochs + ep] = (float)(ep_loss / steps_per_epoch);
        }
        if (r == LBM_OK) r = check_err(s, st);
    }
    cudaFree(d_order);
    cudaFree(d_losses);
    cudaFree(d_ty);
    return r;
}

}  // extern "C"

// ------------------------------------------------------------------ the gate

namespace lbm {
namespace sur {

constexpr int KEFF_CHUNK = 32768;        // leaves per pass of patches, inference and gate

// log2 of a leaf size the surrogate path takes (a power of two from 1 to 64), else -1
__host__ __device__ inline int size_class(int s)
{
    for (int c = 0; c <= 6; ++c)
        if (s == (1 << c)) return c;
    return -1;
}

struct GateArgs {
    float lo[3], hi[3];           // accepted range of each patch statistic (bounds included)
    double thr[7];                // ln(1 + spread_max) per log2 leaf size
    int margin;                   // oversampling margin of the fallback local problems
    int smax;                     // largest patch the local solver holds (64 FP32, 45 FP64)
};

// The gate for leaves [base, base + n): the members' mean and sample standard deviation (two
// passes, FP64) of log K*_xx and log K*_yy from y [nmodels][n][2], and the range test of the
// patch statistics. An accepted leaf gets K* = diag(exp(mean xx), exp(mean yy)) and fallback 0;
// a rejected one gets fallback 1 and is counted under its patch size (size + 2 margin) in the
// queue table, for the local solver. A leaf size the path does not take sets DT_BAD.
__global__ void gate_kernel(const float *y, int nmodels, int n, int base, const int *leaves, const float *stats,
                            GateArgs g, double *keff, int *fallback, int *table)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int gi = base + i;
        const int sz = leaves[3 * gi + 2], c = size_class(sz), ps = sz + 2 * g.margin;
        if (c < 0 || ps > g.smax) {
            atomicExch(&table[DT_BAD], 1);
            fallback[gi] = 1;
            continue;
        }
        bool ok = true;
        double m[2];
        for (int k = 0; k < 2; ++k) {
            double a = 0.0;
            for (int j = 0; j < nmodels; ++j) a += (double)y[((int64_t)j * n + i) * 2 + k];
            m[k] = a / nmodels;
            double q = 0.0;
            for (int j = 0; j < nmodels; ++j) {
                const double d = (double)y[((int64_t)j * n + i) * 2 + k] - m[k];
                q += d * d;
            }
            const double sd = nmodels > 1 ? sqrt(q / (nmodels - 1)) : 0.0;
            if (!(sd <= g.thr[c]) || !isfinite(m[k])) ok = false;
        }
        for (int k = 0; k < 3; ++k) {
            const float v = stats[3 * (int64_t)i + k];
            if (!(v >= g.lo[k] && v <= g.hi[k])) ok = false;
        }
        fallback[gi] = ok ? 0 : 1;
        if (ok) {
            keff[4 * (int64_t)gi] = exp(m[0]);
            keff[4 * (int64_t)gi + 1] = 0.0;
            keff[4 * (int64_t)gi + 2] = 0.0;
            keff[4 * (int64_t)gi + 3] = exp(m[1]);
        } else {
            atomicAdd(&table[DT_COUNT + ps], 1);
        }
    }
}

// One thread: the classes of the rejected leaves in descending patch size, the offsets of their
// job ranges and the scatter cursors; nothing if an invalid leaf was seen.
__global__ void queue_table_kernel(int *table)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int nclass = 0, off = 0;
    if (!table[DT_BAD])
        for (int sz = 64; sz >= 1; --sz) {
            const int k = table[DT_COUNT + sz];
            if (k == 0) continue;
            table[DT_SIZE + nclass] = sz;
            table[DT_OFF + nclass] = off;
            table[DT_CURSOR + sz] = off;
            off += 2 * k;
            ++nclass;
        }
    table[DT_OFF + nclass] = off;
    table[DT_NCLASS] = nclass;
    table[DT_NFALLBACK] = off / 2;
}

// Both drives of every rejected leaf into its class's job range (order within a class is free:
// each job's result depends only on its own leaf).
__global__ void queue_scatter_kernel(const int *leaves, int n, const int *fallback, int margin, int smax, int *table,
                                     int *jobs)
{
    if (table[DT_BAD]) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (!fallback[i]) continue;
        const int ps = leaves[3 * i + 2] + 2 * margin;
        const int pos = atomicAdd(&table[DT_CURSOR + ps], 2);
        jobs[pos] = 2 * i;
        jobs[pos + 1] = 2 * i + 1;
    }
}

__global__ void uniform_leaves_kernel(int cx, int cy, int block, int *leaves)
{
    const int64_t n = (int64_t)cx * cy;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        leaves[3 * i] = (int)(i % cx) * block;
        leaves[3 * i + 1] = (int)(i / cx) * block;
        leaves[3 * i + 2] = block;
    }
}

static lbm_status ensure_keff_work(lbm_surrogate *s, int chunk, int64_t n)
{
    cudaError_t e = cudaSuccess;
    if (chunk > s->kcap) {
        cudaFree(s->kx); cudaFree(s->kstats); cudaFree(s->ky); cudaFree(s->kcw);
        s->kx = s->kstats = s->ky = nullptr;
        s->kcw = nullptr;
        s->kcap = 0;
        e = cudaMalloc(&s->kx, sizeof(float) * (size_t)chunk * IN_PLANES * PIX);
        if (e == cudaSuccess) e = cudaMalloc(&s->kstats, sizeof(float) * (size_t)chunk * 3);
        if (e == cudaSuccess) e = cudaMalloc(&s->ky, sizeof(float) * (size_t)chunk * 2 * s->nmodels);
        if (e == cudaSuccess) e = cudaMalloc(&s->kcw, sizeof(float4) * (size_t)chunk);
        if (e == cudaSuccess) s->kcap = chunk;
    }
    if (e == cudaSuccess && n > s->jcap) {
        cudaFree(s->jobs); cudaFree(s->fb); cudaFree(s->stt);
        s->jobs = s->fb = s->stt = nullptr;
        s->jcap = 0;
        e = cudaMalloc(&s->jobs, sizeof(int) * 2 * (size_t)n);
        if (e == cudaSuccess) e = cudaMalloc(&s->fb, sizeof(int) * (size_t)n);
        if (e == cudaSuccess) e = cudaMalloc(&s->stt, sizeof(int) * (size_t)n);
        if (e == cudaSuccess) s->jcap = n;
    }
    if (e == cudaSuccess && !s->table) e = cudaMalloc(&s->table, sizeof(int) * DT_INTS);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ENOMEM, "surrogate K* buffers for %lld leaves: %s", (long long)n, cudaGetErrorString(e));
    }
    return LBM_OK;
}

}  // namespace sur
}  // namespace lbm

extern "C" {

lbm_status lbm_surrogate_set_gate(lbm_surrogate *s, const float spread_by_log2size[7])
{
    if (!s || !spread_by_log2size) return fail(LBM_EINVAL, "bad surrogate or gate");
    for (int c = 0; c < 7; ++c)
        if (!(spread_by_log2size[c] > 0.0f)) return fail(LBM_EINVAL, "gate spreads must be > 0");
    for (int c = 0; c < 7; ++c) s->gate_spread[c] = spread_by_log2size[c];
    return LBM_OK;
}

lbm_status lbm_surrogate_get_gate(const lbm_surrogate *s, float spread_by_log2size[7])
{
    if (!s || !spread_by_log2size) return fail(LBM_EINVAL, "bad surrogate or gate");
    for (int c = 0; c < 7; ++c) spread_by_log2size[c] = s->gate_spread[c];
    return LBM_OK;
}

lbm_status lbm_surrogate_keff(lbm_surrogate *s, const lbm_params *p, const float *kappa_dev,
                              const lbm_leaf *leaves_dev, int32_t n, double spread_max, double g_const,
                              double tol_rel, int64_t max_steps, double *keff_dev, int32_t *fallback_dev,
                              int32_t *status_dev, int32_t *n_fallback, void *cuda_stream)
{
    using namespace lbm::sur;
    if (!s || !p) return fail(LBM_EINVAL, "surrogate or params is NULL");
    if (p->nx < 1 || p->ny < 1) return fail(LBM_EINVAL, "nx, ny must be >= 1");
    if (!std::isfinite(p->tau) || p->tau < 0.5) return fail(LBM_EINVAL, "tau must be finite and >= 0.5");
    if (!std::isfinite(p->nu) || !std::isfinite(p->eps) || p->eps < 0.0)
        return fail(LBM_EINVAL, "nu must be finite and eps finite and >= 0");
    if (p->margin < 0 || p->margin > 32 || p->margin >= p->nx || p->margin >= p->ny)
        return fail(LBM_EINVAL, "margin %d outside [0, 32] or not below the field size", p->margin);
    if (p->warm_start != 0 && p->warm_start != 1) return fail(LBM_EINVAL, "warm_start must be 0 or 1");
    if (n < 0) return fail(LBM_EINVAL, "n must be >= 0");
    if (!(spread_max >= 0.0)) return fail(LBM_EINVAL, "spread_max must be >= 0 (0: the ensemble's per-size gate)");
    if (!std::isfinite(g_const) || g_const == 0.0) return fail(LBM_EINVAL, "g_const must be finite and non-zero");
    if (!std::isfinite(tol_rel) || tol_rel < 0.0) return fail(LBM_EINVAL, "tol_rel must be finite and >= 0");
    if (max_steps < 1 || max_steps >= (int64_t)1 << 31) return fail(LBM_EINVAL, "max_steps must be in [1, 2^31 - 1]");
    if (n == 0) {
        if (n_fallback) *n_fallback = 0;
        return LBM_OK;
    }
    if (!is_device_ptr(kappa_dev) || !is_device_ptr(leaves_dev) || !is_device_ptr(keff_dev) ||
        (fallback_dev && !is_device_ptr(fallback_dev)) || (status_dev && !is_device_ptr(status_dev)))
        return fail(LBM_EINVAL, "kappa, leaves, keff (and fallback, status) must be device pointers");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int chunk = n < KEFF_CHUNK ? n : KEFF_CHUNK;
    lbm_status r = ensure_keff_work(s, chunk, n);
    if (r == LBM_OK) r = ensure_work(s, chunk < 2048 ? chunk : 2048);
    if (r != LBM_OK) return r;
    int *fb = fallback_dev ? fallback_dev : s->fb;
    int *stt = status_dev ? status_dev : s->stt;
    const int *lv = reinterpret_cast<const int *>(leaves_dev);
    GateArgs ga;
    for (int k = 0; k < 3; ++k) { ga.lo[k] = s->stat_lo[k]; ga.hi[k] = s->stat_hi[k]; }
    for (int c = 0; c < 7; ++c) ga.thr[c] = std::log1p(spread_max > 0.0 ? spread_max : (double)s->gate_spread[c]);
    ga.margin = p->margin;
    ga.smax = p->storage == LBM_F64 ? 45 : 64;
    SUR_CUDA(cudaMemsetAsync(s->table, 0, sizeof(int) * DT_INTS, st));
    SUR_CUDA(cudaMemsetAsync(stt, 0, sizeof(int32_t) * n, st));
    SUR_CUDA(cudaMemsetAsync(s->err, 0, sizeof(int), st));
    const int B = chunk < 2048 ? chunk : 2048;
    for (int b0 = 0; b0 < n; b0 += chunk) {
        const int nc = n - b0 < chunk ? n - b0 : chunk;
        patch_kernel<<<nc, 256, 0, st>>>(kappa_dev, p->nx, p->ny, lv + 3 * (int64_t)b0, s->kx, s->kstats,
                                         s->table + DT_BAD);
        count_launches(1);
        for (int m = 0; m < s->nmodels; ++m) {
            SUR_CUDA(pack_model(s, m, st));
            for (int c0 = 0; c0 < nc; c0 += B) {
                const int nb = nc - c0 < B ? nc - c0 : B;
                input_kernel<<<nblk((int64_t)nb * PIX), 256, 0, st>>>(s->kx + (int64_t)c0 * IN_PLANES * PIX, nullptr,
                                                                     nb, s->in_shift, s->in_scale, s->act[0]);
                count_launches(1);
                SUR_CUDA(forward(s, m, nb, st));
                SUR_CUDA(cudaMemcpyAsync(s->ky + ((int64_t)m * nc + c0) * 2, s->y, sizeof(float) * 2 * nb,
                                         cudaMemcpyDeviceToDevice, st));
            }
        }
        SUR_CUDA(launch_base(s->kx, nc, s->target_mode, s->kcw, st));
        destandardise_kernel<<<nblk((int64_t)s->nmodels * nc * 2), 256, 0, st>>>(
            s->ky, nc, s->nmodels, s->kcw, s->y_mean[0], s->y_std[0], s->y_mean[1], s->y_std[1]);
        gate_kernel<<<nblk(nc), 256, 0, st>>>(s->ky, s->nmodels, nc, b0, lv, s->kstats, ga, keff_dev, fb, s->table);
        count_launches(2);
        SUR_CUDA(cudaGetLastError());
    }
    queue_table_kernel<<<1, 32, 0, st>>>(s->table);
    queue_scatter_kernel<<<nblk(n), 256, 0, st>>>(lv, n, fb, p->margin, ga.smax, s->table, s->jobs);
    count_launches(2);
    SUR_CUDA(cudaGetLastError());
    r = launch_local_from_table(p, kappa_dev, leaves_dev, s->jobs, s->table, g_const, tol_rel, max_steps, 64, keff_dev,
                                stt, nullptr, st, local_time_limit());
    if (r != LBM_OK) return r;
    int h[DT_INTS - DT_BAD];
    int herr = 0;
    SUR_CUDA(cudaMemcpyAsync(h, s->table + DT_BAD, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
    SUR_CUDA(cudaMemcpyAsync(&herr, s->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SUR_CUDA(cudaStreamSynchronize(st));
    if (h[0]) return fail(LBM_EINVAL, "a leaf is not a power of two from 1 to %d cells (with margin) inside the field",
                          ga.smax);
    if (herr) return fail(LBM_ETIMEOUT, "surrogate: a tensor-core wait gave up (results not valid)");
    if (n_fallback) *n_fallback = h[DT_NFALLBACK - DT_BAD];
    if (h[DT_ABORT - DT_BAD] || h[DT_WORST - DT_BAD] == LBM_ETIMEOUT)
        return fail(LBM_ETIMEOUT, "local problems exceeded the time limit; unfinished leaves carry LBM_ETIMEOUT");
    if (h[DT_WORST - DT_BAD] == LBM_ENOTCONV)
        return fail(LBM_ENOTCONV, "some fallback leaves did not meet the tolerance within max_steps (status per leaf)");
    return LBM_OK;
}

}  // extern "C"

namespace lbm {

// Upscaling with the ensemble and the LBM fallback (see lbm_upscale in lbm.h): one leaf per block.
lbm_status upscale_with_surrogate(const lbm_params *p, const float *kappa_dev, int32_t block, lbm_surrogate *s,
                                  double spread_max, double g_const, double tol_rel, int64_t max_steps,
                                  double *keff_dev, int32_t *n_fallback, void *cuda_stream)
{
    using namespace sur;
    const int cx = p->nx / block, cy = p->ny / block;
    const int64_t n64 = (int64_t)cx * cy;
    if (n64 > (int64_t)1 << 26) return fail(LBM_EINVAL, "too many blocks for the surrogate path");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (n64 > s->ulcap) {
        cudaFree(s->ul);
        s->ul = nullptr;
        s->ulcap = 0;
        const cudaError_t e = cudaMalloc(&s->ul, sizeof(lbm_leaf) * (size_t)n64);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(LBM_ENOMEM, "block list: %s", cudaGetErrorString(e));
        }
        s->ulcap = n64;
    }
    uniform_leaves_kernel<<<nblk(n64), 256, 0, st>>>(cx, cy, block, reinterpret_cast<int *>(s->ul));
    count_launches(1);
    return lbm_surrogate_keff(s, p, kappa_dev, s->ul, (int32_t)n64, spread_max, g_const, tol_rel, max_steps, keff_dev,
                              nullptr, nullptr, n_fallback, cuda_stream);
}

}  // namespace lbm
