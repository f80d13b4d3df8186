// surrogate_kernels.cuh -- kernels of the learned K* surrogate (an addition to
// the paper's method: the paper gets every K* from local LBM, Section 3; here a
// small CNN predicts log K*_xx and log K*_yy from the subdomain's permeability
// patch and local LBM remains the fallback and the judge of its error).
//
// Network: six 3x3 'same' convolutions 2(->16 padded) -> 32 -> 32 -> 64 -> 64 ->
// 64 -> 64 with ReLU, global average pooling over the 32 x 32 patch, a linear
// head to 2 outputs. Activations are BF16 NHWC [B][32][32][C]; FP32 master
// weights; accumulation in FP32.
//
//  * conv3x3_tc_kernel: implicit GEMM on the tensor cores (tcgen05, TMEM). One
//    CTA = 128 output pixels (4 rows of one image) x all output channels; the
//    9 taps are the 9 K-blocks (K-block = all input channels of one tap). The
//    weights of the layer stay resident in shared memory; the im2col tile of a
//    tap is gathered by all 128 threads into a double buffer while the previous
//    tap's MMAs run. Used for the forward pass (epilogue: bias + ReLU) and for
//    the input gradient (flipped, transposed weights; epilogue: ReLU mask).
//  * wgrad_kernel: weight gradient per (image, tap) on CUDA cores in FP32,
//    written as per-image partials and folded in a fixed order (deterministic).
#pragma once

#include "sm100_umma.cuh"
#include <cuda_bf16.h>

namespace lbm {
namespace sur {

constexpr int IMG = 32;                  // patch side
constexpr int PIX = IMG * IMG;           // pixels per patch
constexpr int NLAYER = 6;
constexpr int CIN0 = 16;                 // padded input planes of layer 0 (2 used)
__host__ __device__ constexpr int cin_p(int l) { return l == 0 ? 16 : (l <= 2 ? 32 : 64); }
__host__ __device__ constexpr int cin_real(int l) { return l == 0 ? 2 : (l <= 2 ? 32 : 64); }
__host__ __device__ constexpr int cout_of(int l) { return l <= 1 ? 32 : 64; }

enum Epi { EPI_BIAS_RELU = 0, EPI_MASK = 1 };

struct ConvArgs {
    const __nv_bfloat16 *in;     // [B][32][32][CIN_P]
    const __nv_bfloat16 *wpack;  // B operand, core-matrix layout, [COUT rows][9 * CIN_P]
    const float *bias;           // [COUT] (EPI_BIAS_RELU)
    const __nv_bfloat16 *mask;   // [B][32][32][COUT] (EPI_MASK): output *= (mask > 0)
    __nv_bfloat16 *out;          // [B][32][32][COUT]
    int nimg;
    int *err;                    // set to 1 if a bounded wait gave up
};

constexpr uint32_t WAIT_LIMIT = 1u << 24;   // polls before a wait gives up (~0.1-1 s)

template <int CIN_P, int COUT>
struct ConvShape {
    static constexpr int K = 9 * CIN_P;
    static constexpr uint32_t B_BYTES = (uint32_t)COUT * K * 2;
    static constexpr uint32_t A_BYTES = 128u * CIN_P * 2;
    static constexpr uint32_t SMEM = B_BYTES + 2 * A_BYTES;
    static constexpr uint32_t TMEM_COLS = COUT < 32 ? 32 : COUT;
};

constexpr int CONV_THREADS = 256;          // 8 warps: all gather; warps w and w+4 share TMEM lanes

template <int CIN_P, int COUT, int EPI>
__global__ void __launch_bounds__(CONV_THREADS) conv3x3_tc_kernel(ConvArgs a)
{
    using S = ConvShape<CIN_P, COUT>;
    constexpr int KB = CIN_P;                       // K-block = one tap, all input channels
    constexpr int KG = KB / 8;                      // core matrices along K per tap
    constexpr uint32_t IDESC = umma::idesc_bf16_f32(128, COUT);
    constexpr int HALF = COUT / 2;                  // TMEM columns read by each warpgroup
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sB = smem;
    uint8_t *sA[2] = {smem + S::B_BYTES, smem + S::B_BYTES + S::A_BYTES};
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t s_taddr;
    __shared__ float s_bias[COUT];
    __shared__ int s_fail;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = a.nimg * 8;                 // tile = 4 rows (128 pixels) of one image

    // resident weights (already in the core-matrix layout) and bias, loaded once per CTA
    for (uint32_t i = tid; i < S::B_BYTES / 16; i += CONV_THREADS)
        reinterpret_cast<uint4 *>(sB)[i] = reinterpret_cast<const uint4 *>(a.wpack)[i];
    if (EPI == EPI_BIAS_RELU)
        for (int i = tid; i < COUT; i += CONV_THREADS) s_bias[i] = a.bias[i];
    if (tid == 0) {
        umma::mbar_init(&mbar[0], 1);
        umma::mbar_init(&mbar[1], 1);
        umma::fence_mbar_init();
        s_fail = 0;
    }
    if (warp == 0) umma::tmem_alloc(&s_taddr, S::TMEM_COLS);
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = s_taddr;

    uint32_t phase[2] = {0u, 0u};
    int issued[2] = {0, 0};                        // commits on each barrier not yet waited for
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int img = tile >> 3, rb = tile & 7;
        for (int kb = 0; kb < 9; ++kb) {
            const int b = kb & 1;
            if (issued[b]) {                       // earlier MMAs read this buffer
                if (!umma::mbar_wait_bounded(&mbar[b], phase[b], WAIT_LIMIT)) s_fail = 1;
                phase[b] ^= 1u;
                issued[b] = 0;
                __syncthreads();
                if (s_fail) break;
            }
            const int dy = kb / 3, dx = kb % 3;
            uint8_t *dst = sA[b];
            // eight consecutive threads fill one 128-byte core matrix (8 pixels x 16 bytes)
            for (int i = tid; i < 128 * KG; i += CONV_THREADS) {
                const int cm = i >> 3, rr = i & 7;
                const int rg = cm / KG, g = cm - rg * KG;
                const int r = rg * 8 + rr;
                const int y = rb * 4 + (r >> 5) + dy - 1, x = (r & 31) + dx - 1;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (y >= 0 && y < IMG && x >= 0 && x < IMG)
                    v = *reinterpret_cast<const uint4 *>(a.in + ((int64_t)(img * IMG + y) * IMG + x) * CIN_P + g * 8);
                *reinterpret_cast<uint4 *>(dst + (uint32_t)rg * (KG * 128) + g * 128 + rr * 16) = v;
            }
            umma::fence_proxy_async();
            __syncthreads();
            if (tid == 0) {
                umma::fence_after();
#pragma unroll
                for (int kk = 0; kk < KB / 16; ++kk) {
                    const uint64_t ad = umma::desc(umma::smem_addr(dst) + kk * 256, 128, KG * 128);
                    const uint64_t bd = umma::desc(umma::smem_addr(sB) + ((kb * KB + kk * 16) / 8) * 128, 128,
                                                   (S::K / 8) * 128);
                    umma::mma_bf16(tmem, ad, bd, IDESC, (kb > 0 || kk > 0) ? 1u : 0u);
                }
                umma::commit(&mbar[b]);
            }
            issued[b] = 1;
        }
        if (s_fail) break;
        // the last commit of the tile (tap 8, buffer 0) covers every MMA issued before it;
        // the decision is made CTA-wide because tcgen05.ld is warp-collective
        const bool waited = umma::mbar_wait_bounded(&mbar[0], phase[0], WAIT_LIMIT);
        phase[0] ^= 1u;
        issued[0] = 0;
        if (!__syncthreads_and(waited ? 1 : 0)) {
            s_fail = 1;
            break;
        }
        umma::fence_after();
        const int wq = warp & 3, half = warp >> 2;    // TMEM lane quarter, column half
        const int y = rb * 4 + wq, x = lane;           // this thread's pixel = TMEM lane 32 wq + lane
        const int64_t pix = (int64_t)(img * IMG + y) * IMG + x;
#pragma unroll
        for (int c0 = half * HALF; c0 < (half + 1) * HALF; c0 += 16) {
            float v[16];
            umma::tmem_ld16(tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)c0, v);
            if (EPI == EPI_BIAS_RELU) {
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j] + s_bias[c0 + j], 0.0f);
            } else {
                const uint4 *mp = reinterpret_cast<const uint4 *>(a.mask + pix * COUT + c0);
                const uint4 m0 = mp[0], m1 = mp[1];
                const __nv_bfloat16 *mb0 = reinterpret_cast<const __nv_bfloat16 *>(&m0);
                const __nv_bfloat16 *mb1 = reinterpret_cast<const __nv_bfloat16 *>(&m1);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (!(__bfloat162float(mb0[j]) > 0.0f)) v[j] = 0.0f;
                    if (!(__bfloat162float(mb1[j]) > 0.0f)) v[8 + j] = 0.0f;
                }
            }
            uint4 o[2];
            __nv_bfloat16 *ob = reinterpret_cast<__nv_bfloat16 *>(o);
#pragma unroll
            for (int j = 0; j < 16; ++j) ob[j] = __float2bfloat16_rn(v[j]);
            uint4 *op = reinterpret_cast<uint4 *>(a.out + pix * COUT + c0);
            op[0] = o[0];
            op[1] = o[1];
        }
        // the next tile's first MMA overwrites the accumulator: every read must be done
        umma::fence_before();
        __syncthreads();
    }
    if (s_fail) {
        if (tid == 0) atomicExch(a.err, 1);
        // give in-flight MMAs a chance to finish before the accumulator is released
        if (issued[0]) umma::mbar_wait_bounded(&mbar[0], phase[0], WAIT_LIMIT);
        if (issued[1]) umma::mbar_wait_bounded(&mbar[1], phase[1], WAIT_LIMIT);
    }
    umma::fence_before();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, S::TMEM_COLS);
}

}  // namespace sur
}  // namespace lbm
