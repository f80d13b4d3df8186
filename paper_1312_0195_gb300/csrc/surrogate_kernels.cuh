// surrogate_kernels.cuh -- kernels of the learned K* surrogate (an addition to
// the paper's method: the paper gets every K* from local LBM, Section 3; here a
// small CNN predicts log K*_xx and log K*_yy from the subdomain's permeability
// patch and local LBM remains the fallback and the arbiter of its error).
//
// Network: six 3x3 'same' convolutions 9(->16 padded) -> 32 -> 32 -> 64 -> 64 ->
// 64 -> 64 with ReLU, global average pooling over the 32 x 32 patch, a linear
// head to 2 outputs. The nine input planes are the leaf's log K on a 64 x 64
// plane split into four 32 x 32 phase planes by row and column parity (so a
// 64-cell leaf enters at full resolution), the constant log2(size) / 6, and
// four context planes: the harmonic and arithmetic means of K along each row
// and along each column of the 32 x 32 patch, in log K, broadcast across it. Activations are BF16 in channel-group planes
// [B][C/8][32][32][8] (act_at below); FP32 master weights; accumulation in FP32.
//
//  * conv3x3_tc_kernel: implicit GEMM on the tensor cores (tcgen05, TMEM, TMA)
//    without an im2col copy. A work item is half an image (16 rows x 32
//    columns = 512 output pixels). TMA loads the item's input with a one-pixel
//    zero halo (18 x 34 pixels) into shared memory, one box per 8-channel
//    plane (rows of 34 x 16 contiguous bytes in global memory), so in shared
//    memory a pixel's 8 channels are 16 contiguous bytes and a row of 8 pixels
//    is one 128-byte core matrix. The A operand of a tap (dy, dx) for
//    an M-tile of 16 rows x 8 columns is then just a descriptor into that
//    halo tile: start at (dy, 8 m + dx), 8-row groups one padded image row
//    (544 B) apart, K groups one plane apart. The 9 taps x CIN/16 K-steps of
//    the 4 M-tiles accumulate into TMEM; the layer's weights stay resident in
//    shared memory. Warp-specialised and double-buffered: warp 0 issues the
//    TMA loads, warp 1 the MMAs, warps 2-5 drain the other TMEM buffer
//    (epilogue: bias + ReLU for the forward pass, ReLU mask for the input
//    gradient, which runs with flipped, transposed weights).
//  * wgrad_tc_kernel: the weight gradient as an implicit GEMM over pixels on the
//    tensor cores (see below), per-CTA partials folded in a fixed order.
#pragma once

#include "sm100_umma.cuh"
#include <cuda.h>
#include <cuda_bf16.h>

namespace lbm {
namespace sur {

constexpr int IMG = 32;                  // patch side
constexpr int PIX = IMG * IMG;           // pixels per patch
constexpr int NLAYER = 6;
constexpr int IN_PLANES = 9;             // four phase planes of log K, the size plane, four context planes
constexpr int CIN0 = 16;                 // padded input planes of layer 0 (9 used)
__host__ __device__ constexpr int cin_p(int l) { return l == 0 ? 16 : (l <= 2 ? 32 : 64); }
__host__ __device__ constexpr int cin_real(int l) { return l == 0 ? IN_PLANES : (l <= 2 ? 32 : 64); }
__host__ __device__ constexpr int cout_of(int l) { return l <= 1 ? 32 : 64; }

enum Epi { EPI_BIAS_RELU = 0, EPI_MASK = 1 };

// Element (image b, pixel p, channel c) of a C-channel activation: channel-group planes
// [B][C/8][32][32][8], so one 8-channel plane of an image is 16 KB contiguous.
__host__ __device__ __forceinline__ int64_t act_at(int64_t b, int p, int c, int C)
{
    return ((b * (C >> 3) + (c >> 3)) * PIX + p) * 8 + (c & 7);
}

struct ConvArgs {
    const __nv_bfloat16 *in;     // [B][CIN_P/8][32][32][8] (read through the tensor map)
    const __nv_bfloat16 *wpack;  // B operand, core-matrix layout, [COUT rows][9 * CIN_P]
    const float *bias;           // [COUT] (EPI_BIAS_RELU)
    const __nv_bfloat16 *mask;   // [B][COUT/8][32][32][8] (EPI_MASK): output *= (mask > 0)
    __nv_bfloat16 *out;          // [B][COUT/8][32][32][8]
    int nimg;
    int *err;                    // set to 1 if a bounded wait gave up
};

constexpr uint32_t WAIT_LIMIT = 1u << 24;   // polls before a wait gives up (~0.1-1 s)

constexpr int HALF_ROWS = IMG / 2;                            // output rows per work item
constexpr int HALO_W = IMG + 2;                               // 34 padded columns
constexpr int HALO_H = HALF_ROWS + 2;                         // 18 padded rows
constexpr uint32_t PLANE_TX = HALO_W * HALO_H * 16;           // 9792 bytes per 8-channel TMA box
constexpr uint32_t PLANE = (PLANE_TX + 127u) / 128u * 128u;   // planes start 128-byte aligned
constexpr uint32_t CTRL = 512;                                // barriers, TMEM address, flag, bias
constexpr int CONV_THREADS = 192;                             // TMA warp, MMA warp, 4 epilogue warps

template <int CIN_P, int COUT>
struct ConvShape {
    static constexpr int NG = CIN_P / 8;                      // 8-channel planes per tile
    static constexpr int K = 9 * CIN_P;
    static constexpr uint32_t B_BYTES = (uint32_t)COUT * K * 2;
    static constexpr uint32_t A_BYTES = NG * PLANE;
    static constexpr uint32_t SMEM = CTRL + B_BYTES + 2 * A_BYTES + 128;   // + runtime alignment
    static constexpr uint32_t TMEM_COLS = 2 * 4 * COUT;       // 2 buffers x 4 M-tiles x COUT columns
    static_assert(B_BYTES % 128 == 0, "weight block keeps the tiles 128-byte aligned");
    static_assert(TMEM_COLS == 256 || TMEM_COLS == 512, "TMEM allocation is a power of two >= 32");
};

template <int CIN_P, int COUT, int EPI>
__global__ void __launch_bounds__(CONV_THREADS, 1)
conv3x3_tc_kernel(const __grid_constant__ CUtensorMap tmap, ConvArgs a)
{
    using S = ConvShape<CIN_P, COUT>;
    constexpr int KSTEPS = CIN_P / 16;
    constexpr uint32_t IDESC = umma::idesc_bf16_f32(128, COUT);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((128u - (umma::smem_addr(smem_raw) & 127u)) & 127u);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);      // [2] input tile landed (TMA bytes)
    uint64_t *empty = full + 2;                               // [2] MMAs finished reading the tile
    uint64_t *tfull = full + 4;                               // [2] accumulators complete
    uint64_t *tempty = full + 6;                              // [2] accumulators drained
    uint32_t *s_taddr = reinterpret_cast<uint32_t *>(smem + 64);
    volatile int *s_fail = reinterpret_cast<volatile int *>(smem + 68);
    float *s_bias = reinterpret_cast<float *>(smem + 128);
    uint8_t *sB = smem + CTRL;
    uint8_t *sA = sB + S::B_BYTES;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nitems = a.nimg * 2;

    // resident weights (already in the core-matrix layout) and bias, loaded once per CTA
    for (uint32_t i = tid; i < S::B_BYTES / 16; i += CONV_THREADS)
        reinterpret_cast<uint4 *>(sB)[i] = reinterpret_cast<const uint4 *>(a.wpack)[i];
    if (EPI == EPI_BIAS_RELU)
        for (int i = tid; i < COUT; i += CONV_THREADS) s_bias[i] = a.bias[i];
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            umma::mbar_init(&full[i], 1);
            umma::mbar_init(&empty[i], 1);
            umma::mbar_init(&tfull[i], 1);
            umma::mbar_init(&tempty[i], 4);
        }
        umma::fence_mbar_init();
        *s_fail = 0;
        umma::prefetch_tmap(&tmap);
    }
    if (warp == 1) umma::tmem_alloc(s_taddr, S::TMEM_COLS);
    umma::fence_proxy_async();                 // weights: generic stores, tensor-core reads
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = *s_taddr;

    if (warp == 0) {
        // ---------------------------------------------------------------- TMA producer
        if (lane == 0) {
            int k = 0;
            for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++k) {
                const int b = k & 1;
                if (k >= 2 && !umma::mbar_wait_bounded(&empty[b], ((k >> 1) - 1) & 1, WAIT_LIMIT)) {
                    *s_fail = 1;
                    break;
                }
                if (*s_fail) break;
                const int img = item >> 1, y0 = (item & 1) * HALF_ROWS;
                uint8_t *dst = sA + b * S::A_BYTES;
                umma::mbar_arrive_expect_tx(&full[b], S::NG * PLANE_TX);
#pragma unroll
                for (int g = 0; g < S::NG; ++g)
                    umma::tma_load_4d(dst + g * PLANE, &tmap, &full[b], 0, -1, y0 - 1, img * S::NG + g);
            }
            if (*s_fail)     // loads already issued land before shared memory is released
                for (int kk = k - 2 < 0 ? 0 : k - 2; kk < k; ++kk)
                    umma::mbar_wait_bounded(&full[kk & 1], (kk >> 1) & 1, WAIT_LIMIT);
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t b_base = umma::smem_addr(sB);
            int k = 0;
            for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++k) {
                const int b = k & 1;
                if (!umma::mbar_wait_bounded(&full[b], (k >> 1) & 1, WAIT_LIMIT) ||
                    (k >= 2 && !umma::mbar_wait_bounded(&tempty[b], ((k >> 1) - 1) & 1, WAIT_LIMIT))) {
                    *s_fail = 1;
                    break;
                }
                if (*s_fail) break;
                umma::fence_after();
                const uint32_t a_base = umma::smem_addr(sA + b * S::A_BYTES);
#pragma unroll 1
                for (int m = 0; m < 4; ++m) {
                    const uint32_t d = tmem + (uint32_t)((b * 4 + m) * COUT);
#pragma unroll
                    for (int tap = 0; tap < 9; ++tap) {
                        const int dy = tap / 3, dx = tap % 3;
#pragma unroll
                        for (int c = 0; c < KSTEPS; ++c) {
                            const uint64_t ad = umma::desc(a_base + 2u * c * PLANE +
                                                               (uint32_t)(dy * HALO_W + 8 * m + dx) * 16u,
                                                           PLANE, HALO_W * 16);
                            const uint64_t bd = umma::desc(b_base + ((tap * CIN_P + c * 16) / 8) * 128, 128,
                                                           (S::K / 8) * 128);
                            umma::mma_bf16(d, ad, bd, IDESC, (tap > 0 || c > 0) ? 1u : 0u);
                        }
                    }
                }
                umma::commit(&empty[b]);
                umma::commit(&tfull[b]);
            }
            // the last commits land before TMEM and shared memory are released
            for (int kk = k - 2 < 0 ? 0 : k - 2; kk < k; ++kk)
                umma::mbar_wait_bounded(&empty[kk & 1], (kk >> 1) & 1, WAIT_LIMIT);
        }
    } else {
        // ---------------------------------------------------------------- epilogue, warps 2-5
        const int q = warp & 3;                 // TMEM lane quarter this warp may read
        int k = 0;
        for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++k) {
            const int b = k & 1;
            const bool ok = umma::mbar_wait_bounded(&tfull[b], (k >> 1) & 1, WAIT_LIMIT);
            if (!__all_sync(0xffffffffu, ok)) {   // tcgen05.ld is warp-collective
                *s_fail = 1;
                break;
            }
            umma::fence_after();
            // TMEM lane 32 q + lane = M row: output row 4 q + lane / 8 of the half, column 8 m + lane % 8
            const int img = item >> 1, y = (item & 1) * HALF_ROWS + 4 * q + (lane >> 3);
#pragma unroll 1
            for (int m = 0; m < 4; ++m) {
                const int pix = y * IMG + 8 * m + (lane & 7);
                uint32_t acc[COUT / 16][16];
#pragma unroll
                for (int c = 0; c < COUT / 16; ++c)
                    umma::tmem_ld16_async(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((b * 4 + m) * COUT + 16 * c),
                                          acc[c]);
                umma::tmem_wait_ld();
#pragma unroll
                for (int c = 0; c < COUT / 16; ++c) umma::tmem_hold(acc[c]);
#pragma unroll
                for (int c0 = 0; c0 < COUT; c0 += 16) {
                    float v[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(acc[c0 / 16][j]);
                    if (EPI == EPI_BIAS_RELU) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j] + s_bias[c0 + j], 0.0f);
                    } else {
                        const uint4 m0 = *reinterpret_cast<const uint4 *>(a.mask + act_at(img, pix, c0, COUT));
                        const uint4 m1 = *reinterpret_cast<const uint4 *>(a.mask + act_at(img, pix, c0 + 8, COUT));
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
                    *reinterpret_cast<uint4 *>(a.out + act_at(img, pix, c0, COUT)) = o[0];
                    *reinterpret_cast<uint4 *>(a.out + act_at(img, pix, c0 + 8, COUT)) = o[1];
                }
            }
            umma::fence_before();
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&tempty[b]);
        }
    }
    umma::fence_before();
    __syncthreads();
    if (tid == 0 && *s_fail) atomicExch(a.err, 1);
    if (warp == 1) {
        umma::fence_after();
        umma::tmem_dealloc(tmem, S::TMEM_COLS);
    }
}

// ------------------------------------------------------------ weight gradient (tcgen05)
//
// dW[tap][co][ci] = sum over the pixels p of every image of dout[p][co] in[p + off(tap)][ci], as an
// implicit GEMM on the tensor cores with K = pixels. Both operands come straight from the
// activation layout (a pixel's 8 channels are 16 contiguous bytes), so they are MN-major: a core
// matrix is 8 consecutive pixels (K) of 8 channels (M or N).
//
// One MMA has M = HM output rows x COUT channels of dout (HM = 128 / COUT) and N = HM + 2
// consecutive padded input rows x CIP input channels, K = 16 pixels of a row. TMA lays both tiles
// out row by row, [row][channel group][pixel][8] (the output gradient in 512-byte pixel rows, the
// input with its zero halo in 16-byte channel groups), so the M and N core-matrix groups are evenly
// spaced across rows: block (h, r) of the product pairs dout row y + h with padded input row y + r,
// which is the vertical tap dy = r - h of output row y + h. Per dx (a 16-byte shift of the B
// start address) one MMA therefore covers all three vertical taps of HM output rows (3 HM of the
// HM (HM + 2) blocks are used: 3/4 for COUT = 64, 1/2 for COUT = 32). The three dx accumulators
// take 3 N <= 384 TMEM columns for the whole run of a CTA.
//
// Work units are (quarter image, input-channel part of CIP channels); a CTA keeps one part and
// takes every (grid / P)-th quarter image. Warp 0 issues the TMA loads (STAGES stages, so that
// several tiles are in flight while the MMAs run), warp 1 the MMAs,
// and warps 2-5 read the accumulators once at the end, writing one partial
// [HM][9][COUT][CIP] per CTA (the rows h of a tap are separate partials), folded in a fixed order
// by wgrad_tc_reduce_kernel.
template <int COUT, int CIN_P, int CIP>
struct WgtShape {
    static constexpr int HM = 128 / COUT;                          // output rows per M tile
    static constexpr int NR = HM + 2;                              // padded input rows per N tile
    static constexpr int N = NR * CIP;
    static constexpr int P = CIN_P / CIP;                          // input-channel parts
    static constexpr int ITEMS = 4;                                // work items per image
    static constexpr int ROWS = IMG / ITEMS;                       // output rows per work item
    static constexpr int STAGES = 4;
    static constexpr uint32_t A_ROW = (COUT / 8) * IMG * 16;       // one dout row, all channel groups
    static constexpr uint32_t A_BYTES = ROWS * A_ROW;
    static constexpr uint32_t B_ROW = (CIP / 8) * HALO_W * 16;     // one padded input row
    static constexpr uint32_t B_BYTES = (ROWS + 2) * B_ROW;
    static constexpr uint32_t B_PAD = (B_BYTES + 127u) / 128u * 128u;
    static constexpr uint32_t STAGE = A_BYTES + B_PAD;
    // at least 116 KB so that only one CTA (and its 512 TMEM columns) fits on an SM
    static constexpr uint32_t NEED = CTRL + STAGES * STAGE + 128;
    static constexpr uint32_t SMEM = NEED > 118784u ? NEED : 118784u;
    static constexpr uint32_t TMEM_COLS = 512;
    static_assert(HM * COUT == 128, "M = 128");
    static_assert(N % 16 == 0 && N <= 256 && 3 * N <= (int)TMEM_COLS, "three accumulators fit TMEM");
    static_assert(CIN_P % CIP == 0 && CIP % 8 == 0, "channel parts of whole groups");
    static_assert(A_BYTES % 128 == 0, "stages stay 128-byte aligned");
    static_assert(ROWS % HM == 0 && NEED <= 232448u, "row tiles per item; shared memory per CTA");
};

struct WgtArgs {
    float *part;                 // [grid][HM][9][COUT][CIP]
    int nimg;
    int *err;                    // set to 1 if a bounded wait gave up
};

template <int COUT, int CIN_P, int CIP>
__global__ void __launch_bounds__(CONV_THREADS, 1)
wgrad_tc_kernel(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout, WgtArgs a)
{
    using S = WgtShape<COUT, CIN_P, CIP>;
    constexpr uint32_t IDESC = umma::idesc_bf16_f32_mn(128, S::N);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((128u - (umma::smem_addr(smem_raw) & 127u)) & 127u);
    constexpr int NS = S::STAGES;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);      // [NS] tiles landed (TMA bytes)
    uint64_t *empty = full + NS;                              // [NS] MMAs finished reading the stage
    uint64_t *tfull = full + 2 * NS;                          // accumulators complete
    uint32_t *s_taddr = reinterpret_cast<uint32_t *>(smem + 8 * (2 * NS + 1));
    volatile int *s_fail = reinterpret_cast<volatile int *>(smem + 8 * (2 * NS + 1) + 4);
    uint8_t *stage0 = smem + CTRL;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int part = blockIdx.x % S::P, cstride = gridDim.x / S::P;
    const int nitems = a.nimg * S::ITEMS;

    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            umma::mbar_init(&full[i], 1);
            umma::mbar_init(&empty[i], 1);
        }
        umma::mbar_init(tfull, 1);
        umma::fence_mbar_init();
        *s_fail = 0;
        umma::prefetch_tmap(&tin);
        umma::prefetch_tmap(&tout);
    }
    if (warp == 1) umma::tmem_alloc(s_taddr, S::TMEM_COLS);
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = *s_taddr;

    if (warp == 0) {
        // ---------------------------------------------------------------- TMA producer
        if (lane == 0) {
            int k = 0;
            for (int item = blockIdx.x / S::P; item < nitems; item += cstride, ++k) {
                const int b = k % NS;
                if (k >= NS && !umma::mbar_wait_bounded(&empty[b], ((k / NS) - 1) & 1, WAIT_LIMIT)) {
                    *s_fail = 1;
                    break;
                }
                if (*s_fail) break;
                const int img = item / S::ITEMS, y0 = (item % S::ITEMS) * S::ROWS;
                uint8_t *st = stage0 + b * S::STAGE;
                umma::mbar_arrive_expect_tx(&full[b], S::A_BYTES + S::B_BYTES);
                umma::tma_load_4d(st, &tout, &full[b], 0, 0, y0, img);
                umma::tma_load_5d(st + S::A_BYTES, &tin, &full[b], 0, -1, part * (CIP / 8), y0 - 1, img);
            }
            if (*s_fail)     // loads already issued land before shared memory is released
                for (int kk = k - NS < 0 ? 0 : k - NS; kk < k; ++kk)
                    umma::mbar_wait_bounded(&full[kk % NS], (kk / NS) & 1, WAIT_LIMIT);
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            int k = 0;
            uint32_t acc = 0;
            for (int item = blockIdx.x / S::P; item < nitems; item += cstride, ++k) {
                const int b = k % NS;
                if (!umma::mbar_wait_bounded(&full[b], (k / NS) & 1, WAIT_LIMIT)) {
                    *s_fail = 1;
                    break;
                }
                if (*s_fail) break;
                umma::fence_after();
                const uint32_t a_base = umma::smem_addr(stage0 + b * S::STAGE);
                const uint32_t b_base = a_base + S::A_BYTES;
#pragma unroll 1
                for (int rt = 0; rt < S::ROWS / S::HM; ++rt) {
#pragma unroll
                    for (int x0 = 0; x0 < IMG; x0 += 16) {
                        const uint64_t ad = umma::desc(a_base + (uint32_t)(rt * S::HM) * S::A_ROW + x0 * 16, 128,
                                                       IMG * 16);
#pragma unroll
                        for (int dx = 0; dx < 3; ++dx) {
                            const uint64_t bd = umma::desc(b_base + (uint32_t)(rt * S::HM) * S::B_ROW + (x0 + dx) * 16,
                                                           128, HALO_W * 16);
                            umma::mma_bf16(tmem + (uint32_t)(dx * S::N), ad, bd, IDESC, acc);
                        }
                        acc = 1u;
                    }
                }
                umma::commit(&empty[b]);
            }
            umma::commit(tfull);
            // the last commits land before TMEM and shared memory are released
            umma::mbar_wait_bounded(tfull, 0, WAIT_LIMIT);
        }
    } else {
        // ---------------------------------------------------------------- epilogue, warps 2-5
        const int q = warp & 3;                   // TMEM lane quarter: lanes 32 q .. 32 q + 31
        const bool ok = umma::mbar_wait_bounded(tfull, 0, WAIT_LIMIT);
        if (!__all_sync(0xffffffffu, ok)) {
            *s_fail = 1;
        } else if (!*s_fail) {
            umma::fence_after();
            const int L = 32 * q + lane, h = L / COUT, co = L % COUT;   // h is the same across a warp
            float *dst = a.part + (int64_t)blockIdx.x * S::HM * 9 * COUT * CIP;
#pragma unroll 1
            for (int dx = 0; dx < 3; ++dx)
#pragma unroll 1
                for (int r = 0; r < S::NR; ++r) {
                    const int dy = r - h;
                    if (dy < 0 || dy > 2) continue;            // warp-uniform
                    float *o = dst + (((int64_t)h * 9 + dy * 3 + dx) * COUT + co) * CIP;
#pragma unroll
                    for (int c0 = 0; c0 < CIP; c0 += 16) {
                        float v[16];
                        umma::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(dx * S::N + r * CIP + c0), v);
#pragma unroll
                        for (int j = 0; j < 16; j += 4)
                            *reinterpret_cast<float4 *>(o + c0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                    }
                }
        }
    }
    umma::fence_before();
    __syncthreads();
    if (tid == 0 && *s_fail) atomicExch(a.err, 1);
    if (warp == 1) {
        umma::fence_after();
        umma::tmem_dealloc(tmem, S::TMEM_COLS);
    }
}

}  // namespace sur
}  // namespace lbm
