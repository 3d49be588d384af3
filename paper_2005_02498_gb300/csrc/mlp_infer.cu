// mlp_infer.cu -- fused surrogate inference: raw closure inputs -> sym(Lp),
// the whole 30 -> 256 -> 256 -> 256 -> 6 network in one persistent kernel.
//
// One CTA per SM walks 128-row tiles of the input with 18 warps in three roles:
//   * warps 0-15 ("epilogue warps"): per tile they map and standardise the
//     raw features (sigma / 200 MPa, log10(rho + 1e10)) into the FP16
//     layer-1 operand (and its rounding residual, for the trust region), test
//     the box of the trust region, prefetch the features of the tile after
//     next with cp.async, and run the epilogues: accumulator + bias -> GELU
//     -> FP16 activations in shared memory, 64 columns at a time (warp w:
//     TMEM lanes 32 (w mod 4) .. +31, i.e. its rows, and 16 columns), the
//     Mahalanobis test, and the de-standardised FP64 outputs.  The map of
//     tile t + 1 runs right after the layer-3 epilogue of tile t, so the
//     tensor core starts layer 1 of the next tile while the epilogue warps
//     wait for layer 4 of this one;
//   * warp 16, lane 0 ("MMA issuer"): issues every tcgen05 MMA, each
//     weight K-slice as soon as its activation chunk and its weights are in
//     shared memory, and never waits for an MMA to finish;
//   * warp 17, lane 0 ("weight producer"): streams layers 2 and 3 (a bias
//     block, then the weights in K-chunks) through NST shared-memory stages
//     in bulk copies (cp.async.bulk, completion counted on an mbarrier) from
//     a copy pre-tiled into the canonical operand layout, refilling a stage
//     once the MMAs that read it are done (tcgen05.commit on the stage's
//     "empty" barrier).
// Trust region: the distance d2 = |L^-1 z|^2 is a 128 x 32 x 32 product,
// W = Z L^-T, that the tensor core computes next to layer 1 (into 32 spare
// columns of the second accumulator) in split FP16: z = z_hi + z_lo with
// z_hi the layer-1 operand itself, s L^-1 = L_hi + L_lo with s a power of
// two that brings max |L^-1| to [2^13, 2^14), and W = z_hi L_hi + z_hi L_lo +
// z_lo L_hi (the dropped z_lo L_lo term is ~2^-22 relative).  The epilogue
// warps of the first column slice read their row of W once layer 1 is done
// and sum w_i^2 / s^2 in FP32.
// Two TMEM accumulators of 256 columns alternate between the layers (1 -> A,
// 2 -> B, 3 -> A, 4 -> B), and the activations of a layer are handed over in
// 64-column chunks, each with its own mbarrier: while the epilogue warps turn
// chunk c + 1 of layer l's accumulator into activations, the tensor core
// already runs layer l + 1 on chunk c (its K-slice 64 c .. 64 c + 63).  So
// the GELU work of a layer runs beside the next layer's MMAs instead of
// between them.  Per tile: xbar (layer-1 operand ready, 512 arrivals),
// hbar[4] (activation chunk ready, 512 arrivals each; a chunk's barrier
// cannot run two phases ahead of the MMA issuer, because its next phase needs
// the next layer's accumulator, which needs this phase), accbar[4] (layer l's
// MMAs complete, tcgen05.commit; one barrier per layer, because layer 1 of the
// next tile may complete before the epilogue has waited for layer 4 of this
// one), full[NST] / empty[NST] (the weight stages).  Every wait has an
// iteration limit; a wait that gives up raises a CTA-wide abort flag, every
// role leaves its loop, the MMA issuer waits (bounded) for its last MMAs and
// the producer for its last bulk copies, and the kernel frees its tensor
// memory and sets the error flag.
//
// Operands are FP16 (the trained weights are BF16, which FP16 holds exactly
// in its normal range; activations and inputs are rounded to FP16, relative
// step 2^-11), accumulators FP32.  GELU here is 0.5 z (1 + erf(z / sqrt 2))
// with erf(x) ~ tanh(x (A + B x^2)), A = 1.12967582605, B = 0.0997927024 (a
// minimax fit of erf on [0, 6] made for this kernel; |error| <= 2.8e-4), the
// tanh by the hardware f16x2 approximation, and the whole activation in f16x2
// arithmetic: the kernel stores a' = z (1 + tanh(u)) = 2 GELU(z) and takes
// the factor 1/2 into the next layer's weights (W2, W3, W4 are scaled by 1/2
// when they are staged, exactly).  Every hidden layer's bias is already in
// its accumulator, split into two FP16 parts (b_hi = fp16(b), b_lo = fp16(b -
// b_hi)): layer 1's rides in the two padding columns of its K = 32 operand
// (inputs 1 there, W1's columns the bias), layers 2 and 3 start with one
// K = 16 MMA of a constant operand (1 in K columns 0 and 1) against a bias
// block streamed ahead of the layer's weights.  So an activation pair costs
// one conversion, four f16x2 FMA-pipe operations and one special-function
// operation.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "ptadd_internal.cuh"
#include "tc_gemm.cuh"

namespace ptadd {

namespace {

constexpr int EW = 16;             // epilogue warps
constexpr int IT = 32 * EW;        // epilogue threads (rows per tile: 128)
constexpr int IT_ALL = IT + 64;    // + the MMA warp and the weight-producer warp
constexpr int NF = 30, NO = 6;
constexpr int X_BYTES = 128 * 32 * 2;   // layer-1 A operand (FP16), SBO 512
constexpr int W1_BYTES = 256 * 32 * 2;  // SBO 512
constexpr int W4_BYTES = 16 * 256 * 2;  // SBO 4096
constexpr int H_BYTES = 128 * 256 * 2;  // hidden activations, SBO 4096
constexpr int KCH = 64;                 // K per streamed weight chunk
constexpr int NST = 2;                  // weight stages in shared memory
constexpr int CPL = 256 / KCH;          // chunks per layer (W2, W3)
constexpr int WC_BYTES = 256 * KCH * 2; // one K-chunk of W2 or W3, 8-row groups 16 KCH bytes apart
constexpr int BB_BYTES = 256 * 16 * 2;  // a layer's bias block: 256 rows x K 16 (b_hi, b_lo, 0...), SBO 256
constexpr int IPL = CPL + 1;            // stream items per layer: the bias block, then the K-chunks
constexpr int LAYER_BYTES = BB_BYTES + CPL * WC_BYTES;
constexpr int ONES_BYTES = 128 * 16 * 2;  // A operand of the bias MMA: K columns 0, 1 = 1, the rest 0
constexpr int NV_FLOATS = 4 * NF + 2 * NO + NF * NF + 1;
constexpr int LI_BYTES = 32 * 32 * 2;   // L_hi or L_lo: 32 rows (i) x 32 K (j), SBO 512
constexpr int MAHA_COL = 288;           // TMEM columns of W (second accumulator, clear of layer 4's 16)
constexpr int OFF_X = 0;
constexpr int OFF_XLO = OFF_X + X_BYTES;  // z_lo, the same layout
constexpr int OFF_W1 = OFF_XLO + X_BYTES;
constexpr int OFF_LH = OFF_W1 + W1_BYTES;
constexpr int OFF_LL = OFF_LH + LI_BYTES;
constexpr int OFF_W4 = OFF_LL + LI_BYTES;
constexpr int OFF_H = OFF_W4 + W4_BYTES;
constexpr int OFF_WC = OFF_H + H_BYTES;
constexpr int OFF_ONES = OFF_WC + NST * WC_BYTES;
constexpr int OFF_NV = OFF_ONES + ONES_BYTES;
constexpr int OFF_B = OFF_NV + ((NV_FLOATS * 4 + 15) / 16) * 16;   // layer 4's bias (16)
constexpr int OFF_F = OFF_B + 16 * 4;                              // raw features of a tile [128][30]
constexpr int OFF_BOX = OFF_F + 128 * NF * 8;                      // box test per quarter row [2][4][128]
static_assert(OFF_F % 16 == 0, "bulk copies into the staging buffer need 16-byte alignment");
constexpr int INFER_SMEM = OFF_BOX + 2 * 4 * 128;

__device__ __forceinline__ uint32_t canon(int r, int k, int sbo)
{
    return (uint32_t)((r >> 3) * sbo + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Item k (0 <= k < 2 IPL) of the per-tile weight stream: the bias block of
// layer 2, W2's K-chunks, then the same for layer 3; its offset in the staged
// copy and its size.
__device__ __forceinline__ uint32_t item_offset(int k)
{
    const int l = k / IPL, i = k % IPL;
    return (uint32_t)(l * LAYER_BYTES + (i ? BB_BYTES + (i - 1) * WC_BYTES : 0));
}
__device__ __forceinline__ uint32_t item_bytes(int k) { return (k % IPL) ? (uint32_t)WC_BYTES : (uint32_t)BB_BYTES; }

__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint32_t mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
// bytes (a multiple of 16, both addresses 16-byte aligned) from global to shared, completion on mbar
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(mbar)
                 : "memory");
}
// Raw features of one tile (rows r0 .. r0 + valid - 1, 240 valid bytes a row,
// contiguous) into the staging buffer, the same layout: one bulk copy with its
// completion on mbar when the input is 16-byte aligned (issued by one thread),
// else 8-byte asynchronous copies by every epilogue thread.
__device__ __forceinline__ void issue_features(bool bulk, uint32_t dst, const double* feat, int64_t r0, int valid,
                                               uint32_t mbar)
{
    if (bulk) {
        if (threadIdx.x == 0) {
            fence_async_smem();  // the buffer's last reads were generic
            mbar_expect_tx(mbar, (uint32_t)valid * 240u);
            bulk_g2s(dst, feat + r0 * 30, (uint32_t)valid * 240u, mbar);
        }
    } else {
        for (int e = threadIdx.x; e < valid * 30; e += IT) cp_async8(dst + (uint32_t)e * 8, feat + r0 * 30 + e);
        cp_async_commit();
    }
}

// 2 GELU(z) of two values in f16x2 (see the header for the approximation)
__device__ __forceinline__ uint32_t gelu2x2_f16(float2 z)
{
    const __half2 h = __floats2half2_rn(z.x, z.y);
    const __half2 z2 = __hmul2(h, h);
    const __half2 u = __hmul2(h, __hfma2(z2, __float2half2_rn(0.03528185f), __float2half2_rn(0.79880562f)));
    uint32_t t;  // K3 = B / (2 sqrt 2), K1 = A / sqrt 2
    asm("tanh.approx.f16x2 %0, %1;" : "=r"(t) : "r"(*reinterpret_cast<const uint32_t*>(&u)));
    const __half2 g = __hfma2(h, *reinterpret_cast<const __half2*>(&t), h);
    return *reinterpret_cast<const uint32_t*>(&g);
}

// 16 consecutive FP32 columns of this thread's TMEM lane, without waiting:
// the registers hold the values only after the next tmem_wait_ld().
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t r[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Accumulator values (16 columns from c0) [+ bias] -> 2 GELU as 8 f16x2 words.
template <bool BIAS>
__device__ __forceinline__ void gelu16(const uint32_t r[16], int c0, const float* __restrict__ bias, uint32_t w[8])
{
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float2 z = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
        if (BIAS) z = __fadd2_rn(z, *reinterpret_cast<const float2*>(bias + c0 + 2 * i));
        w[i] = gelu2x2_f16(z);
    }
}
// ... into H (row, columns c0 .. c0 + 15)
__device__ __forceinline__ void store16(const uint32_t w[8], int row, int c0, uint8_t* sH)
{
    *reinterpret_cast<uint4*>(sH + canon(row, c0, 4096)) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4*>(sH + canon(row, c0 + 8, 4096)) = make_uint4(w[4], w[5], w[6], w[7]);
}
// Two consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld2(uint32_t taddr, float v[2])
{
    uint32_t r0, r1;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(taddr) : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    v[0] = __uint_as_float(r0);
    v[1] = __uint_as_float(r1);
}

// 8 BF16 values -> 8 FP16 values times a power of two (exact in FP16's normal range)
__device__ __forceinline__ uint4 bf16x8_to_f16x8(uint4 v, float scale)
{
    uint32_t in[4] = {v.x, v.y, v.z, v.w}, out[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&in[i]));
        const __half2 h = __floats2half2_rn(f.x * scale, f.y * scale);
        out[i] = *reinterpret_cast<const uint32_t*>(&h);
    }
    return make_uint4(out[0], out[1], out[2], out[3]);
}

// IEEE-754 round-to-nearest-even FP64 -> FP32 and exact FP32 -> FP64 on the
// integer pipe, for values in the normal FP32 range (others take the
// hardware conversion, which on this GPU runs on the 1/64-rate FP64 pipe).
__device__ __forceinline__ float d2f_rn(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned e = (unsigned)(b >> 52) & 0x7FFu;
    if (e < 1023u - 126u || e > 1023u + 127u) return (float)x;  // zero, FP32-subnormal range, overflow, inf, nan
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    unsigned f = ((unsigned)(b >> 32) & 0x80000000u) | ((e - 896u) << 23) | (unsigned)(m >> 29);
    const unsigned rest = (unsigned)m & 0x1FFFFFFFu;  // the 29 dropped bits
    f += (rest > 0x10000000u || (rest == 0x10000000u && (f & 1u))) ? 1u : 0u;  // carries into the exponent
    return __uint_as_float(f);
}
__device__ __forceinline__ double f2d(float x)
{
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xFFu;
    if (e == 0u || e == 0xFFu) return (double)x;  // zero, subnormal, inf, nan
    const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                                 ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)b);
}

// Bounded wait on an mbarrier phase that also gives up when another role has
// raised the CTA's abort flag: false if the phase did not complete.
__device__ __forceinline__ bool wait_or_abort(uint32_t mbar, uint32_t parity, volatile int* abort_flag)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(mbar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > MBAR_WAIT_LIMIT) return false;
    }
    return true;
}

// epilogue-warp barrier (named barrier 1; the MMA and producer warps do not take part)
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(IT) : "memory"); }

// sigma / 200 MPa, or log10(rho + 1e10), from the FP64 input rounded to FP32
// (all FP32 arithmetic: the FP64 pipe is slow on this part)
__device__ __forceinline__ float raw_feature(double v, bool stress)
{
    const float x = d2f_rn(v);
    return stress ? x * (float)(1.0 / 200e6) : __log10f(x + 1e10f);
}

struct InferArgs {
    const double* feat;  // [n x 30]
    int64_t n;
    int feat_bulk;       // feat is 16-byte aligned: one bulk copy per tile
    const float* nv;     // xm, xs, ym, ys, box lo, box hi, inverse Cholesky factor, d2 threshold
    const __nv_bfloat16* W[4];
    const __half* Wc;    // per layer 2, 3: bias block, then W / 2 (FP16) in CPL pre-tiled K-chunks of 256 x KCH
    const float* b[4];
    double* lp6;         // [n x 6]
    uint8_t* in_region;  // [n] or null
    int* err;
};

__global__ void __launch_bounds__(IT_ALL, 1) mlp_infer_kernel(InferArgs g)
{
    // every region below starts at a multiple of 16 bytes, all the no-swizzle
    // operand layouts need; pointers derived from the array itself keep the
    // compiler's shared-memory address space (plain shared loads and stores)
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t xbar, hbar[4], accbar[4], full[NST], empty[NST], drainbar, fbar;
    __shared__ uint32_t tmem_base;
    __shared__ unsigned li_max;  // bits of max |L^-1| (non-negative floats order as integers)
    __shared__ volatile int abort_flag;
    uint8_t* base = smem_raw;
    uint8_t* sX = base + OFF_X;
    uint8_t* sW1 = base + OFF_W1;
    uint8_t* sW4 = base + OFF_W4;
    uint8_t* sH = base + OFF_H;
    uint8_t* sXlo = base + OFF_XLO;
    float* snv = reinterpret_cast<float*>(base + OFF_NV);
    uint8_t* sBox = base + OFF_BOX;
    const uint32_t uX = smem_u32(sX), uW1 = smem_u32(sW1), uW4 = smem_u32(sW4), uH = smem_u32(sH);
    const uint32_t uXlo = smem_u32(sXlo), uLH = smem_u32(base + OFF_LH), uLL = smem_u32(base + OFF_LL);
    const uint32_t uWC = smem_u32(base + OFF_WC), uOnes = smem_u32(base + OFF_ONES);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t n_tiles = (g.n + 127) / 128;
    if ((int64_t)blockIdx.x >= n_tiles) return;  // whole CTA, before any allocation
    const int64_t my_tiles = (n_tiles - 1 - blockIdx.x) / gridDim.x + 1;
    const int64_t Q = 2 * IPL * my_tiles;  // items of the W2/W3 stream
    const uint32_t ux = smem_u32(&xbar), uacc0 = smem_u32(&accbar[0]);
    const uint32_t uh0 = smem_u32(&hbar[0]), ufull0 = smem_u32(&full[0]), uempty0 = smem_u32(&empty[0]);
    // each mbarrier is 8 bytes: barrier k of an array at u0 + 8 k

    if (warp == 0) {
        tmem_alloc(smem_u32(&tmem_base), 512);
        tmem_relinquish();
    }
    if (tid == 0) {
        abort_flag = 0;
        mbar_init(ux, IT);
        for (int c = 0; c < 4; ++c) mbar_init(uh0 + 8 * c, IT);
        for (int l = 0; l < 4; ++l) mbar_init(uacc0 + 8 * l, 1);
        li_max = 0u;
        mbar_init(smem_u32(&drainbar), 1);
        mbar_init(smem_u32(&fbar), 1);
        for (int k = 0; k < NST; ++k) {
            mbar_init(ufull0 + 8 * k, 1);
            mbar_init(uempty0 + 8 * k, 1);
        }
    }
    // resident operands and maps
    for (int e = tid; e < 256 * 4; e += IT_ALL) {  // W1: 256 rows x 32 K (4 x 8-element groups)
        const int r = e >> 2, kc = e & 3;
        uint4 v = bf16x8_to_f16x8(*reinterpret_cast<const uint4*>(g.W[0] + (int64_t)r * 32 + kc * 8), 1.0f);
        if (kc == 3) {  // K columns 30, 31: the bias in two FP16 parts
            const float bb = g.b[0][r];
            const __half hi = __float2half_rn(bb), lo = __float2half_rn(bb - __half2float(hi));
            const __half2 h2 = __halves2half2(hi, lo);
            v.w = *reinterpret_cast<const uint32_t*>(&h2);
        }
        *reinterpret_cast<uint4*>(sW1 + (r >> 3) * 512 + kc * 128 + (r & 7) * 16) = v;
    }
    for (int e = tid; e < 16 * 32; e += IT_ALL) {  // W4 / 2: 16 rows x 256 K
        const int r = e >> 5, kc = e & 31;
        *reinterpret_cast<uint4*>(sW4 + (r >> 3) * 4096 + kc * 128 + (r & 7) * 16) =
            bf16x8_to_f16x8(*reinterpret_cast<const uint4*>(g.W[3] + (int64_t)r * 256 + kc * 8), 0.5f);
    }
    for (int e = tid; e < NV_FLOATS; e += IT_ALL)  // (the deviations xs are kept as reciprocals)
        snv[e] = (e >= NF && e < 2 * NF) ? 1.0f / g.nv[e] : g.nv[e];
    const float* gLi = g.nv + 4 * NF + 2 * NO;  // L^-1, NF x NF row-major, lower triangle
    __syncthreads();  // li_max is cleared
    for (int e = tid; e < NF * NF; e += IT_ALL) atomicMax(&li_max, __float_as_uint(fabsf(gLi[e])));
    __syncthreads();
    int li_exp = 0;
    frexpf(__uint_as_float(li_max), &li_exp);
    const int li_k = li_max ? max(-60, min(60, 14 - li_exp)) : 0;  // s = 2^li_k
    const float li_s = ldexpf(1.0f, li_k), inv_s2 = ldexpf(1.0f, -2 * li_k);
    for (int e = tid; e < 32 * 32; e += IT_ALL) {  // s L^-1 = L_hi + L_lo, rows i and K columns j, zero-padded
        const int i = e >> 5, j = e & 31;
        const float v = (i < NF && j <= i) ? gLi[i * NF + j] * li_s : 0.0f;
        const __half hi = __float2half_rn(v);
        *reinterpret_cast<__half*>(base + OFF_LH + canon(i, j, 512)) = hi;
        *reinterpret_cast<__half*>(base + OFF_LL + canon(i, j, 512)) = __float2half_rn(v - __half2float(hi));
    }
    float* sB = reinterpret_cast<float*>(base + OFF_B);
    for (int e = tid; e < 16; e += IT_ALL) sB[e] = g.b[3][e];
    for (int e = tid; e < 128 * 16; e += IT_ALL) {  // the ones operand of the bias MMAs
        const int r = e >> 4, k = e & 15;
        *reinterpret_cast<__half*>(base + OFF_ONES + canon(r, k, 256)) = __float2half_rn(k < 2 ? 1.0f : 0.0f);
    }
    const uint32_t uF = smem_u32(base + OFF_F), ufbar = smem_u32(&fbar);
    const double* sF = reinterpret_cast<const double*>(base + OFF_F);
    const bool fbulk = g.feat_bulk != 0;
    fence_async_smem();  // the resident operands were written by the generic proxy
    tc_fence_before();
    __syncthreads();  // (the barrier inits are visible)
    if (tid < IT)
        issue_features(fbulk, uF, g.feat, (int64_t)blockIdx.x * 128,
                       (int)min((int64_t)128, g.n - (int64_t)blockIdx.x * 128), ufbar);
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    bool ok = true;

    if (warp == EW + 1) {
        // ------------------------------------------------ weight producer
        if ((tid & 31) == 0) {
            int64_t issued = 0;
            for (; issued < Q; ++issued) {
                const uint32_t st = (uint32_t)(issued % NST);
                if (issued >= NST &&  // the stage's previous chunk must have been read by its MMAs
                    !wait_or_abort(uempty0 + 8 * st, (uint32_t)(((issued - NST) / NST) & 1), &abort_flag)) {
                    abort_flag = 1;
                    break;
                }
                const int k = (int)(issued % (2 * IPL));
                mbar_expect_tx(ufull0 + 8 * st, item_bytes(k));
                bulk_g2s(uWC + st * WC_BYTES, reinterpret_cast<const uint8_t*>(g.Wc) + item_offset(k), item_bytes(k),
                         ufull0 + 8 * st);
            }
            // no copy may still be landing when the CTA leaves: wait (bounded)
            // for the last copy into each stage
            for (int64_t j = issued > NST ? issued - NST : 0; j < issued; ++j)
                mbar_wait_bounded(ufull0 + 8 * (uint32_t)(j % NST), (uint32_t)((j / NST) & 1), MBAR_WAIT_LIMIT);
            if (abort_flag) atomicExch(g.err, 1);
        }
    } else if (warp == EW) {
        // ------------------------------------------------ MMA issuer
        if ((tid & 31) == 0) {
            const uint32_t id_h = idesc_f16_f32(128, 256), id_o = idesc_f16_f32(128, 16);
            const uint32_t id_m = idesc_f16_f32(128, 32);
            const uint32_t accA = tmem, accB = tmem + 256;
            int64_t q = 0;              // weight chunks consumed
            uint32_t xph = 0, hph = 0;  // hph bit kc: parity of hbar[kc]
            bool mma_out = false;       // MMAs issued (for the abort path)
            for (int64_t it = 0; it < my_tiles && ok; ++it) {
                // layer 1: X [128 x 32] W1^T -> A
                ok = wait_or_abort(ux, xph, &abort_flag);
                xph ^= 1u;
                if (!ok) break;
                tc_fence_after();
                for (int s = 0; s < 2; ++s)
                    tc_mma_f16(accA, smem_desc(uX + s * 256, 128, 512), smem_desc(uW1 + s * 256, 128, 512), id_h,
                               s ? 1u : 0u);
                // trust region: W = z_hi L_hi + z_hi L_lo + z_lo L_hi (kind::f16 with FP16 operands)
                for (int s = 0; s < 2; ++s) {
                    const uint64_t zh = smem_desc(uX + s * 256, 128, 512), zl = smem_desc(uXlo + s * 256, 128, 512);
                    const uint64_t lh = smem_desc(uLH + s * 256, 128, 512), ll = smem_desc(uLL + s * 256, 128, 512);
                    tc_mma_f16(tmem + MAHA_COL, zh, lh, id_m, s ? 1u : 0u);
                    tc_mma_f16(tmem + MAHA_COL, zh, ll, id_m, 1u);
                    tc_mma_f16(tmem + MAHA_COL, zl, lh, id_m, 1u);
                }
                tc_commit(uacc0);
                mma_out = true;
                // layers 2, 3: H [128 x 256] W^T, K-slice by K-slice as soon as the
                // epilogue has written its activation chunk and the weights have landed
                for (int l = 1; l <= 2 && ok; ++l) {
                    const uint32_t acc = (l == 1) ? accB : accA;
                    for (int jj = 0; jj < CPL; ++jj, ++q) {
                        const int kc = jj * KCH / 64;  // the activation chunk this K-slice lies in
                        if ((jj * KCH) % 64 == 0) {
                            ok = wait_or_abort(uh0 + 8 * kc, (hph >> kc) & 1u, &abort_flag);
                            hph ^= 1u << kc;
                            if (!ok) break;
                        }
                        if (jj == 0) {
                            // the bias first: ones [128 x 16] (b_hi, b_lo, 0..)^T sets the
                            // accumulator (only now: the previous layer's epilogue has read it)
                            const uint32_t st = (uint32_t)(q % NST);
                            ok = wait_or_abort(ufull0 + 8 * st, (uint32_t)((q / NST) & 1), &abort_flag);
                            if (!ok) break;
                            tc_fence_after();
                            tc_mma_f16(acc, smem_desc(uOnes, 128, 256), smem_desc(uWC + st * WC_BYTES, 128, 256), id_h,
                                       0u);
                            tc_commit(uempty0 + 8 * st);
                            ++q;
                        }
                        const uint32_t st = (uint32_t)(q % NST);
                        ok = wait_or_abort(ufull0 + 8 * st, (uint32_t)((q / NST) & 1), &abort_flag);
                        if (!ok) break;
                        tc_fence_after();
                        const uint32_t ub = uWC + st * WC_BYTES;
                        for (int s = 0; s < KCH / 16; ++s)
                            tc_mma_f16(acc, smem_desc(uH + (jj * (KCH / 16) + s) * 256, 128, 4096),
                                       smem_desc(ub + s * 256, 128, 16 * KCH), id_h, 1u);
                        tc_commit(uempty0 + 8 * st);  // the stage is free once these MMAs are done
                    }
                    if (!ok) break;
                    tc_commit(uacc0 + 8 * l);
                }
                if (!ok) break;
                // layer 4: H [128 x 256] W4^T -> B (16 columns, 6 used)
                for (int kc = 0; kc < 4 && ok; ++kc) {
                    ok = wait_or_abort(uh0 + 8 * kc, (hph >> kc) & 1u, &abort_flag);
                    hph ^= 1u << kc;
                    if (!ok) break;
                    tc_fence_after();
                    for (int s = 4 * kc; s < 4 * kc + 4; ++s)
                        tc_mma_f16(accB, smem_desc(uH + s * 256, 128, 4096), smem_desc(uW4 + s * 256, 128, 4096),
                                   id_o, s ? 1u : 0u);
                }
                if (!ok) break;
                tc_commit(uacc0 + 24);
            }
            if (!ok) {
                abort_flag = 1;
                // the tensor core may still be busy: wait (bounded) for a commit
                // of everything issued before the tensor memory is freed
                if (mma_out) {
                    tc_commit(smem_u32(&drainbar));
                    mbar_wait_bounded(smem_u32(&drainbar), 0u, MBAR_WAIT_LIMIT);
                }
                atomicExch(g.err, 1);
            }
        }
    } else {
        // ------------------------------------------------ epilogue warps
        const int lg = warp & 3, cs = warp >> 2;  // TMEM lane group (rows) and 16-column slice of a chunk
        const int erow = 32 * lg + (tid & 31);
        const uint32_t tmem_row = tmem + ((uint32_t)(32 * lg) << 16);
        // input-map roles: row and quarter (8 of the 32 operand columns)
        const int mrow = tid & 127, part = tid >> 7;
        const float* xm = snv;
        const float* xr = snv + NF;  // 1 / xs
        const float* ym = snv + 2 * NF;
        const float* ys = ym + NO;
        const float* lo = snv + 2 * NF + 2 * NO;
        const float* hi = lo + NF;
        const float d2_thr = snv[4 * NF + 2 * NO + NF * NF];
        uint32_t accph = 0;  // bit l: parity of accbar[l]
        auto wait_acc = [&](int l) {
            const bool w = wait_or_abort(uacc0 + 8 * l, (accph >> l) & 1u, &abort_flag);
            accph ^= 1u << l;
            if (!w) abort_flag = 1;
            tc_fence_after();
            return w;
        };
        // hand a finished operand chunk to the MMA issuer
        auto publish = [&](uint32_t mbar) {
            fence_async_smem();
            tc_fence_before();
            mbar_arrive(mbar);
        };
        // the input map of tile it: raw features (prefetched into the staging
        // buffer) -> the FP16 layer-1 operand z_hi, its residual z_lo and this
        // quarter row's box test; then the prefetch of tile it + 1
        int fpend = 0;  // tile whose feature copy is in flight, or -1
        auto map_tile = [&](int64_t it) {
            const int64_t r0 = ((int64_t)blockIdx.x + it * gridDim.x) * 128;
            const int valid = (int)min((int64_t)128, g.n - r0);
            if (fbulk) {
                if (!wait_or_abort(ufbar, (uint32_t)(it & 1), &abort_flag)) abort_flag = 1;
                fpend = -1;
                // (on abort the values read below are stale but in bounds; the tile loop ends)
            } else {
                cp_async_wait0();
                epi_sync();
            }
            float zc[8];
            bool box = true;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int k = 8 * part + i;  // warp-uniform: part is
                zc[i] = k >= NF ? 1.0f       // the bias columns
                                : mrow < valid ? (raw_feature(sF[mrow * NF + k], k < 6) - xm[k]) * xr[k] : 0.0f;
                if (k < NF) box = box && zc[i] >= lo[k] && zc[i] <= hi[k];
            }
            uint32_t w4[4], l4[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const __half2 h = __floats2half2_rn(zc[2 * i], zc[2 * i + 1]);
                const float2 hf = __half22float2(h);
                const __half2 r = __floats2half2_rn(zc[2 * i] - hf.x, zc[2 * i + 1] - hf.y);  // 0 for the bias columns
                w4[i] = *reinterpret_cast<const uint32_t*>(&h);
                l4[i] = *reinterpret_cast<const uint32_t*>(&r);
            }
            *reinterpret_cast<uint4*>(sX + canon(mrow, 8 * part, 512)) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
            *reinterpret_cast<uint4*>(sXlo + canon(mrow, 8 * part, 512)) = make_uint4(l4[0], l4[1], l4[2], l4[3]);
            sBox[(it & 1) * 512 + part * 128 + mrow] = box ? 1 : 0;
            publish(ux);
            epi_sync();  // the staging buffer has been read; the box tests are visible
            if (it + 1 < my_tiles) {
                const int64_t rn = ((int64_t)blockIdx.x + (it + 1) * gridDim.x) * 128;
                issue_features(fbulk, uF, g.feat, rn, (int)min((int64_t)128, g.n - rn), ufbar);
                fpend = (int)(it + 1);
            }
        };
        map_tile(0);
        for (int64_t it = 0; it < my_tiles && ok; ++it) {
            if (abort_flag) {
                ok = false;
                break;
            }
            const int64_t r0 = ((int64_t)blockIdx.x + it * gridDim.x) * 128;
            const int valid = (int)min((int64_t)128, g.n - r0);
            // 1. hidden layers: activations chunk by chunk, each handed over at once
            for (int l = 0; l < 3 && ok; ++l) {
                ok = wait_acc(l);
                if (!ok) break;
                if (l == 0 && cs == 0) {
                    // trust region of this row: its row of W lies in columns the
                    // layer-2 MMAs overwrite, so it is read before the first hand-over
                    float wv[32];
                    tmem_ld16(tmem_row + (uint32_t)MAHA_COL, wv);
                    tmem_ld16(tmem_row + (uint32_t)MAHA_COL + 16u, wv + 16);
                    float d2 = 0.0f;
#pragma unroll
                    for (int i = 0; i < NF; ++i) d2 = fmaf(wv[i], wv[i], d2);
                    const uint8_t* bx = sBox + (it & 1) * 512 + erow;  // this tile's half: the next tile's map
                    const bool box = bx[0] & bx[128] & bx[256] & bx[384];  // may already be writing the other
                    if (erow < valid && g.in_region) g.in_region[r0 + erow] = (box && d2 * inv_s2 <= d2_thr) ? 1 : 0;
                }
                const uint32_t acc_col = (l == 1) ? 256u : 0u;
                // the load of chunk kc + 1 runs while chunk kc is turned into activations
                uint32_t ra[16], rb[16];
                tmem_ld16_async(tmem_row + acc_col + (uint32_t)(16 * cs), ra);
                // chunk kc is handed over one step late, after chunk kc + 1's
                // arithmetic, so that its proxy fence finds the stores done
#pragma unroll
                for (int kc = 0; kc < 4; ++kc) {
                    const int c0 = 64 * kc + 16 * cs;
                    tmem_wait_ld();
                    uint32_t* cur = (kc & 1) ? rb : ra;
                    uint32_t* nxt = (kc & 1) ? ra : rb;
                    if (kc < 3) tmem_ld16_async(tmem_row + acc_col + (uint32_t)(c0 + 64), nxt);
                    uint32_t w[8];
                    gelu16<false>(cur, c0, nullptr, w);  // (every layer's bias is in its accumulator)
                    if (kc > 0) publish(uh0 + 8 * (kc - 1));
                    store16(w, erow, c0, sH);
                }
                publish(uh0 + 24);
                // the next tile's input map, while layer 2 finishes: its operand
                // may be published now, because the MMA issuer starts the next
                // tile's layer 1 only after this tile's layer 4, i.e. after
                // every layer-3 chunk (accumulator A) has been read
                if (l == 0 && it + 1 < my_tiles) map_tile(it + 1);
            }
            if (!ok) break;
            // 2. layer 4 -> FP64 outputs (two columns per thread of the first three column slices)
            if (!(ok = wait_acc(3))) break;
            if (cs < 3) {
                float v[2];
                tmem_ld2(tmem_row + 256u + (uint32_t)(2 * cs), v);
                if (erow < valid) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const int o = 2 * cs + c;
                        g.lp6[(r0 + erow) * NO + o] = f2d((v[c] + sB[o]) * ys[o] + ym[o]);
                    }
                }
            }
            tc_fence_before();
        }
        cp_async_wait0();
        // a feature copy still landing (the loop ended early): wait (bounded) for it
        if (fbulk && tid == 0 && fpend >= 0) mbar_wait_bounded(ufbar, (uint32_t)(fpend & 1), MBAR_WAIT_LIMIT);
        if (!ok && (tid & 31) == 0) atomicExch(g.err, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// The staged copy of layers 2 and 3, LAYER_BYTES each: the bias block
// (256 rows x K 16 in the canonical no-swizzle K-major layout, 8-row groups
// 256 B apart: row r holds b_hi = fp16(b_r), b_lo = fp16(b_r - b_hi), then
// zeros), then W / 2 (row-major 256 x 256 BF16 in, FP16 out) in CPL K-chunks
// of 256 rows x KCH in the same layout (K-adjacent core matrices 128 B apart,
// 8-row groups 16 KCH bytes apart), WC_BYTES each; every item is one
// contiguous bulk copy into shared memory.
__global__ void tile_weights_kernel(const __nv_bfloat16* __restrict__ W2, const __nv_bfloat16* __restrict__ W3,
                                    const float* __restrict__ b2, const float* __restrict__ b3,
                                    __half* __restrict__ Wc)
{
    constexpr int G = KCH / 8;  // 16-byte groups per row of a chunk
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    uint8_t* base = reinterpret_cast<uint8_t*>(Wc);
    if (v < 2 * CPL * 256 * G) {  // one 16-byte group of W: chunk j, row r, group kk
        const int j = v / (256 * G), r = (v / G) % 256, kk = v % G;
        const int l = j / CPL;
        const __nv_bfloat16* W = l == 0 ? W2 : W3;
        const int k0 = KCH * (j % CPL) + 8 * kk;
        uint8_t* dst = base + (size_t)l * LAYER_BYTES + BB_BYTES + (size_t)(j % CPL) * WC_BYTES + (r >> 3) * (16 * KCH) +
                       kk * 128 + (r & 7) * 16;
        *reinterpret_cast<uint4*>(dst) = bf16x8_to_f16x8(*reinterpret_cast<const uint4*>(W + r * 256 + k0), 0.5f);
    } else if (v < 2 * CPL * 256 * G + 2 * 256) {  // one row of a bias block
        const int u = v - 2 * CPL * 256 * G, l = u / 256, r = u % 256;
        const float bb = (l == 0 ? b2 : b3)[r];
        const __half hi = __float2half_rn(bb), lo = __float2half_rn(bb - __half2float(hi));
        const __half2 h2 = __halves2half2(hi, lo);
        uint8_t* dst = base + (size_t)l * LAYER_BYTES + (r >> 3) * 256 + (r & 7) * 16;
        *reinterpret_cast<uint4*>(dst) = make_uint4(*reinterpret_cast<const uint32_t*>(&h2), 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(dst + 128) = make_uint4(0u, 0u, 0u, 0u);
    }
}

}  // namespace

cudaError_t launch_mlp_infer(const double* feat, int64_t n, const float* nv, const __nv_bfloat16* const W[4],
                             const float* const b[4], __nv_bfloat16* wc, double* lp6, uint8_t* in_region, int* err,
                             cudaStream_t s)
{
    static bool attr_set[64] = {};  // the attribute is per function and device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        e = cudaFuncSetAttribute(mlp_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, INFER_SMEM);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    if (n <= 0) return cudaSuccess;
    // the staged FP16 weights live in the 2-byte-per-element scratch wc
    __half* wh = reinterpret_cast<__half*>(wc);
    tile_weights_kernel<<<(2 * CPL * 256 * (KCH / 8) + 2 * 256 + 255) / 256, 256, 0, s>>>(W[1], W[2], b[1], b[2], wh);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = (n + 127) / 128;
    InferArgs g{};
    g.feat = feat;
    g.n = n;
    g.feat_bulk = ((uintptr_t)feat & 15u) == 0;
    g.nv = nv;
    for (int l = 0; l < 4; ++l) {
        g.W[l] = W[l];
        g.b[l] = b[l];
    }
    g.Wc = wh;
    g.lp6 = lp6;
    g.in_region = in_region;
    g.err = err;
    mlp_infer_kernel<<<(unsigned)(tiles < sms ? tiles : sms), IT_ALL, INFER_SMEM, s>>>(g);
    return cudaGetLastError();
}

}  // namespace ptadd
