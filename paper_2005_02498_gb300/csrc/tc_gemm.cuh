// tc_gemm.cuh -- BF16 x BF16 -> FP32 GEMM tile on the 5th-generation tensor
// cores (tcgen05.mma, accumulator in tensor memory), with fused epilogues for
// the surrogate MLP.
//
//   C[M x N] = A[M x K] * B[N x K]^T     (A and B K-contiguous, "TN")
//
// One CTA of 128 threads owns a 128-row x 64-column tile of C.  K runs in
// chunks of 64 through two shared-memory stages: the chunks are copied with
// cp.async into the canonical no-swizzle K-major layout of the tensor core
// (8-row x 16-byte core matrices; core matrices adjacent in K are 128 B apart
// (leading byte offset), 8-row groups are 1024 B apart (stride byte offset)),
// two chunks ahead of the MMAs that read them.  One elected thread issues
// four 128x64x16 MMAs per chunk into the TMEM accumulator and commits them to
// an mbarrier that every thread waits on (with an iteration limit) before
// the chunk's stage is refilled.  The epilogue reads the accumulator back
// with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = rows of the tile).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ptadd {

// ------------------------------------------------------------------ PTX
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols));
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false if the phase did not complete within `cycles` SM clocks.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity, long long cycles)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(mbar, parity))
        if (clock64() - t0 > cycles) return false;
    return true;
}

// One tcgen05.mma of kind::f16 issued by the calling thread: D (TMEM, FP32)
// (+)= A B^T with A and B both BF16 or both FP16, the type set by the
// instruction descriptor (idesc_bf16_f32 / idesc_f16_f32); accumulate = 0
// overwrites D.
__device__ __forceinline__ void tc_mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void tc_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor, no swizzle, K-major canonical layout.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo_bytes, uint32_t sbo_bytes)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo_bytes >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of this tensor-core generation
    return d;                // base offset 0, swizzle mode 0 (none)
}
// Instruction descriptor: D FP32, A/B BF16, both K-major, M = 128, N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// the same with both operands FP16 (A and B type fields 0)
__host__ __device__ constexpr uint32_t idesc_f16_f32(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---------------------------------------------------------------- GEMM
enum GemmEpi : int {
    EPI_STORE = 0,      // C -> out_f32 (row-major)
    EPI_BIAS = 1,       // C + bias -> out_f32
    EPI_BIAS_GELU = 2,  // z = C + bias -> out_f32 (z), GELU(z) -> out_bf16 (+ transposed)
    EPI_DGELU = 3,      // C * GELU'(zin) -> out_bf16 (+ transposed)
    EPI_STORE_T = 4,    // C -> out_f32 transposed: out[c * ld_out + r]
};

struct GemmArgs {
    const __nv_bfloat16* A;
    int64_t lda;
    const __nv_bfloat16* B;
    int64_t ldb;
    int64_t M;
    int N;  // multiple of 16, <= 256
    int K;  // multiple of 16
    int epi;
    const float* bias;
    float* out_f32;
    int64_t ld_out;
    __nv_bfloat16* out_bf16;
    int64_t ld_bf16;
    __nv_bfloat16* out_bf16_t;  // element (r, c) at [c * ld_t + r]
    int64_t ld_t;
    const float* zin;
    int64_t ld_z;
    int* err;  // set to 1 if an MMA wait gave up
    int withhold_mma;  // self-test of the bounded waits: issue no MMA and no commit
};

constexpr int GEMM_THREADS = 128;
constexpr int GEMM_KC = 64;                          // K per chunk
constexpr int GEMM_NT = 64;                          // output columns per CTA
constexpr int GEMM_A_BYTES = 128 * GEMM_KC * 2;      // 16 KB per stage
constexpr int GEMM_B_BYTES = GEMM_NT * GEMM_KC * 2;  // 8 KB per stage
constexpr int GEMM_STAGE = GEMM_A_BYTES + GEMM_B_BYTES;
constexpr int GEMM_SMEM = 2 * GEMM_STAGE + 1024;     // two stages + alignment slack
constexpr long long MBAR_WAIT_LIMIT = 4000000000LL;  // ~2 s of SM clocks

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// Asynchronous copy of a [rows x 64] K-chunk (columns k0..k0+63 of a
// K-contiguous matrix, rows row0..row0+rows-1) into the canonical layout at
// dst (shared-window address); rows >= row_lim or columns >= K are filled
// with zeros (source size 0).  A warp covers 8 rows x 4 core-matrix columns:
// 64 contiguous bytes per row in global memory, 128 contiguous bytes per 8
// threads in shared memory.  rows is a multiple of 8.
__device__ __forceinline__ void load_chunk_async(uint32_t dst, const __nv_bfloat16* src, int64_t ld, int64_t row0,
                                                 int rows, int64_t row_lim, int k0, int K)
{
    for (int v = threadIdx.x; v < rows * 8; v += GEMM_THREADS) {
        const int r = (v >> 6) * 8 + (v & 7), kk = (v >> 3) & 7;
        const int64_t gr = row0 + r;
        const int gk = k0 + 8 * kk;
        const bool in = gr < row_lim && gk < K;
        const __nv_bfloat16* p = in ? src + gr * ld + gk : src;
        const uint32_t bytes = in ? 16u : 0u;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst + (r >> 3) * 1024 + kk * 128 +
                                                                          (r & 7) * 16),
                     "l"(__cvta_generic_to_global(p)), "r"(bytes)
                     : "memory");
    }
}

// Launch: ceil(M / 128) x ceil(N / GEMM_NT) CTAs of GEMM_THREADS threads,
// GEMM_SMEM bytes of dynamic shared memory (tc_gemm.cu).
cudaError_t launch_tc_gemm(const GemmArgs& g, cudaStream_t s);

// Fused surrogate inference (mlp_infer.cu): raw features [n x 30] -> sym(Lp)
// [n x 6] in FP64 and the trust-region flags; nv = the FP32 maps (xm, xs, ym,
// ys, box, Cholesky factor, threshold), W/b the BF16 weights and FP32 biases,
// wc a device buffer of 8 x 256 x 64 BF16 for the pre-tiled W2/W3 chunks
// (rewritten by every launch).  Two launches: the tiling, the fused kernel.
cudaError_t launch_mlp_infer(const double* feat, int64_t n, const float* nv, const __nv_bfloat16* const W[4],
                             const float* const b[4], __nv_bfloat16* wc, double* lp6, uint8_t* in_region, int* err,
                             cudaStream_t s);

}  // namespace ptadd
