// tc_gemm.cu -- host side of the tcgen05 GEMM (tc_gemm.cuh): launcher and
// the ptadd_gemm_bf16 utility entry point.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "ptadd_internal.cuh"
#include "tc_gemm.cuh"

namespace ptadd {

__global__ void __launch_bounds__(GEMM_THREADS, 1) tc_gemm_kernel(GemmArgs g)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    uint8_t* base = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = base;
    uint8_t* sB = base + GEMM_A_BYTES;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = (int64_t)blockIdx.x * 128;
    const int N = g.N;
    const uint32_t ncols = N <= 32 ? 32u : N <= 64 ? 64u : N <= 128 ? 128u : 256u;
    const uint32_t mb = smem_u32(&mbar);

    if (warp == 0) {
        tmem_alloc(smem_u32(&tmem_base), ncols);
        tmem_relinquish();
    }
    if (threadIdx.x == 0) mbar_init(mb, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = idesc_bf16_f32(128, N);
    uint32_t phase = 0;
    bool ok = true;

    for (int k0 = 0; k0 < g.K; k0 += GEMM_KC) {
        const int kc = min(GEMM_KC, g.K - k0);
        load_chunk(sA, g.A, g.lda, row0, 128, g.M, k0, g.K);
        load_chunk(sB, g.B, g.ldb, 0, N, N, k0, g.K);
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
            for (int s = 0; s < kc / 16; ++s) {
                const uint64_t ad = smem_desc(a0 + s * 256, 128, 1024);
                const uint64_t bd = smem_desc(b0 + s * 256, 128, 1024);
                tc_mma_bf16(tmem, ad, bd, idesc, (k0 > 0 || s > 0) ? 1u : 0u);
            }
            tc_commit(mb);
        }
        // every thread waits for the MMAs before the chunk buffers are reused
        if (!mbar_wait_bounded(mb, phase, MBAR_WAIT_LIMIT)) ok = false;
        phase ^= 1u;
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
    }
    tc_fence_after();

    if (ok) {
        const int64_t r = row0 + warp * 32 + lane;
        const bool live = r < g.M;
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (!live) continue;
            if (g.epi == EPI_STORE || g.epi == EPI_BIAS) {
#pragma unroll
                for (int i = 0; i < 16; ++i) g.out_f32[r * g.ld_out + c0 + i] = v[i] + (g.epi == EPI_BIAS ? g.bias[c0 + i] : 0.f);
            } else if (g.epi == EPI_STORE_T) {
#pragma unroll
                for (int i = 0; i < 16; ++i) g.out_f32[(int64_t)(c0 + i) * g.ld_out + r] = v[i];
            } else if (g.epi == EPI_BIAS_GELU) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float z = v[i] + g.bias[c0 + i];
                    if (g.out_f32) g.out_f32[r * g.ld_out + c0 + i] = z;
                    const __nv_bfloat16 h = __float2bfloat16_rn(gelu_f(z));
                    if (g.out_bf16) g.out_bf16[r * g.ld_bf16 + c0 + i] = h;
                    if (g.out_bf16_t) g.out_bf16_t[(int64_t)(c0 + i) * g.ld_t + r] = h;
                }
            } else {  // EPI_DGELU
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float dz = v[i] * gelu_grad_f(g.zin[r * g.ld_z + c0 + i]);
                    const __nv_bfloat16 h = __float2bfloat16_rn(dz);
                    if (g.out_bf16) g.out_bf16[r * g.ld_bf16 + c0 + i] = h;
                    if (g.out_bf16_t) g.out_bf16_t[(int64_t)(c0 + i) * g.ld_t + r] = h;
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicExch(g.err, 1);
        // give the tensor core a last bounded chance to finish before TMEM is freed
        mbar_wait_bounded(mb, phase ^ 1u, MBAR_WAIT_LIMIT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, ncols);
}


cudaError_t launch_tc_gemm(const GemmArgs& g, cudaStream_t s)
{
    static bool attr_set[64] = {};  // the attribute is per function and device
    int dev = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 != cudaSuccess) return e0;
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    if (g.M <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((g.M + 127) / 128);
    tc_gemm_kernel<<<grid, GEMM_THREADS, GEMM_SMEM, s>>>(g);
    return cudaGetLastError();
}

}  // namespace ptadd

using namespace ptadd;

extern "C" ptadd_status ptadd_gemm_bf16(int device, int64_t M, int32_t N, int32_t K, const uint16_t* A,
                                        const uint16_t* B, float* C)
{
    if (!A || !B || !C) {
        set_error("ptadd_gemm_bf16: null array");
        return PTADD_ERR_ARG;
    }
    if (M < 1 || N < 16 || N > 256 || N % 16 || K < 16 || K % 16 || M > (int64_t)1 << 26) {
        set_error("ptadd_gemm_bf16: need M >= 1, N a multiple of 16 in [16, 256], K a multiple of 16");
        return PTADD_ERR_ARG;
    }
    PTADD_CUDA(cudaSetDevice(device));
    __nv_bfloat16 *dA = nullptr, *dB = nullptr;
    float* dC = nullptr;
    int* derr = nullptr;
    cudaStream_t s = nullptr;
    ptadd_status st = PTADD_OK;
    auto fail = [&](cudaError_t e, const char* what) {
        set_error("ptadd_gemm_bf16: %s: %s", what, cudaGetErrorString(e));
        st = PTADD_ERR_CUDA;
    };
    cudaError_t e = cudaMalloc(&dA, (size_t)M * K * 2);
    if (e == cudaSuccess) e = cudaMalloc(&dB, (size_t)N * K * 2);
    if (e == cudaSuccess) e = cudaMalloc(&dC, (size_t)M * N * 4);
    if (e == cudaSuccess) e = cudaMalloc(&derr, sizeof(int));
    if (e != cudaSuccess) {
        set_error("ptadd_gemm_bf16: cudaMalloc failed: %s", cudaGetErrorString(e));
        st = PTADD_ERR_NOMEM;
    }
    if (st == PTADD_OK) {
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dA, A, (size_t)M * K * 2, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dB, B, (size_t)N * K * 2, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(int), s);
        if (e != cudaSuccess) fail(e, "copy in");
    }
    if (st == PTADD_OK) {
        GemmArgs g{};
        g.A = dA;
        g.lda = K;
        g.B = dB;
        g.ldb = K;
        g.M = M;
        g.N = N;
        g.K = K;
        g.epi = EPI_STORE;
        g.out_f32 = dC;
        g.ld_out = N;
        g.err = derr;
        e = launch_tc_gemm(g, s);
        if (e != cudaSuccess) fail(e, "launch");
    }
    int herr = 0;
    if (st == PTADD_OK) {
        e = cudaMemcpyAsync(C, dC, (size_t)M * N * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) fail(e, "run");
    }
    if (st == PTADD_OK && herr) {
        set_error("ptadd_gemm_bf16: a tensor-core wait gave up");
        st = PTADD_ERR_TIMEOUT;
    }
    if (s) cudaStreamDestroy(s);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dC);
    cudaFree(derr);
    return st;
}
