// tc_gemm.cu -- host side of the tcgen05 GEMM (tc_gemm.cuh): launcher and
// the ptadd_gemm_bf16 utility entry point.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <vector>

#include "ptadd_internal.cuh"
#include "tc_gemm.cuh"

namespace ptadd {

__device__ __forceinline__ void gemm_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void gemm_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void gemm_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__global__ void __launch_bounds__(GEMM_THREADS) tc_gemm_kernel(GemmArgs g)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    uint8_t* base = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t ubase = smem_u32(base);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = (int64_t)blockIdx.x * 128;
    const int n0 = blockIdx.y * GEMM_NT;
    const int NT = min(GEMM_NT, g.N - n0);  // a multiple of 16
    const uint32_t mb = smem_u32(&mbar);
    const int nk = (g.K + GEMM_KC - 1) / GEMM_KC;
    auto issue = [&](int k) {
        const uint32_t st = ubase + (uint32_t)(k & 1) * GEMM_STAGE;
        load_chunk_async(st, g.A, g.lda, row0, 128, g.M, k * GEMM_KC, g.K);
        load_chunk_async(st + GEMM_A_BYTES, g.B, g.ldb, n0, NT, g.N, k * GEMM_KC, g.K);
    };

    if (warp == 0) {
        tmem_alloc(smem_u32(&tmem_base), 64);
        tmem_relinquish();
    }
    if (threadIdx.x == 0) mbar_init(mb, 1);
    issue(0);
    gemm_commit();
    if (nk > 1) issue(1);
    gemm_commit();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = idesc_bf16_f32(128, NT);
    uint32_t phase = 0;
    bool ok = true;

    for (int k = 0; k < nk; ++k) {
        gemm_wait1();  // chunk k has landed (the newest group is chunk k + 1)
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0 && !g.withhold_mma) {
            tc_fence_after();
            const uint32_t a0 = ubase + (uint32_t)(k & 1) * GEMM_STAGE, b0 = a0 + GEMM_A_BYTES;
            const int kc = min(GEMM_KC, g.K - k * GEMM_KC);
            for (int s = 0; s < kc / 16; ++s)
                tc_mma_f16(tmem, smem_desc(a0 + s * 256, 128, 1024), smem_desc(b0 + s * 256, 128, 1024), idesc,
                           (k > 0 || s > 0) ? 1u : 0u);
            tc_commit(mb);
        }
        // every thread waits for the MMAs before the chunk's stage is refilled
        if (!mbar_wait_bounded(mb, phase, MBAR_WAIT_LIMIT)) ok = false;
        phase ^= 1u;
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        if (k + 2 < nk) issue(k + 2);
        gemm_commit();
    }
    gemm_wait0();
    tc_fence_after();

    if (ok) {
        const int64_t r = row0 + warp * 32 + lane;
        const bool live = r < g.M;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < NT; c0 += 16) {
            float v[16];
            tmem_ld16(trow + (uint32_t)c0, v);
            if (!live) continue;
            const int c = n0 + c0;  // first global column of this group (a multiple of 16)
            if (g.epi == EPI_STORE || g.epi == EPI_BIAS) {
                float4* o = reinterpret_cast<float4*>(g.out_f32 + r * g.ld_out + c);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    float4 w = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                    if (g.epi == EPI_BIAS) {
                        w.x += g.bias[c + 4 * i];
                        w.y += g.bias[c + 4 * i + 1];
                        w.z += g.bias[c + 4 * i + 2];
                        w.w += g.bias[c + 4 * i + 3];
                    }
                    o[i] = w;
                }
            } else if (g.epi == EPI_STORE_T) {
#pragma unroll
                for (int i = 0; i < 16; ++i) g.out_f32[(int64_t)(c + i) * g.ld_out + r] = v[i];
            } else {
                // EPI_BIAS_GELU: z = C + bias (kept in FP32 if asked), h = GELU(z);
                // EPI_DGELU: h = C * GELU'(zin).  h -> BF16, row-major and/or transposed
                uint32_t hw[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    float h0, h1;
                    if (g.epi == EPI_BIAS_GELU) {
                        const float z0 = v[2 * i] + g.bias[c + 2 * i], z1 = v[2 * i + 1] + g.bias[c + 2 * i + 1];
                        v[2 * i] = z0;
                        v[2 * i + 1] = z1;
                        h0 = gelu_f(z0);
                        h1 = gelu_f(z1);
                    } else {
                        const float2 zi = *reinterpret_cast<const float2*>(g.zin + r * g.ld_z + c + 2 * i);
                        h0 = v[2 * i] * gelu_grad_f(zi.x);
                        h1 = v[2 * i + 1] * gelu_grad_f(zi.y);
                    }
                    const __nv_bfloat162 h = __floats2bfloat162_rn(h0, h1);
                    hw[i] = *reinterpret_cast<const uint32_t*>(&h);
                }
                if (g.epi == EPI_BIAS_GELU && g.out_f32) {
                    float4* o = reinterpret_cast<float4*>(g.out_f32 + r * g.ld_out + c);
#pragma unroll
                    for (int i = 0; i < 4; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                }
                if (g.out_bf16) {
                    uint4* o = reinterpret_cast<uint4*>(g.out_bf16 + r * g.ld_bf16 + c);
                    o[0] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    o[1] = make_uint4(hw[4], hw[5], hw[6], hw[7]);
                }
                if (g.out_bf16_t) {
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&hw[i]);
                        g.out_bf16_t[(int64_t)(c + 2 * i) * g.ld_t + r] = h.x;
                        g.out_bf16_t[(int64_t)(c + 2 * i + 1) * g.ld_t + r] = h.y;
                    }
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
    if (warp == 0) tmem_dealloc(tmem, 64);
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
    const dim3 grid((unsigned)((g.M + 127) / 128), (unsigned)((g.N + GEMM_NT - 1) / GEMM_NT));
    tc_gemm_kernel<<<grid, GEMM_THREADS, GEMM_SMEM, s>>>(g);
    return cudaGetLastError();
}

}  // namespace ptadd

using namespace ptadd;

static ptadd_status gemm_bf16(int device, int64_t M, int32_t N, int32_t K, const uint16_t* A, const uint16_t* B,
                              float* C, int withhold_mma)
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
        g.withhold_mma = withhold_mma;
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

extern "C" ptadd_status ptadd_gemm_bf16(int device, int64_t M, int32_t N, int32_t K, const uint16_t* A,
                                        const uint16_t* B, float* C)
{
    return gemm_bf16(device, M, N, K, A, B, C, 0);
}

extern "C" ptadd_status ptadd_gemm_timeout_selftest(int device)
{
    std::vector<uint16_t> zeros(128 * 64, 0);
    std::vector<float> out(128 * 64, 0.0f);
    return gemm_bf16(device, 128, 64, 64, zeros.data(), zeros.data(), out.data(), 1);
}
