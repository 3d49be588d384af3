// tc_gemm.cu -- host side of the tcgen05 GEMM (tc_gemm.cuh): launcher and
// the ptadd_gemm_bf16 utility entry point.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "ptadd_internal.cuh"
#include "tc_gemm.cuh"

namespace ptadd {

cudaError_t launch_tc_gemm(const GemmArgs& g, cudaStream_t s)
{
    static bool attr_set = false;  // per process; the attribute is per function
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
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
