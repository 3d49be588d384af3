// mlp.cu -- the surrogate closure: a multilayer perceptron
//   30 -> 256 -> 256 -> 256 -> 6, GELU on the hidden layers,
// BF16 weights and activations, FP32 accumulation on the tensor cores
// (tc_gemm.cuh), FP32 master weights and Adam moments.
//
// Every layer is one tcgen05 GEMM "C = A B^T" with both operands K-contiguous:
//   forward   Z_l = H_{l-1} W_l^T + b_l        (A = H_{l-1} [B x din], B = W_l [dout x din])
//   dH        dH_{l-1} = dZ_l W_l              (A = dZ_l [B x dout], B = W_l^T [din x dout])
//   dW        dW_l = dZ_l^T H_{l-1}            (A = dZ_l^T [dout x B], B = H_{l-1}^T [din x B])
// so the epilogues also write transposed BF16 copies of H and dZ, and Adam
// keeps W and W^T in BF16 next to the FP32 master.  Padding: the 30 inputs
// sit in 32 columns, the 6 outputs in 16 rows of the last layer; padded
// weights stay exactly zero (their gradients are zero).
//
// The closure-level calls (ptadd_surrogate_*) add the input map
//   x = [sigma / 200 MPa (6), log10(rho_m + 1e10) (12), log10(rho_s + 1e10) (12)],
// standardisation of x and of the 6 outputs (sym(Lp) in Voigt order) by the
// training-set mean and standard deviation, and the trust region: inside the
// per-feature [min, max] box of the training inputs AND within the 99th
// percentile of the training inputs' Mahalanobis distance.  (Shrinking the box
// by 5 % per feature would keep only 0.9^30 = 4 % of in-distribution points
// with 30 independent features.)
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "ptadd_internal.cuh"
#include "tc_gemm.cuh"

namespace ptadd {

constexpr int NIN = 30, NOUT = 6, NH = 256;
constexpr int DIN_P[4] = {32, 256, 256, 256};
constexpr int DOUT_P[4] = {256, 256, 256, 16};
constexpr int DIN_U[4] = {30, 256, 256, 256};
constexpr int DOUT_U[4] = {256, 256, 256, 6};
constexpr double RHO_FLOOR = 1e10;
constexpr double SIG_SCALE = 200e6;

struct MlpDev {
    bool ready = false;
    int64_t cap = 0;  // row capacity of the work buffers (multiple of 128)
    float *W[4] = {}, *b[4] = {}, *mW[4] = {}, *vW[4] = {}, *mb[4] = {}, *vb[4] = {}, *gW[4] = {}, *gb[4] = {};
    __nv_bfloat16 *Wb[4] = {}, *Wt[4] = {};
    __nv_bfloat16* Wc = nullptr;  // layers 2, 3 staged for the fused inference kernel (bias block + 4 x 256 x 64 each)
    __nv_bfloat16 *X = nullptr, *Xt = nullptr, *Hb[3] = {}, *Ht[3] = {}, *dY = nullptr, *dYt = nullptr;
    __nv_bfloat16 *dZ[3] = {}, *dZt[3] = {};
    float *Z[3] = {}, *Y = nullptr, *T = nullptr, *loss_part = nullptr;
    int* err = nullptr;
    int64_t step = 0;
    // closure-level maps (host)
    bool have_norm = false;
    double xm[NIN], xs[NIN], ym[NOUT], ys[NOUT];
    double box_lo[NIN], box_hi[NIN];
    double chol[NIN * NIN];  // lower Cholesky factor of the training covariance (standardised x)
    double d2_thr = 0.0;
    float* d_norm = nullptr;  // device copy (FP32): xm, xs, ym, ys, box_lo, box_hi, chol^-1, d2_thr
};

namespace {

template <typename T>
ptadd_status m_alloc(T** p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
        *p = nullptr;
        return PTADD_ERR_NOMEM;
    }
    return PTADD_OK;
}

void free_work(MlpDev& m)
{
    void* ptrs[] = {m.X, m.Xt, m.dY, m.dYt, m.Y, m.T, m.loss_part};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int l = 0; l < 3; ++l) {
        cudaFree(m.Hb[l]);
        cudaFree(m.Ht[l]);
        cudaFree(m.dZ[l]);
        cudaFree(m.dZt[l]);
        cudaFree(m.Z[l]);
        m.Hb[l] = m.Ht[l] = m.dZ[l] = m.dZt[l] = nullptr;
        m.Z[l] = nullptr;
    }
    m.X = m.Xt = m.dY = m.dYt = nullptr;
    m.Y = m.T = m.loss_part = nullptr;
    m.cap = 0;
}

void free_mlp(MlpDev& m)
{
    free_work(m);
    for (int l = 0; l < 4; ++l) {
        void* ptrs[] = {m.W[l], m.b[l], m.mW[l], m.vW[l], m.mb[l], m.vb[l], m.gW[l], m.gb[l], m.Wb[l], m.Wt[l]};
        for (void* p : ptrs)
            if (p) cudaFree(p);
    }
    if (m.err) cudaFree(m.err);
    if (m.d_norm) cudaFree(m.d_norm);
    if (m.Wc) cudaFree(m.Wc);
    m = MlpDev{};
}

ptadd_status alloc_params(MlpDev& m)
{
    ptadd_status st = PTADD_OK;
    for (int l = 0; l < 4 && st == PTADD_OK; ++l) {
        const size_t nw = (size_t)DOUT_P[l] * DIN_P[l], nb = DOUT_P[l];
        float** f[] = {&m.W[l], &m.mW[l], &m.vW[l], &m.gW[l]};
        for (float** p : f)
            if (st == PTADD_OK) st = m_alloc(p, nw);
        float** g[] = {&m.b[l], &m.mb[l], &m.vb[l], &m.gb[l]};
        for (float** p : g)
            if (st == PTADD_OK) st = m_alloc(p, nb);
        if (st == PTADD_OK) st = m_alloc(&m.Wb[l], nw);
        if (st == PTADD_OK) st = m_alloc(&m.Wt[l], nw);
    }
    if (st == PTADD_OK) st = m_alloc(&m.err, 1);
    if (st == PTADD_OK) st = m_alloc(&m.Wc, (size_t)2 * (256 * 16 + 4 * 256 * 64));
    if (st == PTADD_OK) st = m_alloc(&m.d_norm, 4 * NIN + 2 * NOUT + NIN * NIN + 1);
    return st;
}

ptadd_status ensure_work(MlpDev& m, int64_t rows)
{
    const int64_t need = (rows + 127) / 128 * 128;
    if (m.cap >= need) return PTADD_OK;
    free_work(m);
    ptadd_status st = PTADD_OK;
#define WA(p, n) \
    if (st == PTADD_OK) st = m_alloc(&(p), (size_t)(n));
    WA(m.X, need * 32);
    WA(m.Xt, need * 32);
    for (int l = 0; l < 3; ++l) {
        WA(m.Hb[l], need * NH);
        WA(m.Ht[l], need * NH);
        WA(m.dZ[l], need * NH);
        WA(m.dZt[l], need * NH);
        WA(m.Z[l], need * NH);
    }
    WA(m.dY, need * 16);
    WA(m.dYt, need * 16);
    WA(m.Y, need * 16);
    WA(m.T, need * 16);
    WA(m.loss_part, (need + 255) / 256);
#undef WA
    if (st != PTADD_OK) {
        free_work(m);
        return st;
    }
    m.cap = need;
    return PTADD_OK;
}

// ------------------------------------------------------------- kernels
// BF16 copies of W (row-major) and W^T.
__global__ void mlp_sync_bf16(const float* __restrict__ W, int dout, int din, __nv_bfloat16* __restrict__ Wb,
                              __nv_bfloat16* __restrict__ Wt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dout * din) return;
    const int o = i / din, c = i % din;
    const __nv_bfloat16 v = __float2bfloat16_rn(W[i]);
    Wb[i] = v;
    Wt[(int64_t)c * dout + o] = v;
}

// Adam on one parameter array (FP32 master), Kingma & Ba bias correction.
__global__ void mlp_adam(int n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                         float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Normalised inputs [n x 30] (FP32) -> X [rows x 32] BF16 and X^T [32 x rows]; zero padding.
__global__ void mlp_pack_x(int64_t n, int64_t rows, const float* __restrict__ xn, const int32_t* __restrict__ idx,
                           __nv_bfloat16* __restrict__ X, __nv_bfloat16* __restrict__ Xt)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= rows * 32) return;
    const int64_t r = i / 32;
    const int c = (int)(i % 32);
    float v = 0.0f;
    if (r < n && c < NIN) {
        const int64_t src = idx ? idx[r] : r;
        v = xn[src * NIN + c];
    }
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    X[r * 32 + c] = h;
    Xt[(int64_t)c * rows + r] = h;
}

__global__ void mlp_pack_t(int64_t n, int64_t rows, const float* __restrict__ yn, const int32_t* __restrict__ idx,
                           float* __restrict__ T)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= rows * 16) return;
    const int64_t r = i / 16;
    const int c = (int)(i % 16);
    float v = 0.0f;
    if (r < n && c < NOUT) {
        const int64_t src = idx ? idx[r] : r;
        v = yn[src * NOUT + c];
    }
    T[i] = v;
}

// dY = 2 (Y - T) / (n 6) on the n valid rows and 6 outputs (zero elsewhere),
// BF16 in both layouts; per-block partial loss sums.
__global__ void mlp_loss_dy(int64_t n, int64_t rows, const float* __restrict__ Y, const float* __restrict__ T,
                            __nv_bfloat16* __restrict__ dY, __nv_bfloat16* __restrict__ dYt, float* __restrict__ part)
{
    __shared__ float red[256];
    const int64_t r = blockIdx.x * (int64_t)256 + threadIdx.x;
    const float scale = 1.0f / ((float)n * NOUT);
    float loss = 0.0f;
    if (r < rows) {
        for (int c = 0; c < 16; ++c) {
            float d = 0.0f;
            if (r < n && c < NOUT) {
                const float e = Y[r * 16 + c] - T[r * 16 + c];
                loss += e * e * scale;
                d = 2.0f * e * scale;
            }
            const __nv_bfloat16 h = __float2bfloat16_rn(d);
            dY[r * 16 + c] = h;
            dYt[(int64_t)c * rows + r] = h;
        }
    }
    red[threadIdx.x] = loss;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Bias gradients: row sums of the transposed dZ^T [dout x rows] (one warp per row).
__global__ void mlp_bias_grad(int dout, int64_t rows, const __nv_bfloat16* __restrict__ dZt, float* __restrict__ gb)
{
    const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (row >= dout) return;
    float s = 0.0f;
    for (int64_t k = lane; k < rows; k += 32) s += __bfloat162float(dZt[(int64_t)row * rows + k]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) gb[row] = s;
}

// Y [rows x 16] -> normalised outputs [n x 6]
__global__ void mlp_unpack_y(int64_t n, const float* __restrict__ Y, float* __restrict__ yn)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n * NOUT) return;
    yn[i] = Y[(i / NOUT) * 16 + (i % NOUT)];
}

// ------------------------------------------------------------ passes
GemmArgs gemm(const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb, int64_t M, int N, int K,
              int epi, int* err)
{
    GemmArgs g{};
    g.A = A;
    g.lda = lda;
    g.B = B;
    g.ldb = ldb;
    g.M = M;
    g.N = N;
    g.K = K;
    g.epi = epi;
    g.err = err;
    return g;
}

// forward of `rows` packed rows (X already packed); train = keep Z, H^T
cudaError_t forward(MlpDev& m, int64_t rows, bool train, cudaStream_t s, int64_t* launches)
{
    const __nv_bfloat16* in = m.X;
    int64_t ld_in = 32;
    for (int l = 0; l < 3; ++l) {
        GemmArgs g = gemm(in, ld_in, m.Wb[l], DIN_P[l], rows, NH, DIN_P[l], EPI_BIAS_GELU, m.err);
        g.bias = m.b[l];
        g.out_f32 = train ? m.Z[l] : nullptr;
        g.ld_out = NH;
        g.out_bf16 = m.Hb[l];
        g.ld_bf16 = NH;
        g.out_bf16_t = train ? m.Ht[l] : nullptr;
        g.ld_t = rows;
        cudaError_t e = launch_tc_gemm(g, s);
        if (e != cudaSuccess) return e;
        in = m.Hb[l];
        ld_in = NH;
    }
    GemmArgs g = gemm(in, NH, m.Wb[3], NH, rows, 16, NH, EPI_BIAS, m.err);
    g.bias = m.b[3];
    g.out_f32 = m.Y;
    g.ld_out = 16;
    *launches += 4;
    return launch_tc_gemm(g, s);
}

// loss, backward, bias gradients (rows padded to a multiple of 16; n valid)
cudaError_t backward(MlpDev& m, int64_t n, int64_t rows, cudaStream_t s, int64_t* launches)
{
    const unsigned nb = (unsigned)((rows + 255) / 256);
    mlp_loss_dy<<<nb, 256, 0, s>>>(n, rows, m.Y, m.T, m.dY, m.dYt, m.loss_part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const __nv_bfloat16* dz = m.dY;   // [rows x dout]
    const __nv_bfloat16* dzt = m.dYt; // [dout x rows]
    for (int l = 3; l >= 0; --l) {
        // dW_l = dZ_l^T H_{l-1}
        const __nv_bfloat16* hin_t = l > 0 ? m.Ht[l - 1] : m.Xt;
        GemmArgs g = gemm(dzt, rows, hin_t, rows, DOUT_P[l], DIN_P[l], (int)rows, EPI_STORE, m.err);
        g.out_f32 = m.gW[l];
        g.ld_out = DIN_P[l];
        e = launch_tc_gemm(g, s);
        if (e != cudaSuccess) return e;
        mlp_bias_grad<<<(DOUT_P[l] + 7) / 8, 256, 0, s>>>(DOUT_P[l], rows, dzt, m.gb[l]);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        *launches += 2;
        if (l == 0) break;
        // dZ_{l-1} = (dZ_l W_l) * GELU'(Z_{l-1})
        GemmArgs h = gemm(dz, DOUT_P[l], m.Wt[l], DOUT_P[l], rows, DIN_P[l], DOUT_P[l], EPI_DGELU, m.err);
        h.zin = m.Z[l - 1];
        h.ld_z = NH;
        h.out_bf16 = m.dZ[l - 1];
        h.ld_bf16 = NH;
        h.out_bf16_t = m.dZt[l - 1];
        h.ld_t = rows;
        e = launch_tc_gemm(h, s);
        if (e != cudaSuccess) return e;
        *launches += 1;
        dz = m.dZ[l - 1];
        dzt = m.dZt[l - 1];
    }
    *launches += 1;
    return cudaSuccess;
}

cudaError_t sync_bf16(MlpDev& m, cudaStream_t s)
{
    for (int l = 0; l < 4; ++l) {
        const int n = DOUT_P[l] * DIN_P[l];
        mlp_sync_bf16<<<(n + 255) / 256, 256, 0, s>>>(m.W[l], DOUT_P[l], DIN_P[l], m.Wb[l], m.Wt[l]);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t adam_all(MlpDev& m, float lr, float b1, float b2, float eps, cudaStream_t s)
{
    m.step += 1;
    const float c1 = 1.0f - powf(b1, (float)m.step), c2 = 1.0f - powf(b2, (float)m.step);
    for (int l = 0; l < 4; ++l) {
        const int nw = DOUT_P[l] * DIN_P[l], nbias = DOUT_P[l];
        mlp_adam<<<(nw + 255) / 256, 256, 0, s>>>(nw, m.W[l], m.gW[l], m.mW[l], m.vW[l], lr, b1, b2, eps, c1, c2);
        mlp_adam<<<(nbias + 255) / 256, 256, 0, s>>>(nbias, m.b[l], m.gb[l], m.mb[l], m.vb[l], lr, b1, b2, eps, c1,
                                                     c2);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return sync_bf16(m, s);
}

// packed (unpadded, oracle order) <-> padded device layout
int64_t packed_count()
{
    int64_t c = 0;
    for (int l = 0; l < 4; ++l) c += (int64_t)DOUT_U[l] * DIN_U[l] + DOUT_U[l];
    return c;
}

ptadd_status read_loss(MlpDev& m, int64_t rows, cudaStream_t s, float* loss)
{
    const int nb = (int)((rows + 255) / 256);
    std::vector<float> part(nb);
    PTADD_CUDA(cudaMemcpyAsync(part.data(), m.loss_part, nb * sizeof(float), cudaMemcpyDeviceToHost, s));
    int err = 0;
    PTADD_CUDA(cudaMemcpyAsync(&err, m.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    PTADD_CUDA(cudaStreamSynchronize(s));
    if (err) {
        set_error("a tensor-core wait gave up");
        return PTADD_ERR_TIMEOUT;
    }
    double t = 0.0;
    for (float p : part) t += p;
    if (loss) *loss = (float)t;
    return PTADD_OK;
}

}  // namespace

void mlp_free(ptadd_ctx* ctx)
{
    if (ctx && ctx->mlp) {
        free_mlp(*ctx->mlp);
        delete ctx->mlp;
        ctx->mlp = nullptr;
    }
}

}  // namespace ptadd

using namespace ptadd;

static ptadd_status marg(const char* m)
{
    set_error("%s", m);
    return PTADD_ERR_ARG;
}

static ptadd_status need_mlp(ptadd_ctx* ctx)
{
    if (!ctx) return marg("null context");
    PTADD_CUDA(cudaSetDevice(ctx->device));
    if (!ctx->mlp || !ctx->mlp->ready) {
        set_error("surrogate not initialised (ptadd_mlp_init / ptadd_mlp_set_params)");
        return PTADD_ERR_STATE;
    }
    return PTADD_OK;
}

// splitmix64 (Steele, Lea & Flood 2014) for the weight initialisation
static uint64_t splitmix64(uint64_t& s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

extern "C" {

int64_t ptadd_mlp_param_count(void) { return packed_count(); }

ptadd_status ptadd_mlp_set_params(ptadd_ctx* ctx, const float* p, int64_t count)
{
    if (!ctx) return marg("null context");
    if (!p || count != packed_count()) return marg("parameter array must hold ptadd_mlp_param_count() floats");
    PTADD_CUDA(cudaSetDevice(ctx->device));
    if (!ctx->mlp) {
        ctx->mlp = new (std::nothrow) MlpDev();
        if (!ctx->mlp) return marg("host allocation failed");
        ptadd_status st = alloc_params(*ctx->mlp);
        if (st != PTADD_OK) {
            free_mlp(*ctx->mlp);
            delete ctx->mlp;
            ctx->mlp = nullptr;
            return st;
        }
    }
    MlpDev& m = *ctx->mlp;
    cudaStream_t s = ctx->own_stream;
    int64_t off = 0;
    for (int l = 0; l < 4; ++l) {
        std::vector<float> W((size_t)DOUT_P[l] * DIN_P[l], 0.0f), b(DOUT_P[l], 0.0f);
        for (int o = 0; o < DOUT_U[l]; ++o)
            for (int c = 0; c < DIN_U[l]; ++c) W[(size_t)o * DIN_P[l] + c] = p[off++];
        for (int o = 0; o < DOUT_U[l]; ++o) b[o] = p[off++];
        PTADD_CUDA(cudaMemcpyAsync(m.W[l], W.data(), W.size() * 4, cudaMemcpyHostToDevice, s));
        PTADD_CUDA(cudaMemcpyAsync(m.b[l], b.data(), b.size() * 4, cudaMemcpyHostToDevice, s));
        PTADD_CUDA(cudaMemsetAsync(m.mW[l], 0, W.size() * 4, s));
        PTADD_CUDA(cudaMemsetAsync(m.vW[l], 0, W.size() * 4, s));
        PTADD_CUDA(cudaMemsetAsync(m.mb[l], 0, b.size() * 4, s));
        PTADD_CUDA(cudaMemsetAsync(m.vb[l], 0, b.size() * 4, s));
        PTADD_CUDA(cudaStreamSynchronize(s));  // W, b are host temporaries
    }
    PTADD_CUDA(sync_bf16(m, s));
    PTADD_CUDA(cudaMemsetAsync(m.err, 0, sizeof(int), s));
    PTADD_CUDA(cudaStreamSynchronize(s));
    m.step = 0;
    m.ready = true;
    return PTADD_OK;
}

ptadd_status ptadd_mlp_get_params(ptadd_ctx* ctx, float* p, int64_t count)
{
    ptadd_status st = need_mlp(ctx);
    if (st != PTADD_OK) return st;
    if (!p || count != packed_count()) return marg("parameter array must hold ptadd_mlp_param_count() floats");
    MlpDev& m = *ctx->mlp;
    cudaStream_t s = ctx->own_stream;
    int64_t off = 0;
    for (int l = 0; l < 4; ++l) {
        std::vector<float> W((size_t)DOUT_P[l] * DIN_P[l]), b(DOUT_P[l]);
        PTADD_CUDA(cudaMemcpyAsync(W.data(), m.W[l], W.size() * 4, cudaMemcpyDeviceToHost, s));
        PTADD_CUDA(cudaMemcpyAsync(b.data(), m.b[l], b.size() * 4, cudaMemcpyDeviceToHost, s));
        PTADD_CUDA(cudaStreamSynchronize(s));
        for (int o = 0; o < DOUT_U[l]; ++o)
            for (int c = 0; c < DIN_U[l]; ++c) p[off++] = W[(size_t)o * DIN_P[l] + c];
        for (int o = 0; o < DOUT_U[l]; ++o) p[off++] = b[o];
    }
    return PTADD_OK;
}

ptadd_status ptadd_mlp_init(ptadd_ctx* ctx, uint64_t seed)
{
    if (!ctx) return marg("null context");
    // Glorot-uniform weights U(-sqrt(6/(din+dout)), +), zero biases
    std::vector<float> p((size_t)packed_count());
    uint64_t s = seed;
    size_t off = 0;
    for (int l = 0; l < 4; ++l) {
        const double a = sqrt(6.0 / (DIN_U[l] + DOUT_U[l]));
        for (int i = 0; i < DOUT_U[l] * DIN_U[l]; ++i) {
            const double u = (double)(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
            p[off++] = (float)((2.0 * u - 1.0) * a);
        }
        for (int i = 0; i < DOUT_U[l]; ++i) p[off++] = 0.0f;
    }
    return ptadd_mlp_set_params(ctx, p.data(), (int64_t)p.size());
}

ptadd_status ptadd_mlp_loss_grad(ptadd_ctx* ctx, int64_t n, const float* xn, const float* yn, float* grad,
                                 float* loss)
{
    ptadd_status st = need_mlp(ctx);
    if (st != PTADD_OK) return st;
    if (n < 1 || !xn || !yn) return marg("need n >= 1 and inputs");
    MlpDev& m = *ctx->mlp;
    cudaStream_t s = ctx->own_stream;
    const int64_t rows = (n + 15) / 16 * 16;
    st = ensure_work(m, rows);
    if (st != PTADD_OK) return st;
    float *dx = nullptr, *dy = nullptr;
    if ((st = m_alloc(&dx, (size_t)n * NIN)) != PTADD_OK) return st;
    if ((st = m_alloc(&dy, (size_t)n * NOUT)) != PTADD_OK) {
        cudaFree(dx);
        return st;
    }
    int64_t launches = 0;
    cudaError_t e = cudaMemcpyAsync(dx, xn, (size_t)n * NIN * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dy, yn, (size_t)n * NOUT * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        mlp_pack_x<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, s>>>(n, rows, dx, nullptr, m.X, m.Xt);
        mlp_pack_t<<<(unsigned)((rows * 16 + 255) / 256), 256, 0, s>>>(n, rows, dy, nullptr, m.T);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = forward(m, rows, true, s, &launches);
    if (e == cudaSuccess) e = backward(m, n, rows, s, &launches);
    if (e != cudaSuccess) {
        cudaFree(dx);
        cudaFree(dy);
        set_error("surrogate gradient: %s", cudaGetErrorString(e));
        return PTADD_ERR_CUDA;
    }
    st = read_loss(m, rows, s, loss);
    cudaFree(dx);
    cudaFree(dy);
    if (st != PTADD_OK) return st;
    if (grad) {
        int64_t off = 0;
        for (int l = 0; l < 4; ++l) {
            std::vector<float> W((size_t)DOUT_P[l] * DIN_P[l]), b(DOUT_P[l]);
            PTADD_CUDA(cudaMemcpyAsync(W.data(), m.gW[l], W.size() * 4, cudaMemcpyDeviceToHost, s));
            PTADD_CUDA(cudaMemcpyAsync(b.data(), m.gb[l], b.size() * 4, cudaMemcpyDeviceToHost, s));
            PTADD_CUDA(cudaStreamSynchronize(s));
            for (int o = 0; o < DOUT_U[l]; ++o)
                for (int c = 0; c < DIN_U[l]; ++c) grad[off++] = W[(size_t)o * DIN_P[l] + c];
            for (int o = 0; o < DOUT_U[l]; ++o) grad[off++] = b[o];
        }
    }
    ctx->kernel_launches += launches + 2;
    return PTADD_OK;
}

ptadd_status ptadd_mlp_train(ptadd_ctx* ctx, int64_t n, const float* xn, const float* yn, int epochs, int batch,
                             float lr, uint64_t seed, float* loss_per_epoch)
{
    ptadd_status st = need_mlp(ctx);
    if (st != PTADD_OK) return st;
    if (n < 16 || !xn || !yn || epochs < 0 || batch < 16 || batch % 16 || !(lr > 0))
        return marg("need n >= 16, inputs, epochs >= 0, batch a positive multiple of 16, lr > 0");
    MlpDev& m = *ctx->mlp;
    cudaStream_t s = ctx->own_stream;
    const int64_t rows = batch;
    st = ensure_work(m, rows);
    if (st != PTADD_OK) return st;
    float *dx = nullptr, *dy = nullptr, *dloss = nullptr;
    int32_t* didx = nullptr;
    // per-minibatch loss partials of an epoch, kept on the device and read once
    // per epoch (reading them per minibatch would stall the stream every time)
    const int nb = (int)((rows + 255) / 256);
    const int64_t nbatches = n / batch;
    if ((st = m_alloc(&dx, (size_t)n * NIN)) != PTADD_OK) return st;
    if ((st = m_alloc(&dy, (size_t)n * NOUT)) != PTADD_OK || (st = m_alloc(&didx, (size_t)n)) != PTADD_OK ||
        (st = m_alloc(&dloss, (size_t)std::max<int64_t>(1, nbatches) * nb)) != PTADD_OK) {
        cudaFree(dx);
        cudaFree(dy);
        cudaFree(didx);
        return st;
    }
    std::vector<float> hloss((size_t)std::max<int64_t>(1, nbatches) * nb);
    std::vector<int32_t> perm(n);
    std::iota(perm.begin(), perm.end(), 0);
    uint64_t rs = seed;
    int64_t launches = 0;
    cudaError_t e = cudaMemcpyAsync(dx, xn, (size_t)n * NIN * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dy, yn, (size_t)n * NOUT * 4, cudaMemcpyHostToDevice, s);
    for (int ep = 0; ep < epochs && e == cudaSuccess && st == PTADD_OK; ++ep) {
        // Fisher-Yates shuffle of the sample order (host), copied once per epoch
        for (int64_t i = n - 1; i > 0; --i) std::swap(perm[i], perm[splitmix64(rs) % (uint64_t)(i + 1)]);
        e = cudaMemcpyAsync(didx, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s);
        double ep_loss = 0.0;
        int nbatch = 0;
        for (int64_t b0 = 0; b0 + batch <= n && e == cudaSuccess; b0 += batch) {  // full batches only
            mlp_pack_x<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, s>>>(batch, rows, dx, didx + b0, m.X, m.Xt);
            mlp_pack_t<<<(unsigned)((rows * 16 + 255) / 256), 256, 0, s>>>(batch, rows, dy, didx + b0, m.T);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = forward(m, rows, true, s, &launches);
            if (e == cudaSuccess) e = backward(m, batch, rows, s, &launches);
            if (e == cudaSuccess) e = adam_all(m, lr, 0.9f, 0.999f, 1e-8f, s);
            launches += 2 + 8 + 4;
            if (e == cudaSuccess && loss_per_epoch)
                e = cudaMemcpyAsync(dloss + (size_t)nbatch * nb, m.loss_part, nb * sizeof(float),
                                    cudaMemcpyDeviceToDevice, s);
            ++nbatch;
        }
        if (e == cudaSuccess && loss_per_epoch && nbatch)
            e = cudaMemcpyAsync(hloss.data(), dloss, (size_t)nbatch * nb * sizeof(float), cudaMemcpyDeviceToHost, s);
        // a synchronisation per epoch keeps the host copy of perm safe to rewrite
        cudaError_t e2 = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess && loss_per_epoch) {
            // each minibatch's loss as its partials summed in order, then the epoch mean
            for (int b = 0; b < nbatch; ++b) {
                double t = 0.0;
                for (int q = 0; q < nb; ++q) t += hloss[(size_t)b * nb + q];
                ep_loss += (float)t;
            }
            loss_per_epoch[ep] = nbatch ? (float)(ep_loss / nbatch) : 0.0f;
        }
        if (e == cudaSuccess) {  // a tensor-core wait that gave up ends the training at the epoch's end
            int err = 0;
            e = cudaMemcpy(&err, m.err, sizeof(int), cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && err) {
                set_error("a tensor-core wait gave up");
                st = PTADD_ERR_TIMEOUT;
            }
        }
    }
    cudaFree(dx);
    cudaFree(dy);
    cudaFree(didx);
    cudaFree(dloss);
    if (e != cudaSuccess) {
        set_error("surrogate training: %s", cudaGetErrorString(e));
        return PTADD_ERR_CUDA;
    }
    if (st != PTADD_OK) return st;
    int err = 0;
    PTADD_CUDA(cudaMemcpy(&err, m.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        set_error("a tensor-core wait gave up");
        return PTADD_ERR_TIMEOUT;
    }
    ctx->kernel_launches += launches;
    return PTADD_OK;
}

ptadd_status ptadd_mlp_forward(ptadd_ctx* ctx, int64_t n, const float* xn, float* yn)
{
    ptadd_status st = need_mlp(ctx);
    if (st != PTADD_OK) return st;
    if (n < 1 || !xn || !yn) return marg("need n >= 1 and arrays");
    MlpDev& m = *ctx->mlp;
    cudaStream_t s = ctx->own_stream;
    const int64_t chunk = std::min<int64_t>((n + 127) / 128 * 128, 65536);
    st = ensure_work(m, chunk);
    if (st != PTADD_OK) return st;
    float *dx = nullptr, *dy = nullptr;
    if ((st = m_alloc(&dx, (size_t)chunk * NIN)) != PTADD_OK) return st;
    if ((st = m_alloc(&dy, (size_t)chunk * NOUT)) != PTADD_OK) {
        cudaFree(dx);
        return st;
    }
    int64_t launches = 0;
    cudaError_t e = cudaSuccess;
    for (int64_t r0 = 0; r0 < n && e == cudaSuccess; r0 += chunk) {
        const int64_t k = std::min(chunk, n - r0);
        const int64_t rows = (k + 127) / 128 * 128;
        e = cudaMemcpyAsync(dx, xn + r0 * NIN, (size_t)k * NIN * 4, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) break;
        mlp_pack_x<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, s>>>(k, rows, dx, nullptr, m.X, m.Xt);
        e = forward(m, rows, false, s, &launches);
        if (e != cudaSuccess) break;
        mlp_unpack_y<<<(unsigned)((k * NOUT + 255) / 256), 256, 0, s>>>(k, m.Y, dy);
        e = cudaMemcpyAsync(yn + r0 * NOUT, dy, (size_t)k * NOUT * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        launches += 2;
    }
    cudaFree(dx);
    cudaFree(dy);
    if (e != cudaSuccess) {
        set_error("surrogate forward: %s", cudaGetErrorString(e));
        return PTADD_ERR_CUDA;
    }
    ctx->kernel_launches += launches;
    int err = 0;
    PTADD_CUDA(cudaMemcpy(&err, m.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        set_error("a tensor-core wait gave up");
        return PTADD_ERR_TIMEOUT;
    }
    return PTADD_OK;
}


// ----------------------------------------------------------- closures
// Device copy of the maps (FP32): xm, xs, ym, ys, box lo, box hi, the inverse
// of the Cholesky factor (lower triangle, so that the Mahalanobis distance is
// |L^-1 z|^2 by independent dot products), threshold.
static ptadd_status upload_maps(MlpDev& m)
{
    std::vector<double> inv(NIN * NIN, 0.0);
    for (int c = 0; c < NIN; ++c)  // forward substitution for column c of L^-1
        for (int i = c; i < NIN; ++i) {
            double s2 = i == c ? 1.0 : 0.0;
            for (int j = c; j < i; ++j) s2 -= m.chol[i * NIN + j] * inv[j * NIN + c];
            inv[i * NIN + c] = s2 / m.chol[i * NIN + i];
        }
    std::vector<float> nvf(4 * NIN + 2 * NOUT + NIN * NIN + 1);
    for (int c = 0; c < NIN; ++c) {
        nvf[c] = (float)m.xm[c];
        nvf[NIN + c] = (float)m.xs[c];
        nvf[2 * NIN + 2 * NOUT + c] = (float)m.box_lo[c];
        nvf[3 * NIN + 2 * NOUT + c] = (float)m.box_hi[c];
    }
    for (int c = 0; c < NOUT; ++c) {
        nvf[2 * NIN + c] = (float)m.ym[c];
        nvf[2 * NIN + NOUT + c] = (float)m.ys[c];
    }
    for (int i = 0; i < NIN * NIN; ++i) nvf[4 * NIN + 2 * NOUT + i] = (float)inv[i];
    nvf[4 * NIN + 2 * NOUT + NIN * NIN] = (float)m.d2_thr;
    PTADD_CUDA(cudaMemcpy(m.d_norm, nvf.data(), nvf.size() * sizeof(float), cudaMemcpyHostToDevice));
    return PTADD_OK;
}

static double host_feature(const double* raw, int c)
{
    // the inference kernel's arithmetic: the input rounded to FP32, then FP32 operations
    return c < 6 ? (double)((float)raw[c] * (float)(1.0 / SIG_SCALE))
                 : (double)log10f((float)raw[c] + (float)RHO_FLOOR);
}

ptadd_status ptadd_surrogate_fit(ptadd_ctx* ctx, int64_t n, const double* feat, const double* lp6, int epochs,
                                 int batch, float lr, uint64_t seed, float* loss_per_epoch)
{
    if (!ctx) return marg("null context");
    if (n < 64 || !feat || !lp6) return marg("need n >= 64 samples and arrays");
    PTADD_CUDA(cudaSetDevice(ctx->device));
    if (!ctx->mlp || !ctx->mlp->ready) {
        ptadd_status st = ptadd_mlp_init(ctx, seed ^ 0x5EEDull);
        if (st != PTADD_OK) return st;
    }
    MlpDev& m = *ctx->mlp;
    // input map and standardisation
    std::vector<double> z((size_t)n * NIN);
    for (int64_t r = 0; r < n; ++r)
        for (int c = 0; c < NIN; ++c) {
            const double v = host_feature(feat + r * NIN, c);
            if (!isfinite(v)) return marg("non-finite feature (densities must be >= 0)");
            z[r * NIN + c] = v;
        }
    for (int c = 0; c < NIN; ++c) {
        double s1 = 0, s2 = 0;
        for (int64_t r = 0; r < n; ++r) s1 += z[r * NIN + c];
        const double mean = s1 / n;
        for (int64_t r = 0; r < n; ++r) s2 += (z[r * NIN + c] - mean) * (z[r * NIN + c] - mean);
        const double sd = sqrt(s2 / n);
        m.xm[c] = mean;
        m.xs[c] = sd > 1e-12 ? sd : 1.0;
        double lo = INFINITY, hi = -INFINITY;
        for (int64_t r = 0; r < n; ++r) {
            double& v = z[r * NIN + c];
            v = (v - m.xm[c]) / m.xs[c];
            lo = std::min(lo, v);
            hi = std::max(hi, v);
        }
        m.box_lo[c] = lo;
        m.box_hi[c] = hi;
    }
    for (int c = 0; c < NOUT; ++c) {
        double s1 = 0, s2 = 0;
        for (int64_t r = 0; r < n; ++r) {
            if (!isfinite(lp6[r * NOUT + c])) return marg("non-finite label");
            s1 += lp6[r * NOUT + c];
        }
        const double mean = s1 / n;
        for (int64_t r = 0; r < n; ++r) s2 += (lp6[r * NOUT + c] - mean) * (lp6[r * NOUT + c] - mean);
        const double sd = sqrt(s2 / n);
        m.ym[c] = mean;
        m.ys[c] = sd > 0 ? sd : 1.0;
    }
    // Mahalanobis metric of the standardised inputs: covariance + small ridge, Cholesky
    std::vector<double> C(NIN * NIN, 0.0);
    for (int64_t r = 0; r < n; ++r)
        for (int i = 0; i < NIN; ++i)
            for (int j = 0; j <= i; ++j) C[i * NIN + j] += z[r * NIN + i] * z[r * NIN + j] / n;
    for (int i = 0; i < NIN; ++i) C[i * NIN + i] += 1e-6;
    double* L = m.chol;
    for (int i = 0; i < NIN * NIN; ++i) L[i] = 0.0;
    for (int i = 0; i < NIN; ++i)
        for (int j = 0; j <= i; ++j) {
            double s2 = C[i * NIN + j];
            for (int k = 0; k < j; ++k) s2 -= L[i * NIN + k] * L[j * NIN + k];
            if (i == j) {
                if (!(s2 > 0)) return marg("degenerate training inputs (covariance not positive definite)");
                L[i * NIN + i] = sqrt(s2);
            } else {
                L[i * NIN + j] = s2 / L[j * NIN + j];
            }
        }
    std::vector<double> d2(n);
    for (int64_t r = 0; r < n; ++r) {
        double w[NIN], acc = 0.0;
        for (int i = 0; i < NIN; ++i) {
            double s2 = z[r * NIN + i];
            for (int j = 0; j < i; ++j) s2 -= L[i * NIN + j] * w[j];
            w[i] = s2 / L[i * NIN + i];
            acc += w[i] * w[i];
        }
        d2[r] = acc;
    }
    std::vector<double> sorted = d2;
    std::sort(sorted.begin(), sorted.end());
    m.d2_thr = sorted[(size_t)std::min<int64_t>(n - 1, (int64_t)ceil(0.99 * n) - 1)];
    m.have_norm = true;
    ptadd_status st = upload_maps(m);
    if (st != PTADD_OK) return st;
    // normalised training arrays
    std::vector<float> xn((size_t)n * NIN), yn((size_t)n * NOUT);
    for (int64_t i = 0; i < n * NIN; ++i) xn[i] = (float)z[i];
    for (int64_t r = 0; r < n; ++r)
        for (int c = 0; c < NOUT; ++c) yn[r * NOUT + c] = (float)((lp6[r * NOUT + c] - m.ym[c]) / m.ys[c]);
    return ptadd_mlp_train(ctx, n, xn.data(), yn.data(), epochs, batch, lr, seed, loss_per_epoch);
}

// Device arrays: feat_dev [n x 30] raw features, lp6_dev [n x 6] (sym Lp, 1/s),
// in_region_dev [n] (or NULL).  Enqueued on the context's stream.
ptadd_status ptadd_surrogate_predict_dev(ptadd_ctx* ctx, int64_t n, const double* feat_dev, double* lp6_dev,
                                         uint8_t* in_region_dev)
{
    ptadd_status st = need_mlp(ctx);
    if (st != PTADD_OK) return st;
    MlpDev& m = *ctx->mlp;
    if (!m.have_norm) {
        set_error("surrogate has no input/output maps (ptadd_surrogate_fit or ptadd_surrogate_set_state)");
        return PTADD_ERR_STATE;
    }
    if (n < 1 || !feat_dev || !lp6_dev) return marg("need n >= 1 and arrays");
    // one fused persistent kernel: input map, trust region, the four layers, output map
    const __nv_bfloat16* W[4] = {m.Wb[0], m.Wb[1], m.Wb[2], m.Wb[3]};
    const float* b[4] = {m.b[0], m.b[1], m.b[2], m.b[3]};
    PTADD_CUDA(launch_mlp_infer(feat_dev, n, m.d_norm, W, b, m.Wc, lp6_dev, in_region_dev, m.err, ctx->stream));
    ctx->kernel_launches += 2;
    return PTADD_OK;
}

ptadd_status ptadd_surrogate_predict(ptadd_ctx* ctx, int64_t n, const double* feat, double* lp6, uint8_t* in_region)
{
    ptadd_status st = need_mlp(ctx);
    if (st != PTADD_OK) return st;
    if (n < 1 || !feat || !lp6) return marg("need n >= 1 and arrays");
    double *df = nullptr, *dl = nullptr;
    uint8_t* dr = nullptr;
    if ((st = m_alloc(&df, (size_t)n * NIN)) != PTADD_OK) return st;
    if ((st = m_alloc(&dl, (size_t)n * NOUT)) != PTADD_OK || (st = m_alloc(&dr, (size_t)n)) != PTADD_OK) {
        cudaFree(df);
        cudaFree(dl);
        return st;
    }
    cudaStream_t s = ctx->stream;
    cudaError_t e = cudaMemcpyAsync(df, feat, (size_t)n * NIN * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) st = ptadd_surrogate_predict_dev(ctx, n, df, dl, dr);
    if (e == cudaSuccess && st == PTADD_OK) e = cudaMemcpyAsync(lp6, dl, (size_t)n * NOUT * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && st == PTADD_OK && in_region) e = cudaMemcpyAsync(in_region, dr, (size_t)n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(df);
    cudaFree(dl);
    cudaFree(dr);
    if (st != PTADD_OK) return st;
    if (e != cudaSuccess) {
        set_error("surrogate predict: %s", cudaGetErrorString(e));
        return PTADD_ERR_CUDA;
    }
    int err = 0;
    PTADD_CUDA(cudaMemcpy(&err, ctx->mlp->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        set_error("a tensor-core wait gave up");
        return PTADD_ERR_TIMEOUT;
    }
    return PTADD_OK;
}


// state blob: magic, param count, params (FP32), then the input/output maps
static const uint64_t SURR_MAGIC = 0x50544144534d4c31ull;  // "PTADSML1"

static size_t surr_state_bytes()
{
    return 2 * sizeof(uint64_t) + (size_t)packed_count() * sizeof(float) +
           (size_t)(4 * NIN + 2 * NOUT + NIN * NIN + 1) * sizeof(double);
}

ptadd_status ptadd_surrogate_get_state(ptadd_ctx* ctx, void* buf, size_t* bytes)
{
    ptadd_status st = need_mlp(ctx);
    if (st != PTADD_OK) return st;
    if (!bytes) return marg("bytes is NULL");
    MlpDev& m = *ctx->mlp;
    if (!m.have_norm) {
        set_error("surrogate has no input/output maps to save");
        return PTADD_ERR_STATE;
    }
    const size_t need = surr_state_bytes();
    if (!buf) {
        *bytes = need;
        return PTADD_OK;
    }
    if (*bytes < need) return marg("state buffer too small");
    char* p = (char*)buf;
    const uint64_t hdr[2] = {SURR_MAGIC, (uint64_t)packed_count()};
    memcpy(p, hdr, sizeof(hdr));
    p += sizeof(hdr);
    st = ptadd_mlp_get_params(ctx, (float*)p, packed_count());
    if (st != PTADD_OK) return st;
    p += (size_t)packed_count() * sizeof(float);
    double* d = (double*)p;
    memcpy(d, m.xm, sizeof(m.xm));
    memcpy(d + NIN, m.xs, sizeof(m.xs));
    memcpy(d + 2 * NIN, m.ym, sizeof(m.ym));
    memcpy(d + 2 * NIN + NOUT, m.ys, sizeof(m.ys));
    memcpy(d + 2 * NIN + 2 * NOUT, m.box_lo, sizeof(m.box_lo));
    memcpy(d + 3 * NIN + 2 * NOUT, m.box_hi, sizeof(m.box_hi));
    memcpy(d + 4 * NIN + 2 * NOUT, m.chol, sizeof(m.chol));
    d[4 * NIN + 2 * NOUT + NIN * NIN] = m.d2_thr;
    *bytes = need;
    return PTADD_OK;
}

ptadd_status ptadd_surrogate_set_state(ptadd_ctx* ctx, const void* buf, size_t bytes)
{
    if (!ctx) return marg("null context");
    if (!buf || bytes != surr_state_bytes()) return marg("state blob has the wrong size");
    const char* p = (const char*)buf;
    uint64_t hdr[2];
    memcpy(hdr, p, sizeof(hdr));
    if (hdr[0] != SURR_MAGIC || hdr[1] != (uint64_t)packed_count()) return marg("not a surrogate state blob");
    p += sizeof(hdr);
    std::vector<float> params((size_t)packed_count());
    memcpy(params.data(), p, params.size() * sizeof(float));
    ptadd_status st = ptadd_mlp_set_params(ctx, params.data(), packed_count());
    if (st != PTADD_OK) return st;
    p += params.size() * sizeof(float);
    MlpDev& m = *ctx->mlp;
    std::vector<double> nv(4 * NIN + 2 * NOUT + NIN * NIN + 1);
    memcpy(nv.data(), p, nv.size() * sizeof(double));
    memcpy(m.xm, &nv[0], sizeof(m.xm));
    memcpy(m.xs, &nv[NIN], sizeof(m.xs));
    memcpy(m.ym, &nv[2 * NIN], sizeof(m.ym));
    memcpy(m.ys, &nv[2 * NIN + NOUT], sizeof(m.ys));
    memcpy(m.box_lo, &nv[2 * NIN + 2 * NOUT], sizeof(m.box_lo));
    memcpy(m.box_hi, &nv[3 * NIN + 2 * NOUT], sizeof(m.box_hi));
    memcpy(m.chol, &nv[4 * NIN + 2 * NOUT], sizeof(m.chol));
    m.d2_thr = nv[4 * NIN + 2 * NOUT + NIN * NIN];
    st = upload_maps(m);
    if (st != PTADD_OK) return st;
    m.have_norm = true;
    return PTADD_OK;
}

}  // extern "C"
