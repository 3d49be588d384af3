// projection.cu -- the non-negative-dissipation correction of the coupled
// model (Sec. 4, "Ensuring non-negative dissipation"): at a material point
// with Cauchy stress T and dislocation density tensor alpha, a plastic
// distortion rate Lp that dissipates negatively (T : Lp < 0) loses its
// component along T, and a polar dislocation velocity V with
// V . (X(T alpha)) < 0 loses its component along X(T alpha), where
// (X A)_i = e_ijk A_jk for the alternating tensor e.  What remains
// dissipates nothing in the removed direction.
//
// One point: ptadd_dissipation_projection (host).  Many points (the Gauss
// points of a mesh, or the realisations of a batch): one thread per point,
// ptadd_dissipation_projection_dev, on device arrays.  Both run the same
// inline function.
#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>

#include "ptadd_internal.cuh"

namespace ptadd {
namespace {

// 0: corrected in place; 1: non-finite T or Lp; 2: non-finite V or alpha
// (nothing is changed when the result is not 0).
__host__ __device__ inline int project_point(const double T6[6], const double* alpha, double Lp[9], double* V)
{
    // Voigt xx, yy, zz, yz, xz, xy -> full symmetric T (row-major)
    const double T[9] = {T6[0], T6[5], T6[4], T6[5], T6[1], T6[3], T6[4], T6[3], T6[2]};
    double TT = 0.0, d = 0.0;
    for (int k = 0; k < 9; ++k) {
        if (!isfinite(T[k]) || !isfinite(Lp[k])) return 1;
        TT += T[k] * T[k];
        d += T[k] * Lp[k];
    }
    double w[3] = {0.0, 0.0, 0.0}, ww = 0.0, beta = 0.0;
    if (V) {
        double A[9];  // T alpha
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k) s += T[3 * i + k] * alpha[3 * k + j];
                A[3 * i + j] = s;
            }
        // (X A)_i = e_ijk A_jk
        w[0] = A[5] - A[7];
        w[1] = A[6] - A[2];
        w[2] = A[1] - A[3];
        ww = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
        beta = V[0] * w[0] + V[1] * w[1] + V[2] * w[2];
        if (!isfinite(beta) || !isfinite(ww)) return 2;
    }
    if (d < 0.0 && TT > 0.0)
        for (int k = 0; k < 9; ++k) Lp[k] -= d * T[k] / TT;
    if (V && beta < 0.0 && ww > 0.0)
        for (int i = 0; i < 3; ++i) V[i] -= beta * w[i] / ww;
    return 0;
}

__global__ void projection_kernel(int64_t n, const double* __restrict__ T6, const double* __restrict__ alpha,
                                  double* __restrict__ Lp, double* __restrict__ V, int* __restrict__ n_bad)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    double t[6], l[9], a[9], v[3];
    for (int k = 0; k < 6; ++k) t[k] = T6[6 * p + k];
    for (int k = 0; k < 9; ++k) l[k] = Lp[9 * p + k];
    if (V) {
        for (int k = 0; k < 9; ++k) a[k] = alpha[9 * p + k];
        for (int k = 0; k < 3; ++k) v[k] = V[3 * p + k];
    }
    if (project_point(t, a, l, V ? v : nullptr) != 0) {
        if (n_bad) atomicAdd(n_bad, 1);
        return;
    }
    for (int k = 0; k < 9; ++k) Lp[9 * p + k] = l[k];
    if (V)
        for (int k = 0; k < 3; ++k) V[3 * p + k] = v[k];
}

}  // namespace
}  // namespace ptadd

using namespace ptadd;

extern "C" ptadd_status ptadd_dissipation_projection(const double T6[6], const double alpha[9], double Lp[9],
                                                     double V[3])
{
    if (!T6 || !Lp) {
        set_error("ptadd_dissipation_projection: null T or Lp");
        return PTADD_ERR_ARG;
    }
    if (V && !alpha) {
        set_error("ptadd_dissipation_projection: V given without alpha");
        return PTADD_ERR_ARG;
    }
    const int r = project_point(T6, alpha, Lp, V);
    if (r == 1) {
        set_error("ptadd_dissipation_projection: non-finite T or Lp");
        return PTADD_ERR_ARG;
    }
    if (r == 2) {
        set_error("ptadd_dissipation_projection: non-finite V or alpha");
        return PTADD_ERR_ARG;
    }
    return PTADD_OK;
}

extern "C" ptadd_status ptadd_dissipation_projection_dev(int64_t n_points, const double* T6_dev,
                                                         const double* alpha_dev, double* Lp_dev, double* V_dev,
                                                         int* n_bad_dev, void* stream)
{
    if (n_points < 0) {
        set_error("ptadd_dissipation_projection_dev: n_points < 0");
        return PTADD_ERR_ARG;
    }
    if (n_points == 0) return PTADD_OK;
    if (!T6_dev || !Lp_dev || (V_dev && !alpha_dev)) {
        set_error("ptadd_dissipation_projection_dev: null T6 or Lp, or V without alpha");
        return PTADD_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (n_bad_dev) PTADD_CUDA(cudaMemsetAsync(n_bad_dev, 0, sizeof(int), s));
    projection_kernel<<<(unsigned)((n_points + 255) / 256), 256, 0, s>>>(n_points, T6_dev, alpha_dev, Lp_dev, V_dev,
                                                                         n_bad_dev);
    PTADD_CUDA(cudaGetLastError());
    return PTADD_OK;
}
