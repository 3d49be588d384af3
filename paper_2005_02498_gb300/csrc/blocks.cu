// blocks.cu -- the block-level front end of the DD-continuum coupling
// (Sec. 4.2 and 4.2.1): the stress that drives the DD box of each block, and
// the pair of stresses one coupling increment hands to PTA at that block.
//
//   <T>_r  volume average of the Cauchy stress over block r, from the
//          stresses and volume weights of the Gauss points inside it;
//   T^_{r,t-Delta} = <T>^k_r;
//   T^_{r,t}       = <T>^k_r + (Delta* / dt^{k-1}) (<T>^k_r - <T>^{k-1}_r),
//          the linear extrapolation of the block stress over Delta*;
//   if |T^_t - T^_{t-Delta}| < gap_min (0.5 MPa in the paper), T^_t moves
//   along the gap until the gap is gap_min, and mag = gap_min / gap > 1 is
//   returned: the rates PTA gives are divided by mag, which maps them back
//   to the original stress difference.
// Host code; no GPU.
#include <math.h>
#include <stddef.h>

#include <vector>

#include "ptadd_internal.cuh"

using namespace ptadd;

namespace {

// Frobenius norm of the symmetric tensor with Voigt components v
// (xx, yy, zz, yz, xz, xy): the off-diagonal terms count twice.
double voigt_norm(const double* v)
{
    return sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + 2.0 * (v[3] * v[3] + v[4] * v[4] + v[5] * v[5]));
}

}  // namespace

extern "C" ptadd_status ptadd_block_average(int64_t n_gp, const double* T6, const double* w, const int32_t* block,
                                            int32_t n_blocks, double* T6_avg)
{
    if (n_gp < 0 || n_blocks < 1 || !T6_avg || (n_gp > 0 && (!T6 || !w || !block))) {
        set_error("ptadd_block_average: bad sizes or NULL array");
        return PTADD_ERR_ARG;
    }
    std::vector<double> sw(n_blocks, 0.0), st(6 * (size_t)n_blocks, 0.0);
    for (int64_t g = 0; g < n_gp; ++g) {
        const int32_t r = block[g];
        if (r < 0 || r >= n_blocks) {
            set_error("ptadd_block_average: Gauss point %lld has block %d, outside [0, %d)", (long long)g, r,
                      n_blocks);
            return PTADD_ERR_ARG;
        }
        if (!(w[g] > 0.0) || !isfinite(w[g])) {
            set_error("ptadd_block_average: Gauss point %lld has weight %g", (long long)g, w[g]);
            return PTADD_ERR_ARG;
        }
        for (int c = 0; c < 6; ++c) {
            if (!isfinite(T6[6 * g + c])) {
                set_error("ptadd_block_average: non-finite stress at Gauss point %lld", (long long)g);
                return PTADD_ERR_ARG;
            }
            st[6 * (size_t)r + c] += w[g] * T6[6 * g + c];
        }
        sw[r] += w[g];
    }
    for (int32_t r = 0; r < n_blocks; ++r)
        if (!(sw[r] > 0.0)) {
            set_error("ptadd_block_average: block %d holds no Gauss point", r);
            return PTADD_ERR_ARG;
        }
    for (int32_t r = 0; r < n_blocks; ++r)
        for (int c = 0; c < 6; ++c) T6_avg[6 * (size_t)r + c] = st[6 * (size_t)r + c] / sw[r];
    return PTADD_OK;
}

extern "C" ptadd_status ptadd_block_stress_pair(int32_t n_blocks, const double* T6_k, const double* T6_km1,
                                                double delta_star, double dt_prev, double gap_min, double* T6_prev,
                                                double* T6_t, double* mag)
{
    if (n_blocks < 0 || (n_blocks > 0 && (!T6_k || !T6_prev || !T6_t || !mag))) {
        set_error("ptadd_block_stress_pair: bad size or NULL array");
        return PTADD_ERR_ARG;
    }
    if (!(delta_star > 0.0) || !isfinite(delta_star) || !(gap_min >= 0.0) || !isfinite(gap_min) ||
        !isfinite(dt_prev)) {
        set_error("ptadd_block_stress_pair: need delta_star > 0, gap_min >= 0, finite dt_prev");
        return PTADD_ERR_ARG;
    }
    const bool extrapolate = T6_km1 && dt_prev > 0.0;
    for (int32_t r = 0; r < n_blocks; ++r) {
        const double* tk = T6_k + 6 * (size_t)r;
        double gap[6];
        for (int c = 0; c < 6; ++c) {
            if (!isfinite(tk[c]) || (extrapolate && !isfinite(T6_km1[6 * (size_t)r + c]))) {
                set_error("ptadd_block_stress_pair: non-finite stress at block %d", r);
                return PTADD_ERR_ARG;
            }
            gap[c] = extrapolate ? (delta_star / dt_prev) * (tk[c] - T6_km1[6 * (size_t)r + c]) : 0.0;
        }
        const double g = voigt_norm(gap);
        double m = 1.0;
        if (g < gap_min) m = g > 0.0 ? gap_min / g : INFINITY;
        for (int c = 0; c < 6; ++c) {
            T6_prev[6 * (size_t)r + c] = tk[c];
            // a zero gap has no direction to move along: T^_t stays at T^_{t-Delta}
            T6_t[6 * (size_t)r + c] = tk[c] + (isinf(m) ? 0.0 : m * gap[c]);
        }
        mag[r] = m;
    }
    return PTADD_OK;
}
