// projection.cu -- the non-negative-dissipation correction of the coupled
// model (Sec. 4, "Ensuring non-negative dissipation"): at a material point
// with Cauchy stress T and dislocation density tensor alpha, a plastic
// distortion rate Lp that dissipates negatively (T : Lp < 0) loses its
// component along T, and a polar dislocation velocity V with
// V . (X(T alpha)) < 0 loses its component along X(T alpha), where
// (X A)_i = e_ijk A_jk for the alternating tensor e.  What remains
// dissipates nothing in the removed direction.  Host code; no GPU.
#include <math.h>
#include <stddef.h>

#include "ptadd_internal.cuh"

using namespace ptadd;

extern "C" ptadd_status ptadd_dissipation_projection(const double T6[6], const double alpha[9], double Lp[9],
                                                     double V[3])
{
    if (!T6 || !Lp) {
        set_error("ptadd_dissipation_projection: null T or Lp");
        return PTADD_ERR_ARG;
    }
    // Voigt xx, yy, zz, yz, xz, xy -> full symmetric T (row-major)
    const double T[9] = {T6[0], T6[5], T6[4], T6[5], T6[1], T6[3], T6[4], T6[3], T6[2]};
    double TT = 0.0, d = 0.0;
    for (int k = 0; k < 9; ++k) {
        if (!isfinite(T[k]) || !isfinite(Lp[k])) {
            set_error("ptadd_dissipation_projection: non-finite T or Lp");
            return PTADD_ERR_ARG;
        }
        TT += T[k] * T[k];
        d += T[k] * Lp[k];
    }
    if (d < 0.0 && TT > 0.0)
        for (int k = 0; k < 9; ++k) Lp[k] -= d * T[k] / TT;
    if (V) {
        if (!alpha) {
            set_error("ptadd_dissipation_projection: V given without alpha");
            return PTADD_ERR_ARG;
        }
        double A[9];  // T alpha
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k) s += T[3 * i + k] * alpha[3 * k + j];
                A[3 * i + j] = s;
            }
        // (X A)_i = e_ijk A_jk
        const double w[3] = {A[5] - A[7], A[6] - A[2], A[1] - A[3]};
        const double ww = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
        const double beta = V[0] * w[0] + V[1] * w[1] + V[2] * w[2];
        if (!isfinite(beta)) {
            set_error("ptadd_dissipation_projection: non-finite V or alpha");
            return PTADD_ERR_ARG;
        }
        if (beta < 0.0 && ww > 0.0)
            for (int i = 0; i < 3; ++i) V[i] -= beta * w[i] / ww;
    }
    return PTADD_OK;
}
