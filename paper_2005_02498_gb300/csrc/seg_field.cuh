// seg_field.cuh -- the segment-pair interaction evaluated by the pair kernels.
//
// For a straight source segment (start x1, length L, unit tangent t, Burgers
// vector b, q = b x t) and a field point x, the nonsingular isotropic stress
// (Sec. 2.1, sigma = S R * alpha with |R| replaced by R_a = sqrt(R.R + a^2))
// contracted with the target's Burgers vector b' is accumulated as
//
//   s += (sigma b')  =  c_Rxb (Rp x b) + c_q q + c_Rp Rp + c_t t + c_b b'
//
// where R(u) = Rp - u t along the source (Rp the perpendicular part of
// x - x1, d^2 = |Rp|^2 + a^2, u in [u1, u2] = [-y, L - y]) and the scalar
// coefficients combine the five line integrals
//   J0 = int rho^-3, J1 = int u rho^-3, J2 = int rho^-5, J3 = int u rho^-5,
//   J4 = int u^2 rho^-5      (rho^2 = u^2 + d^2).
//
// With m = u1/rho1, p = u2/rho2 (cosines of the end points seen from x) the
// closed forms are
//   J0 = (p - m)/d^2,   J4 = J0 (p^2 + p m + m^2)/3,
//   J2 = J0 (3 - p^2 - p m - m^2)/(3 d^2),
//   J1 = 1/rho1 - 1/rho2,   J3 = J1 (1/rho1^2 + 1/(rho1 rho2) + 1/rho2^2)/3.
// They are evaluated without cancellation and with ONE reciprocal:
//   * J1 = L (u1+u2) / (rho1^2 rho2^2 (1/rho1 + 1/rho2));
//   * if both ends lie on one side of the foot of the perpendicular
//     (u1 u2 >= 0): p - m = d^2 L (u1+u2) / (rho1^2 rho2^2 (p+m)), and
//     3 - p^2 - pm - m^2 = d^2 [ (u1^2+u2^2+d^2)/(rho1^2 rho2^2 (1+pm))
//     + 1/rho1^2 + 1/rho2^2 ], so no 1/d^2 appears;
//   * otherwise p - m and 3 - p^2 - pm - m^2 >= 1 are sums of like-signed terms.
// The denominators (p+m)(1+pm) [one side] or d^2 [straddling] and
// (1/rho1 + 1/rho2) share one reciprocal.
#pragma once

#include <cuda_runtime.h>

namespace ptadd {

// ---------------------------------------------------------------- math
// Reciprocal and reciprocal square root.  FP32: the hardware approximations
// (PTX rcp.approx / rsqrt.approx).  FP64: the FP32 approximation as a seed y,
// then ONE third-order (Householder) correction: with e = 1 - x y,
// 1/x = y / (1 - e) ~ y (1 + e + e^2); with e = 1 - x y^2,
// 1/sqrt x = y (1 - e)^(-1/2) ~ y (1 + e/2 + 3 e^2 / 8).  The ~2^-22 error of
// the seed becomes ~2^-66, below the final rounding.
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// The seed's conversions on the integer pipe (the hardware FP64 <-> FP32
// conversions run on the 1/64-rate FP64 pipe here): FP64 -> FP32 by
// truncating the mantissa (the seed's own error is far larger), FP32 -> FP64
// exactly, by moving the IEEE-754 fields.  The domain is that of the FP32
// approximations with flush-to-zero, FP32's normal range, which holds the
// seeds' arguments (squared distances plus a^2 and their products).
__device__ __forceinline__ float d2f_seed(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = min(max((int)((hi >> 20) & 0x7FFu) - 896, 0), 255);
    return __uint_as_float((hi & 0x80000000u) | ((unsigned)e << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
}
__device__ __forceinline__ double f2d_seed(float y)
{
    const unsigned u = __float_as_uint(y);
    const unsigned hi = (u & 0x80000000u) | ((((u >> 23) & 0xFFu) + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
    return __hiloint2double((int)hi, (int)(u << 29));
}
__device__ __forceinline__ double rcp_nr(double x)
{
    const double y = f2d_seed(rcp_approx(d2f_seed(x)));
    const double e = fma(-x, y, 1.0);
    return fma(y, fma(e, e, e), y);
}
__device__ __forceinline__ double rsqrt_nr(double x)
{
    const double y = f2d_seed(rsqrt_approx(d2f_seed(x)));
    const double e = fma(-x * y, y, 1.0);
    return fma(y * e, fma(e, 0.375, 0.5), y);
}

// Per-pair constants that depend on the source and the target only:
// t.b', q.b' and r t.b' with r = -c1/c2.
struct PairK {
    double tb, qb, nrtb;
};

__device__ __forceinline__ void pair_constants(const double t[3], const double q[3], const double bt[3], double nr,
                                               PairK& k)
{
    k.tb = fma(t[0], bt[0], fma(t[1], bt[1], t[2] * bt[2]));
    k.qb = fma(q[0], bt[0], fma(q[1], bt[1], q[2] * bt[2]));
    k.nrtb = nr * k.tb;
}

// Accumulate (sigma b') / c2 of one source at one field point, given
// R0 = x - x1; nr = -c1/c2.  The common factor c2 of the formula is applied
// once per target by the caller, and the integrals J2, J3, J4 enter as
// K_k = 3 J_k, which removes the factors 1/3 and 3 of the closed forms:
//   A0 = a^2 K2 + 2 J0,  A1 = a^2 K3 + 2 J1,
//   c_Rxb = r t.b' A0,   c_q = r t.b' A1 + J1 t.b' - J0 (Rp.b'),
//   c_Rp = (q.Rp)(K2 (Rp.b') - K3 t.b') - J0 q.b',
//   c_t = r (A0 (Rp.(b x b')) + A1 q.b') + J1 q.b' + (q.Rp)(K4 t.b' - K3 (Rp.b')),
//   c_b = (q.Rp)(A0 - J0),
// with Rp.(b x b') evaluated as b'.(Rp x b), reusing Rp x b.
__device__ __forceinline__ void seg_sigma_b(double R0x, double R0y, double R0z, const double t[3], double L,
                                            const double b[3], const double q[3], const double bt[3],
                                            const PairK& k, double a2, double nr, double s[3])
{
    const double y = fma(R0x, t[0], fma(R0y, t[1], R0z * t[2]));  // u1 = -y
    const double Rpx = fma(-y, t[0], R0x), Rpy = fma(-y, t[1], R0y), Rpz = fma(-y, t[2], R0z);
    const double d2 = fma(Rpx, Rpx, fma(Rpy, Rpy, fma(Rpz, Rpz, a2)));
    const double u2 = L - y;
    const double r1s = fma(y, y, d2), r2s = fma(u2, u2, d2);
    const double i1 = rsqrt_nr(r1s), i2 = rsqrt_nr(r2s);
    const double m = -y * i1, p = u2 * i2;
    const bool same = (y <= 0.0) || (y >= L);  // u1 u2 >= 0
    const double i1s = i1 * i1, i2s = i2 * i2, i12 = i1s * i2s;
    const double pm = p * m;
    const double S = fma(p, p, fma(m, m, pm));
    const double isum = i1 + i2;
    const double pps = p + m, one_pm = 1.0 + pm;
    const double den = same ? pps * one_pm : d2;
    const double rr = rcp_nr(den * isum);
    const double rden = rr * isum;        // 1/den
    const double Li = L * (u2 - y) * i12;  // L (u1 + u2) / (rho1^2 rho2^2)
    const double J1 = Li * (rr * den);
    const double K3 = J1 * (i1s + fma(i1, i2, i2s));
    const double J0 = same ? (Li * rden) * one_pm : (p - m) * rden;
    const double Wt = same ? fma((r1s + u2 * u2) * i12 * rden, pps, i1s + i2s) : (3.0 - S) * rden;
    const double K2 = J0 * Wt;
    const double K4 = J0 * S;
    const double A0 = fma(a2, K2, J0 + J0);
    const double A1 = fma(a2, K3, J1 + J1);
    // Rp x b
    const double Xx = fma(Rpy, b[2], -Rpz * b[1]);
    const double Xy = fma(Rpz, b[0], -Rpx * b[2]);
    const double Xz = fma(Rpx, b[1], -Rpy * b[0]);
    const double Rb = fma(Rpx, bt[0], fma(Rpy, bt[1], Rpz * bt[2]));
    const double Rw = fma(Xx, bt[0], fma(Xy, bt[1], Xz * bt[2]));
    const double qR = fma(Rpx, q[0], fma(Rpy, q[1], Rpz * q[2]));
    const double cRxb = k.nrtb * A0;
    const double cq = fma(k.nrtb, A1, fma(J1, k.tb, -J0 * Rb));
    const double cRp = fma(qR, fma(K2, Rb, -K3 * k.tb), -J0 * k.qb);
    const double ct = fma(nr, fma(A0, Rw, A1 * k.qb), fma(J1, k.qb, qR * fma(K4, k.tb, -K3 * Rb)));
    const double cb = qR * (A0 - J0);
    s[0] = fma(cRxb, Xx, fma(cq, q[0], fma(cRp, Rpx, fma(ct, t[0], fma(cb, bt[0], s[0])))));
    s[1] = fma(cRxb, Xy, fma(cq, q[1], fma(cRp, Rpy, fma(ct, t[1], fma(cb, bt[1], s[1])))));
    s[2] = fma(cRxb, Xz, fma(cq, q[2], fma(cRp, Rpz, fma(ct, t[2], fma(cb, bt[2], s[2])))));
}

// Gauss-Legendre rule on [0,1]: the textbook 4-point abscissae z and
// weights W on [-1,1] mapped by xi = (1 + z)/2, w = W/2.
__device__ __forceinline__ double gl4_xi(int qp)
{
    constexpr double z0 = 0.8611363115940526, z1 = 0.3399810435848563;
    return qp == 0 ? 0.5 * (1.0 - z0) : qp == 1 ? 0.5 * (1.0 - z1) : qp == 2 ? 0.5 * (1.0 + z1) : 0.5 * (1.0 + z0);
}
__device__ __forceinline__ double gl4_w(int qp)
{
    constexpr double W0 = 0.3478548451374538, W1 = 0.6521451548625461;
    return (qp == 0 || qp == 3) ? 0.5 * W0 : 0.5 * W1;
}

}  // namespace ptadd
