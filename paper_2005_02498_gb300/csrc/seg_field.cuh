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

// Geometry of one (field point, source) pair, given R0 = x - x1: y = R0.t
// (u1 = -y), Rp = R0 - y t (the part of R0 normal to the source), d2 =
// |Rp|^2 + a^2, u2 = L - y, rho1^2 = y^2 + d2, rho2^2 = u2^2 + d2.
struct SegGeo {
    double y, Rp[3], d2, u2, r1s, r2s;
};

__device__ __forceinline__ void seg_geo(double R0x, double R0y, double R0z, const double t[3], double L, double a2,
                                        SegGeo& G)
{
    G.y = fma(R0x, t[0], fma(R0y, t[1], R0z * t[2]));
    G.Rp[0] = fma(-G.y, t[0], R0x);
    G.Rp[1] = fma(-G.y, t[1], R0y);
    G.Rp[2] = fma(-G.y, t[2], R0z);
    G.d2 = fma(G.Rp[0], G.Rp[0], fma(G.Rp[1], G.Rp[1], fma(G.Rp[2], G.Rp[2], a2)));
    G.u2 = L - G.y;
    G.r1s = fma(G.y, G.y, G.d2);
    G.r2s = fma(G.u2, G.u2, G.d2);
}

// both ends of the source on one side of the foot of the perpendicular (u1 u2 >= 0)
__device__ __forceinline__ bool seg_one_side(const SegGeo& G, double L) { return (G.y <= 0.0) || (G.y >= L); }

// Accumulate (sigma b') / c2 of one source at one field point, given its
// geometry; nr = -c1/c2, nra2 = nr a^2, kn = 1 + 2 nr.  The common factor c2
// of the formula is applied once per target by the caller, the integrals
// J2, J3, J4 enter as K_k = 3 J_k (which removes the factors 1/3 and 3 of
// the closed forms), and the coefficient of the term along b' goes to sb
// (the caller multiplies the sum by b' once):
//   B0 = a^2 K2 + J0,  A0 = B0 + J0 (= a^2 K2 + 2 J0),
//   C1 = r (a^2 K3 + 2 J1) + J1 = (r a^2) K3 + (1 + 2r) J1,
//   c_Rxb = r t.b' A0,   c_q = C1 t.b' - J0 (Rp.b'),
//   c_Rp = (q.Rp)(K2 (Rp.b') - K3 t.b') - J0 q.b',
//   c_t = r A0 (Rp.(b x b')) + C1 q.b' + (q.Rp)(K4 t.b' - K3 (Rp.b')),
//   c_b = (q.Rp) B0,
// with Rp.(b x b') evaluated as b'.(Rp x b), reusing Rp x b.  SAME = 1: the
// caller knows the pair is one-sided; the one-side integrals then come from
// the single reciprocal rr = 1 / ((p + m)(1 + pm)(1/rho1 + 1/rho2)) through
// Q = Li rr: J0 = Li / (p + m) = Q (1 + pm) isum, J1 = Li / isum =
// Q (p + m)(1 + pm), K2 = J0 W = Q (isum Aw + (1 + pm) isum ssum), where
// W = Aw / (1 + pm) + ssum and Aw = ssum - d^2 / (rho1^2 rho2^2) =
// (u1^2 + u2^2 + d^2) / (rho1^2 rho2^2) >= ssum / 2.  SAME = 0: either form,
// chosen per pair.
template <int SAME>
__device__ __forceinline__ void seg_sigma_b_geo(const SegGeo& G, const double t[3], double L, const double b[3],
                                                const double q[3], const double bt[3], const PairK& k, double a2,
                                                double nr, double nra2, double kn, double s[3], double& sb)
{
    const double y = G.y, d2 = G.d2, u2 = G.u2, r1s = G.r1s, r2s = G.r2s;
    const double Rpx = G.Rp[0], Rpy = G.Rp[1], Rpz = G.Rp[2];
    const double i1 = rsqrt_nr(r1s), i2 = rsqrt_nr(r2s);
    const double m = -y * i1, p = u2 * i2;
    const double i1s = i1 * i1, i2s = i2 * i2, i12 = i1s * i2s;
    const double pm = p * m;
    const double S = fma(p, p, fma(m, m, pm));
    const double isum = i1 + i2, ssum = i1s + i2s;
    const double pps = p + m, one_pm = 1.0 + pm;
    const double Li = L * (u2 - y) * i12;  // L (u1 + u2) / (rho1^2 rho2^2)
    double J0, J1, K2;
    if (SAME) {
        const double T = one_pm * isum, den = pps * one_pm;
        const double rr = rcp_nr(pps * T);
        const double Z = fma(isum, fma(-d2, i12, ssum), T * ssum);
        const double Q = Li * rr;
        J0 = Q * T;
        J1 = Q * den;
        K2 = Q * Z;
    } else {
        const bool same = seg_one_side(G, L);
        const double den = same ? pps * one_pm : d2;
        const double rr = rcp_nr(den * isum);
        const double rden = rr * isum;  // 1/den
        J1 = Li * (rr * den);
        J0 = same ? (Li * rden) * one_pm : (p - m) * rden;
        const double Wt = same ? fma((r1s + u2 * u2) * i12 * rden, pps, ssum) : (3.0 - S) * rden;
        K2 = J0 * Wt;
    }
    const double K3 = J1 * fma(i1, i2, ssum);
    const double K4 = J0 * S;
    const double B0 = fma(a2, K2, J0);
    const double A0 = B0 + J0;
    const double C1 = fma(nra2, K3, kn * J1);
    // Rp x b
    const double Xx = fma(Rpy, b[2], -Rpz * b[1]);
    const double Xy = fma(Rpz, b[0], -Rpx * b[2]);
    const double Xz = fma(Rpx, b[1], -Rpy * b[0]);
    const double Rb = fma(Rpx, bt[0], fma(Rpy, bt[1], Rpz * bt[2]));
    const double Rw = fma(Xx, bt[0], fma(Xy, bt[1], Xz * bt[2]));
    const double qR = fma(Rpx, q[0], fma(Rpy, q[1], Rpz * q[2]));
    const double cRxb = k.nrtb * A0;
    const double cq = fma(C1, k.tb, -J0 * Rb);
    const double cRp = fma(qR, fma(K2, Rb, -K3 * k.tb), -J0 * k.qb);
    const double ct = fma(nr * A0, Rw, fma(C1, k.qb, qR * fma(K4, k.tb, -K3 * Rb)));
    sb = fma(qR, B0, sb);
    s[0] = fma(cRxb, Xx, fma(cq, q[0], fma(cRp, Rpx, fma(ct, t[0], s[0]))));
    s[1] = fma(cRxb, Xy, fma(cq, q[1], fma(cRp, Rpy, fma(ct, t[1], s[1]))));
    s[2] = fma(cRxb, Xz, fma(cq, q[2], fma(cRp, Rpz, fma(ct, t[2], s[2]))));
}

// (sigma b') / c2 of one source at one field point, added to s (the term
// along b' included), given R0 = x - x1.
__device__ __forceinline__ void seg_sigma_b(double R0x, double R0y, double R0z, const double t[3], double L,
                                            const double b[3], const double q[3], const double bt[3],
                                            const PairK& k, double a2, double nr, double s[3])
{
    SegGeo G;
    seg_geo(R0x, R0y, R0z, t, L, a2, G);
    double sb = 0.0;
    seg_sigma_b_geo<0>(G, t, L, b, q, bt, k, a2, nr, nr * a2, 1.0 + 2.0 * nr, s, sb);
    s[0] = fma(sb, bt[0], s[0]);
    s[1] = fma(sb, bt[1], s[1]);
    s[2] = fma(sb, bt[2], s[2]);
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
