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
// (PTX rcp.approx / rsqrt.approx).  FP64: the FP32 approximation as a seed,
// then two Newton-Raphson steps in FP64 (y <- y + y (1 - x y) for 1/x,
// y <- y + y (1/2 - x/2 y^2) for 1/sqrt x), which square the ~2^-22 seed
// error twice.
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
__device__ __forceinline__ double rcp_nr(double x)
{
    double y = (double)rcp_approx(__double2float_rn(x));
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}
__device__ __forceinline__ double rsqrt_nr(double x)
{
    double y = (double)rsqrt_approx(__double2float_rn(x));
    const double hx = 0.5 * x;
    double e = fma(-hx * y, y, 0.5);
    y = fma(y, e, y);
    e = fma(-hx * y, y, 0.5);
    return fma(y, e, y);
}

template <typename T> struct RMath;
template <> struct RMath<double> {
    static __device__ __forceinline__ double rcp(double x) { return rcp_nr(x); }
    static __device__ __forceinline__ double rsqrt(double x) { return rsqrt_nr(x); }
};
template <> struct RMath<float> {
    static __device__ __forceinline__ float rcp(float x) { return rcp_approx(x); }
    static __device__ __forceinline__ float rsqrt(float x) { return rsqrt_approx(x); }
};

// Per-pair constants that depend on the source and the target only.
template <typename T> struct PairK {
    T tb;     // t . b'
    T qb;     // q . b'
    T w[3];   // b x b'
};

template <typename T>
__device__ __forceinline__ void pair_constants(const T t[3], const T b[3], const T q[3], const T bt[3],
                                               PairK<T>& k)
{
    k.tb = t[0] * bt[0] + t[1] * bt[1] + t[2] * bt[2];
    k.qb = q[0] * bt[0] + q[1] * bt[1] + q[2] * bt[2];
    k.w[0] = b[1] * bt[2] - b[2] * bt[1];
    k.w[1] = b[2] * bt[0] - b[0] * bt[2];
    k.w[2] = b[0] * bt[1] - b[1] * bt[0];
}

// Geometry of one (field point, source) pair from R0 = x - x1.
template <typename T> struct PairGeom {
    T y;             // R0 . t  (u1 = -y)
    T Rp[3];         // perpendicular part of R0
    T d2;            // |Rp|^2 + a^2
    T u2;            // L - y
    T r1s, r2s;      // rho1^2, rho2^2
};

template <typename T>
__device__ __forceinline__ void pair_geom(T R0x, T R0y, T R0z, const T t[3], T L, T a2, PairGeom<T>& g)
{
    g.y = R0x * t[0] + R0y * t[1] + R0z * t[2];
    g.Rp[0] = fma(-g.y, t[0], R0x);
    g.Rp[1] = fma(-g.y, t[1], R0y);
    g.Rp[2] = fma(-g.y, t[2], R0z);
    g.d2 = fma(g.Rp[0], g.Rp[0], fma(g.Rp[1], g.Rp[1], fma(g.Rp[2], g.Rp[2], a2)));
    g.u2 = L - g.y;
    g.r1s = fma(g.y, g.y, g.d2);
    g.r2s = fma(g.u2, g.u2, g.d2);
}

// Accumulate (sigma b') of one source at one field point from its geometry.
template <typename T>
__device__ __forceinline__ void seg_sigma_b_geom(const PairGeom<T>& G, const T t[3], T L, const T b[3],
                                                 const T q[3], const T bt[3], const PairK<T>& k, T a2, T c1,
                                                 T c2, T s[3])
{
    const T y = G.y, u2 = G.u2, d2 = G.d2, r1s = G.r1s, r2s = G.r2s;
    const T Rpx = G.Rp[0], Rpy = G.Rp[1], Rpz = G.Rp[2];
    const T i1 = RMath<T>::rsqrt(r1s), i2 = RMath<T>::rsqrt(r2s);
    const T m = -y * i1, p = u2 * i2;
    const bool same = (y <= T(0)) || (y >= L);  // u1 u2 >= 0
    const T i1s = i1 * i1, i2s = i2 * i2, i12 = i1s * i2s;
    const T pm = p * m;
    const T S = fma(p, p, fma(m, m, pm));
    const T isum = i1 + i2;
    const T den = same ? (p + m) * (T(1) + pm) : d2;
    const T rr = RMath<T>::rcp(den * isum);
    const T rden = rr * isum;  // 1/den
    const T Lsum = L * (u2 - y);  // L (u1 + u2)
    const T J1 = Lsum * i12 * (rr * den);
    const T J3 = J1 * (i1s + fma(i1, i2, i2s)) * T(1.0 / 3.0);
    const T g = Lsum * i12 * rden;
    const T J0 = same ? g * (T(1) + pm) : (p - m) * rden;
    const T Wt = same ? fma((r1s + u2 * u2) * i12 * rden, p + m, i1s + i2s) : (T(3) - S) * rden;
    const T J2 = J0 * Wt * T(1.0 / 3.0);
    const T J4 = J0 * S * T(1.0 / 3.0);

    const T A0 = fma(T(3) * a2, J2, T(2) * J0);
    const T A1 = fma(T(3) * a2, J3, T(2) * J1);
    const T Rb = Rpx * bt[0] + Rpy * bt[1] + Rpz * bt[2];
    const T Rw = Rpx * k.w[0] + Rpy * k.w[1] + Rpz * k.w[2];
    const T qR = Rpx * q[0] + Rpy * q[1] + Rpz * q[2];
    const T c1tb = c1 * k.tb;
    const T c3qR = T(3) * c2 * qR;
    const T cRxb = -c1tb * A0;
    const T cq = fma(-c1tb, A1, c2 * fma(J1, k.tb, -J0 * Rb));
    const T cRp = fma(c3qR, fma(J2, Rb, -J3 * k.tb), -c2 * J0 * k.qb);
    const T ct = fma(-c1, fma(A0, Rw, A1 * k.qb), fma(c2 * J1, k.qb, c3qR * fma(J4, k.tb, -J3 * Rb)));
    const T cb = c2 * qR * (A0 - J0);
    // Rp x b
    const T Xx = Rpy * b[2] - Rpz * b[1];
    const T Xy = Rpz * b[0] - Rpx * b[2];
    const T Xz = Rpx * b[1] - Rpy * b[0];
    s[0] = fma(cRxb, Xx, fma(cq, q[0], fma(cRp, Rpx, fma(ct, t[0], fma(cb, bt[0], s[0])))));
    s[1] = fma(cRxb, Xy, fma(cq, q[1], fma(cRp, Rpy, fma(ct, t[1], fma(cb, bt[1], s[1])))));
    s[2] = fma(cRxb, Xz, fma(cq, q[2], fma(cRp, Rpz, fma(ct, t[2], fma(cb, bt[2], s[2])))));
}

// Accumulate (sigma b') of one source at one field point, given R0 = x - x1.
template <typename T>
__device__ __forceinline__ void seg_sigma_b(T R0x, T R0y, T R0z, const T t[3], T L, const T b[3],
                                            const T q[3], const T bt[3], const PairK<T>& k, T a2, T c1,
                                            T c2, T s[3])
{
    PairGeom<T> G;
    pair_geom(R0x, R0y, R0z, t, L, a2, G);
    seg_sigma_b_geom(G, t, L, b, q, bt, k, a2, c1, c2, s);
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
