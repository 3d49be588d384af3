/*
 * ptadd_oracle.c -- plain FP64 CPU oracle of the discrete-dislocation burst.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library; the product path
 * never does.  It shares no code with the CUDA path.
 *
 * What it computes, in the paper's order (Sec. 2.1, 2.2, 2.3, 2.4):
 *   1. sigma(x) = sigma_app + sum over all straight segments of the segment's
 *      stress at x.  The paper writes the loop stress as sigma = S R * alpha
 *      with S a linear differential operator acting on R = |x - x'| (Sec. 2.1,
 *      unnumbered).  For an isotropic medium that operator gives the line
 *      integral
 *        sigma_ab = mu/(8 pi)      int d_i lap(R) [b_m e_ima t_b + b_m e_imb t_a] dl'
 *                 + mu/(4 pi (1-nu)) int b_m e_imk t_k [d_i d_a d_b R - delta_ab d_i lap(R)] dl'
 *      with derivatives taken at the field point and R = x - x'.  The
 *      nonsingular form replaces |R| by R_a = sqrt(R.R + a^2) (core width a).
 *   2. Peach-Koehler force per length f = (sigma b) x t (Sec. 2.1).
 *   3. Nodal forces with linear shape functions, 4-point Gauss-Legendre.
 *   4. Glide mobility: the Galerkin problem Eq. 2.1 in its lumped form (the
 *      default) or with its consistent mass matrix, the no-climb multiplier
 *      read as projection onto the loop's glide plane.
 *   5. Explicit Euler x_p(t + dt) = x_p(t) + w_p dt (Sec. 2.1).
 *   6. The running time average R^Lambda of Eq. 2.5 for Lambda = Lp (the
 *      volume-averaged segment plastic distortion rate of Sec. 2.2) and
 *      Lambda = rho (total line length per volume, Sec. 2.4).
 *
 * Step 1 is evaluated analytically: along a straight segment every term of
 * the integrand reduces to int u^k (u^2 + d^2)^(-m/2) du with d^2 = |R_perp|^2
 * + a^2, all elementary.  Endpoint differences of those antiderivatives are
 * formed without the cancellation that occurs far away or near the
 * extension of the source line (see line_integrals()).  The brute-force
 * quadrature orc_seg_stress_quad() integrates the same integrand written
 * out index by index; tests compare the two.
 */
#include "ptadd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ---------------------------------------------------------------- Gauss */
/* Textbook 4-point Gauss-Legendre abscissae +-0.33998..., +-0.86113... and
 * weights on [-1,1], mapped to [0,1]. */
static const double GL4_Z[4] = {-0.8611363115940526, -0.3399810435848563,
                                0.3399810435848563, 0.8611363115940526};
static const double GL4_W[4] = {0.3478548451374538, 0.6521451548625461,
                                0.6521451548625461, 0.3478548451374538};

void orc_gauss4(double xi[4], double w[4])
{
    for (int q = 0; q < 4; ++q) {
        xi[q] = 0.5 * (1.0 + GL4_Z[q]);
        w[q] = 0.5 * GL4_W[q];
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------- small vectors */
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double* a, const double* b, double* c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Voigt index pairs: xx, yy, zz, yz, xz, xy */
static const int VA[6] = {0, 1, 2, 1, 0, 0};
static const int VB[6] = {0, 1, 2, 2, 2, 1};

/* ------------------------------------------- analytic line integrals
 * J[0] = int u^0 rho^-3, J[1] = int u rho^-3, J[2] = int rho^-5,
 * J[3] = int u rho^-5,   J[4] = int u^2 rho^-5,   over u in [u1, u2],
 * rho^2 = u^2 + d2, u2 - u1 = L > 0.
 *
 * Antiderivatives:  int rho^-3 = u/(d2 rho),  int u rho^-3 = -1/rho,
 *   int rho^-5 = u(2u^2+3d2)/(3 d2^2 rho^3),  int u rho^-5 = -1/(3 rho^3),
 *   int u^2 rho^-5 = u^3/(3 d2 rho^3).
 * The odd antiderivatives F tend to constants c as u -> +inf; for u >= 0 they
 * are written F(u) = c - T(u) with the tails
 *   T03 = 1/(rho (rho+u)),  T05 = (u + 2 rho)/(3 rho^3 (rho+u)^2),
 *   T25 = (rho^2 + rho u + u^2)/(3 rho^3 (rho+u)),
 * which carry no 1/d2 factor.  When both ends lie on one side of the foot of
 * the perpendicular, the difference is taken between tails; when the foot
 * lies inside the segment, the two odd terms add and the direct form is
 * exact.  The even antiderivatives go through rho2 - rho1 = L (u1+u2)/(rho1+rho2). */
static double tail03(double w, double r) { return 1.0 / (r * (r + w)); }
static double tail05(double w, double r) { return (w + 2.0 * r) / (3.0 * r * r * r * (r + w) * (r + w)); }
static double tail25(double w, double r) { return (r * r + r * w + w * w) / (3.0 * r * r * r * (r + w)); }

static void line_integrals(double u1, double u2, double L, double d2, double J[5])
{
    const double r1 = sqrt(u1 * u1 + d2), r2 = sqrt(u2 * u2 + d2);
    const double dr = L * (u1 + u2) / (r1 + r2); /* rho2 - rho1 */
    const double r1c = r1 * r1 * r1, r2c = r2 * r2 * r2;
    J[1] = dr / (r1 * r2);
    J[3] = dr * (r1 * r1 + r1 * r2 + r2 * r2) / (3.0 * r1c * r2c);
    if (u1 >= 0.0) {
        J[0] = tail03(u1, r1) - tail03(u2, r2);
        J[2] = tail05(u1, r1) - tail05(u2, r2);
        J[4] = tail25(u1, r1) - tail25(u2, r2);
    } else if (u2 <= 0.0) {
        J[0] = tail03(-u2, r2) - tail03(-u1, r1);
        J[2] = tail05(-u2, r2) - tail05(-u1, r1);
        J[4] = tail25(-u2, r2) - tail25(-u1, r1);
    } else {
        J[0] = u2 / (d2 * r2) - u1 / (d2 * r1);
        J[2] = u2 * (2.0 * u2 * u2 + 3.0 * d2) / (3.0 * d2 * d2 * r2c)
             - u1 * (2.0 * u1 * u1 + 3.0 * d2) / (3.0 * d2 * d2 * r1c);
        J[4] = u2 * u2 * u2 / (3.0 * d2 * r2c) - u1 * u1 * u1 / (3.0 * d2 * r1c);
    }
}

/* ----------------------------------------------- one segment, analytic */
void orc_seg_stress(const double mat[5], const double x1[3], const double x2[3],
                    const double bv[3], const double x[3], double sig[6])
{
    const double mu = mat[0], nu = mat[1], a = mat[3];
    const double a2 = a * a;
    double dx[3] = {x2[0] - x1[0], x2[1] - x1[1], x2[2] - x1[2]};
    const double L = sqrt(dot3(dx, dx));
    for (int c = 0; c < 6; ++c) sig[c] = 0.0;
    if (!(L > 0.0)) return;
    double t[3] = {dx[0] / L, dx[1] / L, dx[2] / L};

    /* R(u) = x - x' = Rp - u t, u = s - y, s in [0, L] the arc length from x1 */
    double R0[3] = {x[0] - x1[0], x[1] - x1[1], x[2] - x1[2]};
    const double y = dot3(R0, t);
    double Rp[3] = {R0[0] - y * t[0], R0[1] - y * t[1], R0[2] - y * t[2]};
    const double d2 = dot3(Rp, Rp) + a2;
    double J[5];
    line_integrals(-y, L - y, L, d2, J);

    /* term 1: the vector g = grad(lap R_a) x b = -(2/rho^3 + 3a^2/rho^5)(R x b),
     * R x b = Rp x b + u (b x t);  term 2 uses q = b x t, with q.R = q.Rp. */
    double q[3], Rxb[3];
    cross3(bv, t, q);
    cross3(Rp, bv, Rxb);
    const double qR = dot3(q, Rp);
    const double A0 = 2.0 * J[0] + 3.0 * a2 * J[2];
    const double A1 = 2.0 * J[1] + 3.0 * a2 * J[3];
    double G[3];
    for (int i = 0; i < 3; ++i) G[i] = -(A0 * Rxb[i] + A1 * q[i]);

    const double c1 = mu / (8.0 * ORC_PI);
    const double c2 = mu / (4.0 * ORC_PI * (1.0 - nu));
    for (int c = 0; c < 6; ++c) {
        const int al = VA[c], be = VB[c];
        const double dab = (al == be) ? 1.0 : 0.0;
        const double term1 = G[al] * t[be] + G[be] * t[al];
        const double term2 = -(q[al] * Rp[be] + q[be] * Rp[al]) * J[0]
                           + (q[al] * t[be] + q[be] * t[al]) * J[1]
                           + dab * qR * (J[0] + 3.0 * a2 * J[2])
                           + 3.0 * qR * (Rp[al] * Rp[be] * J[2]
                                         - (Rp[al] * t[be] + t[al] * Rp[be]) * J[3]
                                         + t[al] * t[be] * J[4]);
        sig[c] = c1 * term1 + c2 * term2;
    }
}

/* ----------------------------------------- one segment, brute force */
static int levi(int i, int j, int k)
{
    if (i == j || j == k || i == k) return 0;
    /* even permutations of (0,1,2) */
    if ((i == 0 && j == 1 && k == 2) || (i == 1 && j == 2 && k == 0) || (i == 2 && j == 0 && k == 1))
        return 1;
    return -1;
}

/* Gauss-Legendre nodes/weights on [-1,1] by Newton iteration on the
 * three-term Legendre recurrence (long double). */
static void gauss_legendre(int n, long double* z, long double* w)
{
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int i = 0; i < n; ++i) {
        long double x = cosl(pi * ((long double)i + 0.75L) / ((long double)n + 0.5L));
        long double dp = 0.0L;
        for (int it = 0; it < 200; ++it) {
            long double p0 = 1.0L, p1 = x;
            for (int k = 1; k < n; ++k) {
                long double p2 = ((2.0L * k + 1.0L) * x * p1 - (long double)k * p0) / (long double)(k + 1);
                p0 = p1;
                p1 = p2;
            }
            /* p1 = P_n(x), p0 = P_{n-1}(x) */
            dp = (long double)n * (x * p1 - p0) / (x * x - 1.0L);
            long double dx = p1 / dp;
            x -= dx;
            if (fabsl(dx) < 1e-30L) break;
        }
        z[i] = x;
        w[i] = 2.0L / ((1.0L - x * x) * dp * dp);
    }
}

static void ra_derivs_ld(const long double R[3], long double a, long double d3[27], long double dl[3])
{
    const long double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2] + a * a;
    const long double ra = sqrtl(r2);
    const long double i3 = 1.0L / (ra * r2), i5 = i3 / r2;
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            for (int k = 0; k < 3; ++k) {
                long double v = -(((i == j) ? R[k] : 0.0L) + ((j == k) ? R[i] : 0.0L) + ((i == k) ? R[j] : 0.0L)) * i3
                              + 3.0L * R[i] * R[j] * R[k] * i5;
                d3[(i * 3 + j) * 3 + k] = v;
            }
        }
        dl[i] = -2.0L * R[i] * i3 - 3.0L * a * a * R[i] * i5;
    }
}

void orc_ra_derivs(const double R[3], double a, double d3[27], double dlap[3])
{
    long double Rl[3] = {R[0], R[1], R[2]}, d3l[27], dll[3];
    ra_derivs_ld(Rl, (long double)a, d3l, dll);
    for (int i = 0; i < 27; ++i) d3[i] = (double)d3l[i];
    for (int i = 0; i < 3; ++i) dlap[i] = (double)dll[i];
}

int orc_seg_stress_quad(const double mat[5], const double x1[3], const double x2[3],
                        const double bv[3], const double x[3], int panels, int order,
                        double sig9[9])
{
    if (panels < 1 || order < 1 || order > 64) return -1;
    const long double mu = mat[0], nu = mat[1], a = mat[3];
    const long double pi = 3.141592653589793238462643383279502884L;
    long double z[64], w[64];
    gauss_legendre(order, z, w);
    long double d[3] = {(long double)x2[0] - x1[0], (long double)x2[1] - x1[1], (long double)x2[2] - x1[2]};
    const long double L = sqrtl(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    long double acc[9] = {0};
    if (L > 0.0L) {
        long double t[3] = {d[0] / L, d[1] / L, d[2] / L};
        long double b[3] = {bv[0], bv[1], bv[2]};
        const long double h = L / (long double)panels;
        const long double c1 = mu / (8.0L * pi), c2 = mu / (4.0L * pi * (1.0L - nu));
        for (int p = 0; p < panels; ++p) {
            for (int g = 0; g < order; ++g) {
                const long double s = h * ((long double)p + 0.5L * (1.0L + z[g]));
                const long double wt = 0.5L * h * w[g];
                long double R[3];
                for (int i = 0; i < 3; ++i) R[i] = (long double)x[i] - ((long double)x1[i] + s * t[i]);
                long double d3[27], dl[3];
                ra_derivs_ld(R, a, d3, dl);
                for (int al = 0; al < 3; ++al) {
                    for (int be = 0; be < 3; ++be) {
                        long double term1 = 0.0L, term2 = 0.0L;
                        for (int i = 0; i < 3; ++i)
                            for (int m = 0; m < 3; ++m)
                                term1 += dl[i] * (b[m] * levi(i, m, al) * t[be] + b[m] * levi(i, m, be) * t[al]);
                        for (int i = 0; i < 3; ++i)
                            for (int m = 0; m < 3; ++m)
                                for (int k = 0; k < 3; ++k) {
                                    const int e = levi(i, m, k);
                                    if (!e) continue;
                                    term2 += b[m] * e * t[k] * (d3[(i * 3 + al) * 3 + be] - ((al == be) ? dl[i] : 0.0L));
                                }
                        acc[al * 3 + be] += wt * (c1 * term1 + c2 * term2);
                    }
                }
            }
        }
    }
    for (int i = 0; i < 9; ++i) sig9[i] = (double)acc[i];
    return 0;
}

/* --------------------------------------------------------- networks */
/* next-node table: seg i runs i -> nxt[i]; prv[i] is the node before i. */
static void ring_tables(int64_t n_nodes, int64_t n_loops, const int64_t* off,
                        int64_t* nxt, int64_t* prv, int64_t* loop_of)
{
    for (int64_t k = 0; k < n_loops; ++k) {
        const int64_t b = off[k], e = off[k + 1];
        for (int64_t i = b; i < e; ++i) {
            nxt[i] = (i + 1 < e) ? i + 1 : b;
            prv[i] = (i > b) ? i - 1 : e - 1;
            if (loop_of) loop_of[i] = k;
        }
    }
    (void)n_nodes;
}

/* sigma at x from sigma_app plus (optionally) every segment */
static void total_stress(const double mat[5], int64_t n_nodes, const double* xyz,
                         const int64_t* nxt, const int64_t* loop_of, const double* burgers,
                         const double sig_app[6], int interactions, const double x[3], double sig[6])
{
    for (int c = 0; c < 6; ++c) sig[c] = sig_app[c];
    if (!interactions) return;
    double s[6];
    for (int64_t i = 0; i < n_nodes; ++i) {
        orc_seg_stress(mat, xyz + 3 * i, xyz + 3 * nxt[i], burgers + 3 * loop_of[i], x, s);
        for (int c = 0; c < 6; ++c) sig[c] += s[c];
    }
}

void orc_stress_at(const double mat[5], int64_t n_nodes, const double* xyz,
                   int64_t n_loops, const int64_t* loop_off, const double* burgers,
                   const double sig_app[6], int interactions,
                   int64_t n_pts, const double* pts, double* sig_out)
{
    int64_t* nxt = (int64_t*)malloc(sizeof(int64_t) * (size_t)(3 * (n_nodes > 0 ? n_nodes : 1)));
    int64_t *prv = nxt + n_nodes, *lo = prv + n_nodes;
    ring_tables(n_nodes, n_loops, loop_off, nxt, prv, lo);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < n_pts; ++p)
        total_stress(mat, n_nodes, xyz, nxt, lo, burgers, sig_app, interactions, pts + 3 * p, sig_out + 6 * p);
    free(nxt);
}

/* sigma (Voigt) times a vector */
static void sig_dot(const double s[6], const double v[3], double out[3])
{
    out[0] = s[0] * v[0] + s[5] * v[1] + s[4] * v[2];
    out[1] = s[5] * v[0] + s[1] * v[1] + s[3] * v[2];
    out[2] = s[4] * v[0] + s[3] * v[1] + s[2] * v[2];
}

/* contributions of target segment i -> j to its start node (Fs) and end node (Fe) */
static void segment_force(const double mat[5], int64_t n_nodes, const double* xyz,
                          const int64_t* nxt, const int64_t* lo, const double* burgers,
                          const double sig_app[6], int interactions, int64_t i,
                          double Fs[3], double Fe[3])
{
    double xi[4], w[4];
    orc_gauss4(xi, w);
    const double* xa = xyz + 3 * i;
    const double* xb = xyz + 3 * nxt[i];
    const double* b = burgers + 3 * lo[i];
    double dx[3] = {xb[0] - xa[0], xb[1] - xa[1], xb[2] - xa[2]};
    const double L = sqrt(dot3(dx, dx));
    for (int c = 0; c < 3; ++c) Fs[c] = Fe[c] = 0.0;
    if (!(L > 0.0)) return;
    double t[3] = {dx[0] / L, dx[1] / L, dx[2] / L};
    for (int q = 0; q < 4; ++q) {
        double xq[3] = {xa[0] + xi[q] * dx[0], xa[1] + xi[q] * dx[1], xa[2] + xi[q] * dx[2]};
        double sig[6], sb[3], f[3];
        total_stress(mat, n_nodes, xyz, nxt, lo, burgers, sig_app, interactions, xq, sig);
        sig_dot(sig, b, sb);
        cross3(sb, t, f); /* f = (sigma b) x t, Sec. 2.1 */
        for (int c = 0; c < 3; ++c) {
            Fs[c] += L * w[q] * (1.0 - xi[q]) * f[c];
            Fe[c] += L * w[q] * xi[q] * f[c];
        }
    }
}

void orc_nodal_forces(const double mat[5], int64_t n_nodes, const double* xyz,
                      int64_t n_loops, const int64_t* loop_off, const double* burgers,
                      const uint8_t* pinned, const double sig_app[6], int interactions,
                      int skip_pinned, double* F_out)
{
    int64_t* nxt = (int64_t*)malloc(sizeof(int64_t) * (size_t)(3 * (n_nodes > 0 ? n_nodes : 1)));
    int64_t *prv = nxt + n_nodes, *lo = prv + n_nodes;
    double* FsFe = (double*)calloc((size_t)(6 * (n_nodes > 0 ? n_nodes : 1)), sizeof(double));
    ring_tables(n_nodes, n_loops, loop_off, nxt, prv, lo);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n_nodes; ++i) {
        if (skip_pinned && pinned && pinned[i] && pinned[nxt[i]]) continue;
        segment_force(mat, n_nodes, xyz, nxt, lo, burgers, sig_app, interactions, i,
                      FsFe + 6 * i, FsFe + 6 * i + 3);
    }
    for (int64_t a = 0; a < n_nodes; ++a)
        for (int c = 0; c < 3; ++c) F_out[3 * a + c] = FsFe[6 * a + c] + FsFe[6 * prv[a] + 3 + c];
    free(FsFe);
    free(nxt);
}

void orc_nodal_forces_subset(const double mat[5], int64_t n_nodes, const double* xyz,
                             int64_t n_loops, const int64_t* loop_off, const double* burgers,
                             const double sig_app[6], int interactions,
                             int64_t n_sel, const int64_t* sel, double* F_out)
{
    int64_t* nxt = (int64_t*)malloc(sizeof(int64_t) * (size_t)(3 * (n_nodes > 0 ? n_nodes : 1)));
    int64_t *prv = nxt + n_nodes, *lo = prv + n_nodes;
    ring_tables(n_nodes, n_loops, loop_off, nxt, prv, lo);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < n_sel; ++k) {
        const int64_t a = sel[k];
        double Fs[3], Fe[3], Gs[3], Ge[3];
        segment_force(mat, n_nodes, xyz, nxt, lo, burgers, sig_app, interactions, a, Fs, Fe);
        segment_force(mat, n_nodes, xyz, nxt, lo, burgers, sig_app, interactions, prv[a], Gs, Ge);
        for (int c = 0; c < 3; ++c) F_out[3 * k + c] = Fs[c] + Ge[c];
    }
    free(nxt);
}

void orc_velocities(const double mat[5], int64_t n_nodes, const double* xyz,
                    int64_t n_loops, const int64_t* loop_off, const double* normal,
                    const uint8_t* pinned, const double* F, double* v_out)
{
    const double B = mat[4];
    for (int64_t k = 0; k < n_loops; ++k) {
        const int64_t b = loop_off[k], e = loop_off[k + 1];
        const double* n = normal + 3 * k;
        for (int64_t a = b; a < e; ++a) {
            const int64_t p = (a > b) ? a - 1 : e - 1;
            const int64_t nx = (a + 1 < e) ? a + 1 : b;
            double dp[3], dn[3];
            for (int c = 0; c < 3; ++c) {
                dp[c] = xyz[3 * a + c] - xyz[3 * p + c];
                dn[c] = xyz[3 * nx + c] - xyz[3 * a + c];
            }
            const double M = 0.5 * (sqrt(dot3(dp, dp)) + sqrt(dot3(dn, dn)));
            double* v = v_out + 3 * a;
            if ((pinned && pinned[a]) || !(M > 0.0)) {
                v[0] = v[1] = v[2] = 0.0;
                continue;
            }
            const double* Fa = F + 3 * a;
            const double nF = dot3(n, Fa);
            for (int c = 0; c < 3; ++c) v[c] = (Fa[c] - n[c] * nF) / (B * M);
        }
    }
}

/* Solve A x = rhs (m x m, row-major, 3 right-hand sides as rows of rhs[m][3])
 * by Gaussian elimination with partial pivoting; A and rhs are overwritten. */
static void solve_dense3(int64_t m, double* A, double* rhs)
{
    for (int64_t c = 0; c < m; ++c) {
        int64_t piv = c;
        for (int64_t r = c + 1; r < m; ++r)
            if (fabs(A[r * m + c]) > fabs(A[piv * m + c])) piv = r;
        if (piv != c) {
            for (int64_t k = 0; k < m; ++k) {
                const double t = A[c * m + k];
                A[c * m + k] = A[piv * m + k];
                A[piv * m + k] = t;
            }
            for (int e = 0; e < 3; ++e) {
                const double t = rhs[3 * c + e];
                rhs[3 * c + e] = rhs[3 * piv + e];
                rhs[3 * piv + e] = t;
            }
        }
        for (int64_t r = c + 1; r < m; ++r) {
            const double f = A[r * m + c] / A[c * m + c];
            if (f == 0.0) continue;
            for (int64_t k = c; k < m; ++k) A[r * m + k] -= f * A[c * m + k];
            for (int e = 0; e < 3; ++e) rhs[3 * r + e] -= f * rhs[3 * c + e];
        }
    }
    for (int64_t r = m - 1; r >= 0; --r) {
        for (int e = 0; e < 3; ++e) {
            double s = rhs[3 * r + e];
            for (int64_t k = r + 1; k < m; ++k) s -= A[r * m + k] * rhs[3 * k + e];
            rhs[3 * r + e] = s / A[r * m + r];
        }
    }
}

void orc_velocities_consistent(const double mat[5], int64_t n_nodes, const double* xyz,
                               int64_t n_loops, const int64_t* loop_off, const double* normal,
                               const uint8_t* pinned, const double* F, double* v_out)
{
    const double B = mat[4];
    for (int64_t k = 0; k < n_loops; ++k) {
        const int64_t b = loop_off[k], e = loop_off[k + 1], m = e - b;
        const double* n = normal + 3 * k;
        double* A = (double*)calloc((size_t)(m * m), sizeof(double));
        double* r = (double*)malloc(sizeof(double) * (size_t)(3 * m));
        /* assembly: int N_a N_b over segment a -> a+1 of length L gives L/3 on
         * its two diagonal entries and L/6 between them */
        for (int64_t i = 0; i < m; ++i) {
            const int64_t j = (i + 1 < m) ? i + 1 : 0;
            double d[3];
            for (int c = 0; c < 3; ++c) d[c] = xyz[3 * (b + j) + c] - xyz[3 * (b + i) + c];
            const double L = sqrt(dot3(d, d));
            A[i * m + i] += B * L / 3.0;
            A[j * m + j] += B * L / 3.0;
            A[i * m + j] += B * L / 6.0;
            A[j * m + i] += B * L / 6.0;
        }
        for (int64_t i = 0; i < m; ++i) {
            const double* Fa = F + 3 * (b + i);
            const double nF = dot3(n, Fa);
            const int held = (pinned && pinned[b + i]) || !(A[i * m + i] > 0.0);
            for (int c = 0; c < 3; ++c) r[3 * i + c] = held ? 0.0 : Fa[c] - n[c] * nF;
            if (held) { /* Dirichlet row: w_i = 0 */
                for (int64_t q = 0; q < m; ++q) A[i * m + q] = 0.0;
                A[i * m + i] = 1.0;
            }
        }
        solve_dense3(m, A, r);
        memcpy(v_out + 3 * b, r, sizeof(double) * (size_t)(3 * m));
        free(A);
        free(r);
    }
    (void)n_nodes;
}

void orc_lp_rho(int64_t n_nodes, const double* xyz, int64_t n_loops,
                const int64_t* loop_off, const double* burgers, const double* v,
                double volume, double Lp[9], double* rho)
{
    double acc[9] = {0}, len = 0.0;
    for (int64_t k = 0; k < n_loops; ++k) {
        const int64_t b = loop_off[k], e = loop_off[k + 1];
        const double* bv = burgers + 3 * k;
        for (int64_t i = b; i < e; ++i) {
            const int64_t j = (i + 1 < e) ? i + 1 : b;
            double dx[3], vb[3], c[3];
            for (int m = 0; m < 3; ++m) {
                dx[m] = xyz[3 * j + m] - xyz[3 * i + m];
                vb[m] = 0.5 * (v[3 * i + m] + v[3 * j + m]);
            }
            cross3(dx, vb, c); /* L (t x vbar) */
            for (int al = 0; al < 3; ++al)
                for (int be = 0; be < 3; ++be) acc[al * 3 + be] += bv[al] * c[be];
            len += sqrt(dot3(dx, dx));
        }
    }
    for (int m = 0; m < 9; ++m) Lp[m] = acc[m] / volume;
    *rho = len / volume;
    (void)n_nodes;
}

void orc_polar_velocity(int64_t n_nodes, const double* xyz, int64_t n_loops,
                        const int64_t* loop_off, const double* v, double volume,
                        double core_area, double V[3])
{
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t k = 0; k < n_loops; ++k) {
        const int64_t b = loop_off[k], e = loop_off[k + 1];
        for (int64_t i = b; i < e; ++i) {
            const int64_t j = (i + 1 < e) ? i + 1 : b;
            double dx[3];
            for (int m = 0; m < 3; ++m) dx[m] = xyz[3 * j + m] - xyz[3 * i + m];
            const double L = sqrt(dot3(dx, dx));
            for (int m = 0; m < 3; ++m) acc[m] += L * 0.5 * (v[3 * i + m] + v[3 * j + m]);
        }
    }
    for (int m = 0; m < 3; ++m) V[m] = core_area * acc[m] / volume;
    (void)n_nodes;
}

int orc_burst(const double mat[5], int64_t n_nodes, const double* xyz,
              int64_t n_loops, const int64_t* loop_off, const double* burgers,
              const double* normal, const uint8_t* pinned, double volume,
              const double sig_app[6], int interactions, int64_t n_steps, double dt,
              double* xyz_out, double Lp_avg[9], double* rho_avg,
              double* Lp_trace, double* rho_trace, double core_area, double* V_avg,
              int consistent_mass)
{
    const size_t n3 = (size_t)(3 * (n_nodes > 0 ? n_nodes : 1));
    double* x = (double*)malloc(sizeof(double) * n3);
    double* F = (double*)malloc(sizeof(double) * n3);
    double* v = (double*)malloc(sizeof(double) * n3);
    memcpy(x, xyz, sizeof(double) * (size_t)(3 * n_nodes));
    double S_Lp[9] = {0}, S_rho = 0.0, S_t = 0.0, S_V[3] = {0.0, 0.0, 0.0};
    int status = 0;
    for (int64_t s = 0; s < n_steps; ++s) {
        orc_nodal_forces(mat, n_nodes, x, n_loops, loop_off, burgers, pinned, sig_app,
                         interactions, 1, F);
        if (consistent_mass)
            orc_velocities_consistent(mat, n_nodes, x, n_loops, loop_off, normal, pinned, F, v);
        else
            orc_velocities(mat, n_nodes, x, n_loops, loop_off, normal, pinned, F, v);
        double Lp[9], rho;
        orc_lp_rho(n_nodes, x, n_loops, loop_off, burgers, v, volume, Lp, &rho);
        for (int m = 0; m < 9; ++m) S_Lp[m] += Lp[m] * dt;
        S_rho += rho * dt;
        S_t += dt;
        if (V_avg) {
            double V[3];
            orc_polar_velocity(n_nodes, x, n_loops, loop_off, v, volume, core_area, V);
            for (int m = 0; m < 3; ++m) S_V[m] += V[m] * dt;
        }
        if (Lp_trace) memcpy(Lp_trace + 9 * s, Lp, sizeof(Lp));
        if (rho_trace) rho_trace[s] = rho;
        for (int m = 0; m < 9; ++m)
            if (!isfinite(Lp[m])) status = -1;
        for (size_t m = 0; m < (size_t)(3 * n_nodes); ++m) x[m] += v[m] * dt;
    }
    for (int m = 0; m < 9; ++m) Lp_avg[m] = (S_t > 0.0) ? S_Lp[m] / S_t : 0.0;
    *rho_avg = (S_t > 0.0) ? S_rho / S_t : 0.0;
    if (V_avg)
        for (int m = 0; m < 3; ++m) V_avg[m] = (S_t > 0.0) ? S_V[m] / S_t : 0.0;
    if (xyz_out) memcpy(xyz_out, x, sizeof(double) * (size_t)(3 * n_nodes));
    free(x);
    free(F);
    free(v);
    return status;
}
