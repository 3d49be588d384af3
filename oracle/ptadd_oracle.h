/*
 * ptadd_oracle.h -- plain FP64 CPU oracle of the discrete-dislocation burst.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * Everything is SI (m, Pa, s, N) and double precision.  Stress tensors are
 * Voigt 6-vectors in the order xx, yy, zz, yz, xz, xy.
 *
 * Material vector mat[5] = { mu, nu, b (unused here), a (core width), B (drag) }.
 *
 * Network arguments (every function that takes a network):
 *   n_nodes, xyz[n_nodes*3]         node positions
 *   n_loops, loop_off[n_loops+1]    loop k owns nodes [loop_off[k], loop_off[k+1]);
 *                                   segment i runs from node i to the next node of
 *                                   its loop (wrapping), line sense = node order
 *   burgers[n_loops*3]              Burgers vector of each loop (m)
 *   normal[n_loops*3]               unit glide normal of each loop
 *   pinned[n_nodes] (or NULL)       1 = node never moves
 *
 * Parity status: every function here is pinned by tests against closed forms,
 * invariants or brute force (see the test suite); none is "parity unpinned".
 */
#ifndef PTADD_ORACLE_H
#define PTADD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* 4-point Gauss-Legendre rule on [0,1] used for the force integral (Sec. 2.1). */
void orc_gauss4(double xi[4], double w[4]);

/* Nonsingular stress of one straight segment x1->x2 with Burgers vector bv at
 * the field point x: the closed-form line integral of the regularised
 * (R -> R_a = sqrt(R.R + a^2)) isotropic dislocation stress, Sec. 2.1 sigma = S R * alpha. */
void orc_seg_stress(const double mat[5], const double x1[3], const double x2[3],
                    const double bv[3], const double x[3], double sig[6]);

/* The same line integral by brute force: composite Gauss-Legendre in long
 * double with `panels` equal panels of `order` points, integrand written out
 * index by index from its definition.  Returns the full 3x3 tensor (row-major). */
int orc_seg_stress_quad(const double mat[5], const double x1[3], const double x2[3],
                        const double bv[3], const double x[3], int panels, int order,
                        double sig9[9]);

/* Third derivatives d_i d_j d_k R_a (27, i-major) and gradient of the
 * Laplacian d_i lap R_a (3) at separation R, core width a. */
void orc_ra_derivs(const double R[3], double a, double d3[27], double dlap[3]);

/* Total stress sigma_app + sum over all segments at n_pts field points. */
void orc_stress_at(const double mat[5], int64_t n_nodes, const double* xyz,
                   int64_t n_loops, const int64_t* loop_off, const double* burgers,
                   const double sig_app[6], int interactions,
                   int64_t n_pts, const double* pts, double* sig_out);

/* Nodal forces (N) at every node: F_a = sum_{s owns a} L_s sum_q w_q N_a(xi_q) f_q,
 * f_q = (sigma(x_q) b_s) x t_s.  interactions = 0 drops the segment fields
 * (sigma = sigma_app).  skip_pinned = 1 skips target segments whose two nodes
 * are both pinned (their nodes then get no contribution from them). */
void orc_nodal_forces(const double mat[5], int64_t n_nodes, const double* xyz,
                      int64_t n_loops, const int64_t* loop_off, const double* burgers,
                      const uint8_t* pinned, const double sig_app[6], int interactions,
                      int skip_pinned, double* F_out);

/* Forces at a subset of nodes only (sel[n_sel] node indices), same definition. */
void orc_nodal_forces_subset(const double mat[5], int64_t n_nodes, const double* xyz,
                             int64_t n_loops, const int64_t* loop_off, const double* burgers,
                             const double sig_app[6], int interactions,
                             int64_t n_sel, const int64_t* sel, double* F_out);

/* Lumped glide mobility: v_a = (I - n n) F_a / (B M_a), M_a = (L_prev + L_next)/2,
 * v_a = 0 for pinned nodes (Eq. 2.1 with the no-climb multiplier). */
void orc_velocities(const double mat[5], int64_t n_nodes, const double* xyz,
                    int64_t n_loops, const int64_t* loop_off, const double* normal,
                    const uint8_t* pinned, const double* F, double* v_out);

/* Consistent (Galerkin) glide mobility of Eq. 2.1: with linear shape
 * functions N_a the weak form gives, per loop, sum_b B M_ab w_b = (I - n n) F_a
 * with the mass matrix M_ab = int N_a N_b dl (a ring: M_aa = (L_prev + L_next)/3,
 * M_a,a+-1 = L/6 of the segment between them) and w_a = 0 at pinned nodes
 * (Dirichlet rows); solved per loop and component by Gaussian elimination with
 * partial pivoting.  A free node whose two segments have zero length is held
 * at rest, as in the lumped form.  The lumped form is its row-sum diagonal. */
void orc_velocities_consistent(const double mat[5], int64_t n_nodes, const double* xyz,
                               int64_t n_loops, const int64_t* loop_off, const double* normal,
                               const uint8_t* pinned, const double* F, double* v_out);

/* State functions: Lp = (1/V) sum_s L_s b_s (x) (t_s x vbar_s) (row-major 3x3,
 * Sec. 2.2 / Eq. 2.9) and rho = (1/V) sum_s L_s (Sec. 2.4). */
void orc_lp_rho(int64_t n_nodes, const double* xyz, int64_t n_loops,
                const int64_t* loop_off, const double* burgers, const double* v,
                double volume, double Lp[9], double* rho);

/* Polar dislocation velocity (Sec. 2.4, Eq. 2.11): the volume-averaged
 * dislocation velocity V = (1/|B|) sum_s vbar_s L_s A_s, with vbar_s the
 * segment's velocity (the mean of its nodal velocities, the same one that
 * gives Lp = alpha x V segment by segment) and one core area A_s = core_area
 * for every segment.  V[3]. */
void orc_polar_velocity(int64_t n_nodes, const double* xyz, int64_t n_loops,
                        const int64_t* loop_off, const double* v, double volume,
                        double core_area, double V[3]);

/* A burst of n_steps explicit Euler steps at fixed dt (Sec. 2.1), returning the
 * running averages R^Lp and R^rho of Eq. 2.5 over the step-start states,
 * and, if V_avg is not NULL, R^V of the polar velocity (Eq. 2.11, core area
 * core_area).  xyz_out (may alias nothing) receives the final positions;
 * Lp_trace and rho_trace (or NULL) receive the per-step samples.
 * consistent_mass: 0 the lumped mobility, 1 the consistent one.  Returns 0,
 * or -1 if a non-finite value appeared. */
int orc_burst(const double mat[5], int64_t n_nodes, const double* xyz,
              int64_t n_loops, const int64_t* loop_off, const double* burgers,
              const double* normal, const uint8_t* pinned, double volume,
              const double sig_app[6], int interactions, int64_t n_steps, double dt,
              double* xyz_out, double Lp_avg[9], double* rho_avg,
              double* Lp_trace, double* rho_trace, double core_area, double* V_avg,
              int consistent_mass);

/* ---- MLP (mlp_oracle.c): dims[0] -> ... -> dims[L], GELU on hidden layers,
 * linear output, parameters packed per layer as W (dims[l+1] x dims[l],
 * row-major) then b; loss = mean (y - t)^2 over batch and outputs. */
double orc_gelu(double z);
double orc_gelu_grad(double z);
int64_t orc_mlp_param_count(int L, const int* dims);
void orc_mlp_forward(int L, const int* dims, const double* params, int64_t B, const double* X, double* Y);
double orc_mlp_loss_grad(int L, const int* dims, const double* params, int64_t B, const double* X,
                         const double* T, double* grad);
void orc_adam_step(int64_t n, double* p, const double* g, double* m, double* v, int64_t t, double lr,
                   double b1, double b2, double eps);

/* Number of OpenMP threads the oracle uses (for reporting). */
int orc_num_threads(void);

/* Junctions and thermally activated breaking (Sec. 2.2; junction_oracle.c).
 * SplitMix64 output mix (Vigna) and the break fraction f of the k-th
 * junction of a node, in [0, 1). */
uint64_t orc_splitmix64_mix(uint64_t z);
double orc_junction_fraction(uint64_t seed, int64_t node, int64_t k);
/* squared distance from x to the segment x1 -> x2 */
double orc_point_segment_dist2(const double x[3], const double x1[3], const double x2[3]);
/* n_steps DD steps with junctions: jpar = {capture radius r_c (m), maximum
 * breaking time a (s), stuck displacement (m)}.  Junction state per node
 * (in/out): jseg (held sessile segment or -1), jlast (sessile loop last
 * broken from or -1), jcount (junctions formed), jbreak (break time, s);
 * clock = {DD time t, total time jumped} (s, in/out); counts = {formed,
 * broken, jumps} (in/out).  Lp_avg, rho_avg: Eq. 2.5 over the burst's
 * S_t = n_steps dt + the jumps (S_t_out).  Returns 0, or -1 on a
 * non-finite sample. */
int orc_burst_junctions(const double mat[5], int64_t n_nodes, const double* xyz, int64_t n_loops,
                        const int64_t* loop_off, const double* burgers, const double* normal,
                        const uint8_t* pinned, double volume, const double sig_app[6], int interactions,
                        int64_t n_steps, double dt, const double jpar[3], uint64_t seed, int32_t* jseg,
                        int32_t* jlast, int32_t* jcount, double* jbreak, double clock[2], int64_t counts[3],
                        double* xyz_out, double Lp_avg[9], double* rho_avg, double* S_t_out);

#ifdef __cplusplus
}
#endif
#endif
