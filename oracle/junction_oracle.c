/*
 * junction_oracle.c -- plain FP64 CPU oracle of the burst with junctions and
 * thermally activated junction breaking (Sec. 2.2).
 *
 * TEST INFRASTRUCTURE, like the rest of this library: only the test suite,
 * the smoke check and the CPU baseline of the benchmark may load it.  It
 * shares no code with the CUDA path.
 *
 * The paper's mobile segments form junctions where they meet sessile
 * segments; a junction pins the mobile line there and breaks after
 * t_b = f a (Eq. 2.2), f uniform on [0,1), a the maximum breaking time.
 * When every mobile line is held, the configuration is stuck and nothing
 * happens until the next junction breaks.  Readings taken here (the paper
 * leaves them to its DD library):
 *   - sessile segments are the segments whose two nodes are pinned; a free
 *     node p forms a junction with the sessile segment s of another loop
 *     when its distance to s is below the capture radius r_c; among several,
 *     the lowest segment index wins;
 *   - a held node does not move (velocity 0) until its junction breaks;
 *   - a node does not form a junction again with the sessile loop it last
 *     broke away from;
 *   - f of the k-th junction of node p (k = 0, 1, ...) is the top 53 bits of
 *     SplitMix64 (Vigna) output k+1 of the stream seeded with
 *     seed ^ (p * 0xD1B54A32D192ED03), times 2^-53;
 *   - stuck: some junction is held and no free mobile node moved more than
 *     stuck_disp in the step.  The DD clock then jumps to the earliest break
 *     time.  Over the jump the network is frozen: Lp = 0 and rho keeps the
 *     value sampled in the step.
 * One step from positions x_i at DD time t_i:
 *   1. forces and glide velocities at x_i (pinned nodes 0);
 *   2. for every free node: release its junction if its break time is <= t_i;
 *      if it holds none, look for a capture; if it holds one, zero its
 *      velocity;
 *   3. sample Lp and rho at (x_i, v_i), weight dt; Euler step;
 *   4. t_{i+1} = t_i + dt, or the earliest break time if stuck and later.
 */
#include "ptadd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* SplitMix64 output function (Vigna): the state advances by the golden
 * ratio increment and each output is this mix of the new state. */
uint64_t orc_splitmix64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double orc_junction_fraction(uint64_t seed, int64_t node, int64_t k)
{
    const uint64_t s = seed ^ ((uint64_t)node * 0xD1B54A32D192ED03ull);
    const uint64_t z = orc_splitmix64_mix(s + (uint64_t)(k + 1) * 0x9E3779B97F4A7C15ull);
    return (double)(z >> 11) * 0x1.0p-53;
}

/* squared distance from x to the segment x1 -> x2 (closest point clamped to
 * the segment), no fused operations */
double orc_point_segment_dist2(const double x[3], const double x1[3], const double x2[3])
{
    double e[3], w[3];
    for (int c = 0; c < 3; ++c) {
        e[c] = x2[c] - x1[c];
        w[c] = x[c] - x1[c];
    }
    const double ee = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
    double u = 0.0;
    if (ee > 0.0) {
        u = (w[0] * e[0] + w[1] * e[1] + w[2] * e[2]) / ee;
        if (u < 0.0) u = 0.0;
        if (u > 1.0) u = 1.0;
    }
    double d2 = 0.0;
    for (int c = 0; c < 3; ++c) {
        const double r = w[c] - u * e[c];
        d2 += r * r;
    }
    return d2;
}

int orc_burst_junctions(const double mat[5], int64_t n_nodes, const double* xyz, int64_t n_loops,
                        const int64_t* loop_off, const double* burgers, const double* normal,
                        const uint8_t* pinned, double volume, const double sig_app[6], int interactions,
                        int64_t n_steps, double dt, const double jpar[3], uint64_t seed, int32_t* jseg,
                        int32_t* jlast, int32_t* jcount, double* jbreak, double clock[2], int64_t counts[3],
                        double* xyz_out, double Lp_avg[9], double* rho_avg, double* S_t_out)
{
    const double rc2 = jpar[0] * jpar[0], a = jpar[1], stuck = jpar[2];
    const size_t n3 = (size_t)(3 * (n_nodes > 0 ? n_nodes : 1));
    double* x = (double*)malloc(sizeof(double) * n3);
    double* F = (double*)malloc(sizeof(double) * n3);
    double* v = (double*)malloc(sizeof(double) * n3);
    int64_t* loop_of = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_nodes > 0 ? n_nodes : 1));
    int64_t* nxt = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_nodes > 0 ? n_nodes : 1));
    memcpy(x, xyz, sizeof(double) * (size_t)(3 * n_nodes));
    for (int64_t k = 0; k < n_loops; ++k)
        for (int64_t i = loop_off[k]; i < loop_off[k + 1]; ++i) {
            loop_of[i] = k;
            nxt[i] = (i + 1 < loop_off[k + 1]) ? i + 1 : loop_off[k];
        }
    double S_Lp[9] = {0}, S_rho = 0.0, S_t = 0.0;
    int status = 0;
    for (int64_t s = 0; s < n_steps; ++s) {
        const double t = clock[0];
        orc_nodal_forces(mat, n_nodes, x, n_loops, loop_off, burgers, pinned, sig_app, interactions, 1, F);
        orc_velocities(mat, n_nodes, x, n_loops, loop_off, normal, pinned, F, v);
        double vmax2 = 0.0, tmin = INFINITY;
        int64_t held = 0;
        for (int64_t p = 0; p < n_nodes; ++p) {
            if (pinned && pinned[p]) continue;
            if (jseg[p] >= 0 && jbreak[p] <= t) {
                jlast[p] = (int32_t)loop_of[jseg[p]];
                jseg[p] = -1;
                counts[1] += 1;
            }
            if (jseg[p] < 0) {
                for (int64_t q = 0; q < n_nodes; ++q) {
                    if (!(pinned && pinned[q] && pinned[nxt[q]])) continue;  /* not sessile */
                    if (loop_of[q] == loop_of[p] || loop_of[q] == jlast[p]) continue;
                    if (orc_point_segment_dist2(x + 3 * p, x + 3 * q, x + 3 * nxt[q]) < rc2) {
                        jseg[p] = (int32_t)q;
                        jbreak[p] = t + a * orc_junction_fraction(seed, p, jcount[p]);
                        jcount[p] += 1;
                        counts[0] += 1;
                        break;
                    }
                }
            }
            if (jseg[p] >= 0) {
                v[3 * p] = v[3 * p + 1] = v[3 * p + 2] = 0.0;
                held += 1;
                if (jbreak[p] < tmin) tmin = jbreak[p];
            } else {
                const double v2 = v[3 * p] * v[3 * p] + v[3 * p + 1] * v[3 * p + 1] + v[3 * p + 2] * v[3 * p + 2];
                if (v2 > vmax2) vmax2 = v2;
            }
        }
        double Lp[9], rho;
        orc_lp_rho(n_nodes, x, n_loops, loop_off, burgers, v, volume, Lp, &rho);
        for (int m = 0; m < 9; ++m) S_Lp[m] += Lp[m] * dt;
        S_rho += rho * dt;
        S_t += dt;
        for (int m = 0; m < 9; ++m)
            if (!isfinite(Lp[m])) status = -1;
        for (size_t m = 0; m < (size_t)(3 * n_nodes); ++m) x[m] += v[m] * dt;
        double t1 = t + dt;
        if (held > 0 && sqrt(vmax2) * dt < stuck && tmin > t1) {
            const double jump = tmin - t1;
            S_rho += rho * jump;
            S_t += jump;
            clock[1] += jump;
            counts[2] += 1;
            t1 = tmin;
        }
        clock[0] = t1;
    }
    for (int m = 0; m < 9; ++m) Lp_avg[m] = (S_t > 0.0) ? S_Lp[m] / S_t : 0.0;
    *rho_avg = (S_t > 0.0) ? S_rho / S_t : 0.0;
    *S_t_out = S_t;
    if (xyz_out) memcpy(xyz_out, x, sizeof(double) * (size_t)(3 * n_nodes));
    free(x);
    free(F);
    free(v);
    free(loop_of);
    free(nxt);
    return status;
}
