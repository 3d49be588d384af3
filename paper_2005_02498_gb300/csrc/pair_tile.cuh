// pair_tile.cuh -- one work tile of the O(N^2) pair stage: up to TPB target
// segments (one per thread) against a contiguous range of source segments,
// producing the two nodal-force parts (start node, end node) of every target.
//
// Used by the single-realisation kernels (one tile per block, grid-mapped)
// and by the batched persistent kernels (tiles pulled from a cost-sorted work
// queue).  Per target and Gauss point x_q the tile accumulates (sigma b') over
// its sources (seg_field.cuh), adds sigma_app b' if asked, then forms
//   F_start = sum_q w_q (1 - xi_q) (s_q x D),  F_end = sum_q w_q xi_q (s_q x D)
// with D = x_b - x_a (= L t): the Peach-Koehler force (Sec. 2.1) integrated
// against the linear shape functions with the 4-point Gauss rule.
#pragma once

#include <cuda_runtime.h>

#include "ptadd_internal.cuh"
#include "seg_field.cuh"

namespace ptadd {

struct TileArgs {
    const double* pos;      // SoA positions, stride n
    int64_t n;
    const int32_t* nxt;
    const double* src;      // FP64 source records
    const float* src32;     // FP32 source records (mixed)
    const int32_t* tgt;     // target segment list
    int64_t t_begin;        // first entry of tgt for thread 0
    int64_t t_count;        // targets in this tile (<= blockDim.x)
    int64_t js, je;         // source range [js, je)
    int add_app;            // add sigma_app b' (exactly one tile per target does)
    double sh[6];           // sigma_app / mu
    double origin[3];       // FP32 split origin (mixed)
    double* fp;             // output parts: fp[c * fp_stride + (seg - node_base)], c = 0..5
    int64_t fp_stride;
    int64_t node_base;
    unsigned long long* near_count;
};

__device__ __forceinline__ void tile_store(const TileArgs& a, int64_t seg, double Dx, double Dy, double Dz,
                                           const double bt[3], double acc[4][3])
{
    if (a.add_app) {
        const double* s = a.sh;
        const double sb0 = s[0] * bt[0] + s[5] * bt[1] + s[4] * bt[2];
        const double sb1 = s[5] * bt[0] + s[1] * bt[1] + s[3] * bt[2];
        const double sb2 = s[4] * bt[0] + s[3] * bt[1] + s[2] * bt[2];
#pragma unroll
        for (int qp = 0; qp < 4; ++qp) {
            acc[qp][0] += sb0;
            acc[qp][1] += sb1;
            acc[qp][2] += sb2;
        }
    }
    double Fs[3] = {0, 0, 0}, Fe[3] = {0, 0, 0};
#pragma unroll
    for (int qp = 0; qp < 4; ++qp) {
        const double fx = acc[qp][1] * Dz - acc[qp][2] * Dy;
        const double fy = acc[qp][2] * Dx - acc[qp][0] * Dz;
        const double fz = acc[qp][0] * Dy - acc[qp][1] * Dx;
        const double we = gl4_w(qp) * gl4_xi(qp), ws = gl4_w(qp) - we;
        Fs[0] = fma(ws, fx, Fs[0]); Fs[1] = fma(ws, fy, Fs[1]); Fs[2] = fma(ws, fz, Fs[2]);
        Fe[0] = fma(we, fx, Fe[0]); Fe[1] = fma(we, fy, Fe[1]); Fe[2] = fma(we, fz, Fe[2]);
    }
    double* fp = a.fp + (seg - a.node_base);
    const int64_t st = a.fp_stride;
    fp[0 * st] = Fs[0];
    fp[1 * st] = Fs[1];
    fp[2 * st] = Fs[2];
    fp[3 * st] = Fe[0];
    fp[4 * st] = Fe[1];
    fp[5 * st] = Fe[2];
}

// ------------------------------------------------------------------ FP64
// smem: TILE * SRC_STRIDE doubles (as double2).
template <int TILE>
__device__ __forceinline__ void pair_tile_fp64(const TileArgs& a, const Consts& c, double2* tile)
{
    const int64_t n = a.n;
    const bool active = threadIdx.x < a.t_count;
    const int64_t seg = active ? a.tgt[a.t_begin + threadIdx.x] : a.tgt[a.t_begin];
    const double* tr = a.src + (int64_t)SRC_STRIDE * seg;
    const int64_t sb = a.nxt[seg];
    const double xa = a.pos[seg], ya = a.pos[n + seg], za = a.pos[2 * n + seg];
    const double Dx = a.pos[sb] - xa, Dy = a.pos[n + sb] - ya, Dz = a.pos[2 * n + sb] - za;
    const double bt[3] = {tr[8], tr[9], tr[10]};
    double xq[4][3];
#pragma unroll
    for (int qp = 0; qp < 4; ++qp) {
        // x_q = x_a + xi_q (x_b - x_a), rounded as written (no contraction)
        const double xi = gl4_xi(qp);
        xq[qp][0] = __dadd_rn(xa, __dmul_rn(xi, Dx));
        xq[qp][1] = __dadd_rn(ya, __dmul_rn(xi, Dy));
        xq[qp][2] = __dadd_rn(za, __dmul_rn(xi, Dz));
    }
    double acc[4][3];
#pragma unroll
    for (int qp = 0; qp < 4; ++qp) acc[qp][0] = acc[qp][1] = acc[qp][2] = 0.0;

    for (int64_t j0 = a.js; j0 < a.je; j0 += TILE) {
        const int cnt = (int)min((int64_t)TILE, a.je - j0);
        __syncthreads();
        const double2* g = reinterpret_cast<const double2*>(a.src + (int64_t)SRC_STRIDE * j0);
        for (int e = threadIdx.x; e < cnt * (SRC_STRIDE / 2); e += blockDim.x) tile[e] = g[e];
        __syncthreads();
        for (int jj = 0; jj < cnt; ++jj) {
            const double* r = reinterpret_cast<const double*>(tile + jj * (SRC_STRIDE / 2));
            const double L = r[3];
            if (!(L > 0.0)) continue;  // zero-length source: no field (uniform branch)
            const double x1[3] = {r[0], r[1], r[2]};
            const double t[3] = {r[4], r[5], r[6]};
            const double b[3] = {r[8], r[9], r[10]};
            const double q[3] = {r[12], r[13], r[14]};
            PairK<double> k;
            pair_constants(t, b, q, bt, k);
#pragma unroll
            for (int qp = 0; qp < 4; ++qp)
                seg_sigma_b(xq[qp][0] - x1[0], xq[qp][1] - x1[1], xq[qp][2] - x1[2], t, L, b, q, bt, k, c.a2,
                            c.c1, c.c2, acc[qp]);
        }
    }
    if (active) tile_store(a, seg, Dx, Dy, Dz, bt, acc);
}

// ----------------------------------------------------------------- mixed
// Every (Gauss point, source) pair is first located in FP32 from hi/lo-split
// coordinates; if the point lies within 10 a of the source segment the pair
// is evaluated in FP64 from the FP64 records, otherwise in FP32.  Per Gauss
// point the contributions are summed in FP32 with Kahan compensation (the
// FP64 near-field values enter as hi + lo floats); the compensated sums go to
// FP64 before the PK force and the nodal assembly.
__device__ __forceinline__ void kahan_add(float& s, float& c, float v)
{
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// smem: TILE * SRC32_STRIDE floats (as float4).
template <int TILE>
__device__ __forceinline__ void pair_tile_mixed(const TileArgs& a, const Consts& c, float near2, float4* tile)
{
    const int64_t n = a.n;
    const bool active = threadIdx.x < a.t_count;
    const int64_t seg = active ? a.tgt[a.t_begin + threadIdx.x] : a.tgt[a.t_begin];
    const double* tr = a.src + (int64_t)SRC_STRIDE * seg;
    const int64_t sb = a.nxt[seg];
    const double xa = a.pos[seg], ya = a.pos[n + seg], za = a.pos[2 * n + seg];
    const double Dx = a.pos[sb] - xa, Dy = a.pos[n + sb] - ya, Dz = a.pos[2 * n + sb] - za;
    const double bt[3] = {tr[8], tr[9], tr[10]};
    const float btf[3] = {(float)bt[0], (float)bt[1], (float)bt[2]};
    float xh[4][3], xl[4][3];
#pragma unroll
    for (int qp = 0; qp < 4; ++qp) {
        const double xi = gl4_xi(qp);
        const double q0 = __dadd_rn(xa, __dmul_rn(xi, Dx)) - a.origin[0];
        const double q1 = __dadd_rn(ya, __dmul_rn(xi, Dy)) - a.origin[1];
        const double q2 = __dadd_rn(za, __dmul_rn(xi, Dz)) - a.origin[2];
        const double h0 = rint(q0), h1 = rint(q1), h2 = rint(q2);
        xh[qp][0] = (float)h0; xh[qp][1] = (float)h1; xh[qp][2] = (float)h2;
        xl[qp][0] = (float)(q0 - h0); xl[qp][1] = (float)(q1 - h1); xl[qp][2] = (float)(q2 - h2);
    }
    float sh[4][3], sc[4][3];
#pragma unroll
    for (int qp = 0; qp < 4; ++qp)
#pragma unroll
        for (int e = 0; e < 3; ++e) sh[qp][e] = sc[qp][e] = 0.0f;
    const float a2f = (float)c.a2, c1f = (float)c.c1, c2f = (float)c.c2;
    unsigned near_here = 0;

    for (int64_t j0 = a.js; j0 < a.je; j0 += TILE) {
        const int cnt = (int)min((int64_t)TILE, a.je - j0);
        __syncthreads();
        const float4* g = reinterpret_cast<const float4*>(a.src32 + (int64_t)SRC32_STRIDE * j0);
        for (int e = threadIdx.x; e < cnt * (SRC32_STRIDE / 4); e += blockDim.x) tile[e] = g[e];
        __syncthreads();
        for (int jj = 0; jj < cnt; ++jj) {
            const float* r = reinterpret_cast<const float*>(tile + jj * (SRC32_STRIDE / 4));
            const float L = r[6];
            if (!(L > 0.0f)) continue;  // zero-length source (uniform branch)
            const float h1[3] = {r[0], r[1], r[2]}, l1[3] = {r[3], r[4], r[5]};
            const float t[3] = {r[7], r[8], r[9]};
            const float b[3] = {r[10], r[11], r[12]};
            const float q[3] = {r[13], r[14], r[15]};
            PairK<float> k;
            pair_constants(t, b, q, btf, k);
#pragma unroll
            for (int qp = 0; qp < 4; ++qp) {
                const float R0x = (xh[qp][0] - h1[0]) + (xl[qp][0] - l1[0]);
                const float R0y = (xh[qp][1] - h1[1]) + (xl[qp][1] - l1[1]);
                const float R0z = (xh[qp][2] - h1[2]) + (xl[qp][2] - l1[2]);
                PairGeom<float> G;
                pair_geom(R0x, R0y, R0z, t, L, a2f, G);
                // squared point-to-segment distance (+ a^2)
                const float dd = G.y < 0.0f ? G.r1s : (G.y > L ? G.r2s : G.d2);
                if (dd >= near2) {
                    float v[3] = {0.0f, 0.0f, 0.0f};
                    seg_sigma_b_geom(G, t, L, b, q, btf, k, a2f, c1f, c2f, v);
                    kahan_add(sh[qp][0], sc[qp][0], v[0]);
                    kahan_add(sh[qp][1], sc[qp][1], v[1]);
                    kahan_add(sh[qp][2], sc[qp][2], v[2]);
                } else {
                    // near field: FP64 from the FP64 records
                    ++near_here;
                    const double* r64 = a.src + (int64_t)SRC_STRIDE * (j0 + jj);
                    const double x1d[3] = {r64[0], r64[1], r64[2]};
                    const double td[3] = {r64[4], r64[5], r64[6]};
                    const double bd[3] = {r64[8], r64[9], r64[10]};
                    const double qd[3] = {r64[12], r64[13], r64[14]};
                    PairK<double> kd;
                    pair_constants(td, bd, qd, bt, kd);
                    const double xi = gl4_xi(qp);
                    const double xq0 = __dadd_rn(xa, __dmul_rn(xi, Dx));
                    const double xq1 = __dadd_rn(ya, __dmul_rn(xi, Dy));
                    const double xq2 = __dadd_rn(za, __dmul_rn(xi, Dz));
                    double vd[3] = {0.0, 0.0, 0.0};
                    seg_sigma_b(xq0 - x1d[0], xq1 - x1d[1], xq2 - x1d[2], td, r64[3], bd, qd, bt, kd, c.a2, c.c1,
                                c.c2, vd);
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        const float hi = (float)vd[e];
                        const float lo = (float)(vd[e] - (double)hi);
                        kahan_add(sh[qp][e], sc[qp][e], hi);
                        kahan_add(sh[qp][e], sc[qp][e], lo);
                    }
                }
            }
        }
    }
    // count the FP64 point-pairs (one atomic per warp)
    if (a.near_count) {
        unsigned w = active ? near_here : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(a.near_count, (unsigned long long)w);
    }
    if (!active) return;
    double acc[4][3];
#pragma unroll
    for (int qp = 0; qp < 4; ++qp)
#pragma unroll
        for (int e = 0; e < 3; ++e) acc[qp][e] = (double)sh[qp][e] - (double)sc[qp][e];
    tile_store(a, seg, Dx, Dy, Dz, bt, acc);
}

}  // namespace ptadd
