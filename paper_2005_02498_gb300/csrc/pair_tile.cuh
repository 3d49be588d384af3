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
    const double* k64;      // device copy of {a2, c1, c2} for the near-field path (mixed)
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
    double acc[4][3];  // (sigma b') / c2 at the Gauss points, without the term along b'
    double accb[4];    // coefficient sums of the term along b'
#pragma unroll
    for (int qp = 0; qp < 4; ++qp) acc[qp][0] = acc[qp][1] = acc[qp][2] = accb[qp] = 0.0;
    const double nr = -c.c1 / c.c2, nra2 = nr * c.a2, kn = 1.0 - 2.0 * c.c1 / c.c2;

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
            PairK k;
            pair_constants(t, q, bt, nr, k);
            // per Gauss point the geometry, then a vote: where every pair of
            // the warp is one-sided the straddling forms are not evaluated
            // (the FP64 pipe is the bound, so the branches cost nothing there)
#pragma unroll
            for (int qp = 0; qp < 4; ++qp) {
                SegGeo G;
                seg_geo(xq[qp][0] - x1[0], xq[qp][1] - x1[1], xq[qp][2] - x1[2], t, L, c.a2, G);
                if (__all_sync(0xffffffffu, seg_one_side(G, L)))
                    seg_sigma_b_geo<1>(G, t, L, b, q, bt, k, c.a2, nr, nra2, kn, acc[qp], accb[qp]);
                else
                    seg_sigma_b_geo<0>(G, t, L, b, q, bt, k, c.a2, nr, nra2, kn, acc[qp], accb[qp]);
            }
        }
    }
#pragma unroll
    for (int qp = 0; qp < 4; ++qp)
#pragma unroll
        for (int e = 0; e < 3; ++e) acc[qp][e] = c.c2 * fma(accb[qp], bt[e], acc[qp][e]);
    if (active) tile_store(a, seg, Dx, Dy, Dz, bt, acc);
}

// ----------------------------------------------------------------- mixed
// Every (Gauss point, source) pair is first located in FP32 (coordinates
// relative to an integer origin near the target, so that R0 = x - x1 keeps
// FP32 resolution anywhere in the box); if the point lies within 10 a of the
// source segment the pair is evaluated in FP64 from the FP64 records,
// otherwise in FP32.  Per Gauss point the FP32 contributions are summed in
// three levels: plainly over the sources of each staged tile, with Kahan
// compensation over the tiles of the work item's source range, and in FP64
// over work items (where the FP64 near-field values also go); the FP64 sums
// feed the PK force and the nodal assembly.
//
// The FP32 work is packed: Gauss points (0,1) and (2,3) travel as the two
// lanes of a float2, so every add, multiply and fused multiply-add of the
// field formula is one FADD2/FMUL2/FFMA2 instruction for two points.  The
// shared-memory tile holds every source scalar duplicated into both lanes.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b, rounded once
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
// -a (a sign flip the compiler may fold into the instruction that uses it)
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 f2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 sel2(bool cx, bool cy, float2 a, float2 b)
{
    return make_float2(cx ? a.x : b.x, cy ? a.y : b.y);
}
// s + v with Kahan compensation c (s - c is the compensated sum)
__device__ __forceinline__ void kahan_add2(float2& s, float2& c, float2 v)
{
    const float2 y = sub2(v, c);
    const float2 t = add2(s, y);
    c = sub2(sub2(t, s), y);
    s = t;
}
// sources summed plainly before a compensated add: no fewer than a staged
// tile holds, so each tile's sources form one plain group
constexpr int SUM_GROUP = 256;
// sources of one group handled per loop iteration (two independent chains)
constexpr int MIX_UNROLL = 2;
// keep a register value opaque, so the compiler holds it instead of
// recomputing it from its (FP64) inputs inside the loop
__device__ __forceinline__ void opaque(float& x) { asm volatile("" : "+f"(x)); }

// Shared-memory record of one source for the packed loop (float2 units, every
// scalar in both lanes): x1 hi (0-2), x1 lo (3-5), L (6), t (7-9), b (10-12),
// q = b x t (13-15), -t (16-18), -b (19-21), L^2 (22), 2L (23).  The negated
// copies let the field formula use plain fused multiply-adds where it
// subtracts.
constexpr int MIX_REC = 24;

struct Src2 {
    float2 t[3], nt[3], L, b[3], nb[3], q[3], LL, L2;
};

// Quantities of one (source, target) pair shared by the four Gauss points:
// t.b', -t.b', q.b', -q.b'.
struct Pair2 {
    float2 tb, ntb, qb, nqb;
};

// Geometry of a (Gauss-point pair, source), given R0 = x - x1: ny = -y with
// y = R0.t, Rp = R0 - y t (the part of R0 normal to the source), d2 =
// |Rp|^2 + a^2, u2 = L - y, rho1^2 = y^2 + d2, rho2^2 = u2^2 + d2.
struct Geo2 {
    float2 ny, Rp[3], d2, u2, r1s, r2s;
};

__device__ __forceinline__ void seg_geo2(const float2 R0[3], const Src2& S, float2 a2, Geo2& G)
{
    G.ny = fma2(R0[0], S.nt[0], fma2(R0[1], S.nt[1], mul2(R0[2], S.nt[2])));
#pragma unroll
    for (int e = 0; e < 3; ++e) G.Rp[e] = fma2(G.ny, S.t[e], R0[e]);
    G.d2 = fma2(G.Rp[0], G.Rp[0], fma2(G.Rp[1], G.Rp[1], fma2(G.Rp[2], G.Rp[2], a2)));
    G.u2 = add2(S.L, G.ny);
    G.r1s = fma2(G.ny, G.ny, G.d2);
    G.r2s = fma2(G.u2, G.u2, G.d2);
}

// The packed field of one source at two Gauss points (lanes) in coefficient
// form:
//   (sigma b') / c2 = cRxb (Rp x b) + cq q + cRp Rp + ct t + cb b',
// the formula of seg_sigma_b (FP64: c2 taken out, K_k = 3 J_k, (b x b').Rp
// as b'.(Rp x b)) regrouped so that each coefficient costs few operations:
//   B0 = a^2 K2 + J0 (= A0 - J0),  C1 = r A1 + J1 = (r a^2) K3 + (1 + 2r) J1,
//   cRxb = (r A0) t.b',  cq = C1 t.b' - J0 (Rp.b'),
//   ct = (r A0) Rw + C1 q.b' + (q.Rp)(K4 t.b' - K3 (Rp.b')),
//   cRp = (q.Rp)(K2 (Rp.b') - K3 t.b') - J0 q.b',  cb = (q.Rp) B0,
// with r = -c1/c2 (nr) and Rw = b'.(Rp x b).  L (u1 + u2) = L (L + 2 ny)
// comes from L^2 and 2L of the record.  The reciprocal of a lane flagged near
// is replaced by 0; every coefficient carries it as a factor (all other
// factors are finite, rho >= a > 0), so such a lane contributes exactly 0 and
// the caller adds the terms unconditionally.  SAME = 1: every lane of the
// warp has both ends of the source on one side of the foot of the
// perpendicular (u1 u2 >= 0), so the straddling forms are not evaluated,
// and the one-side integrals come from the single reciprocal
// rr = 1 / ((p + m)(1 + pm)(1/rho1 + 1/rho2)) through Q = Li rr:
//   J0 = Li / (p + m) = Q (1 + pm) isum,  J1 = Li / isum = Q (p + m)(1 + pm),
//   K2 = J0 W = Q (isum Aw + (1 + pm) isum ssum),
// with W = Aw / (1 + pm) + ssum and Aw = ssum - d^2 / (rho1^2 rho2^2)
// = (u1^2 + u2^2 + d^2) / (rho1^2 rho2^2) (at least ssum / 2, so the
// difference loses at most one bit).  Every coefficient is linear in
// J0, J1, K2, so there they are formed without the factor Q, which the
// caller applies to their sum (C.Q): the reciprocal's latency then overlaps
// the whole coefficient arithmetic.  Straddling warps form the coefficients
// in full (C.Q = 1).  kn = 1 + 2r.
struct Coef2 {
    float2 cRxb, cq, cRp, ct, cb;
    float2 X[3];  // Rp x b
    float2 Q;     // common factor of the five coefficients
};

template <int SAME>
__device__ __forceinline__ void seg_coef2(const Geo2& G, const Src2& S, const float2 bt[3], const Pair2& P,
                                          float2 a2, float2 nr, float2 nra2, float2 kn, bool nearx, bool neary,
                                          Coef2& C)
{
    const float2 ny = G.ny, d2 = G.d2, u2 = G.u2, r1s = G.r1s, r2s = G.r2s;
    const float2 Rpx = G.Rp[0], Rpy = G.Rp[1], Rpz = G.Rp[2];
    const float2 i1 = make_float2(rsqrt_approx(r1s.x), rsqrt_approx(r1s.y));
    const float2 i2 = make_float2(rsqrt_approx(r2s.x), rsqrt_approx(r2s.y));
    const float2 m = mul2(ny, i1), p = mul2(u2, i2);
    const float2 i1s = mul2(i1, i1), i2s = mul2(i2, i2), i12 = mul2(i1s, i2s);
    const float2 ssum = add2(i1s, i2s);
    const float2 pm = mul2(p, m);
    const float2 S2 = fma2(p, p, fma2(m, m, pm));
    const float2 isum = add2(i1, i2);
    const float2 pps = add2(p, m), one_pm = add2(f2(1.0f), pm);
    const float2 Li = mul2(fma2(ny, S.L2, S.LL), i12);  // L (u1 + u2) / (rho1^2 rho2^2)
    const float2 E3 = fma2(i1, i2, ssum);
    float2 J0, J1, K2;
    if (SAME) {
        const float2 T = mul2(one_pm, isum);
        const float2 den = mul2(pps, one_pm);
        const float2 dis = mul2(pps, T);
        const float2 Aw = fma2(neg2(d2), i12, ssum);
        const float2 Z = fma2(isum, Aw, mul2(T, ssum));
        const float2 rr = sel2(nearx, neary, f2(0.0f), make_float2(rcp_approx(dis.x), rcp_approx(dis.y)));
        C.Q = mul2(Li, rr);
        J0 = T;
        J1 = den;
        K2 = Z;
    } else {
        C.Q = f2(1.0f);
        const bool samex = (ny.x >= 0.0f) || (u2.x <= 0.0f);
        const bool samey = (ny.y >= 0.0f) || (u2.y <= 0.0f);
        const float2 den = sel2(samex, samey, mul2(pps, one_pm), d2);
        const float2 dis = mul2(den, isum);
        const float2 rr = sel2(nearx, neary, f2(0.0f), make_float2(rcp_approx(dis.x), rcp_approx(dis.y)));
        const float2 rden = mul2(rr, isum);
        J1 = mul2(Li, mul2(rr, den));
        const float2 g = mul2(Li, rden);
        // one-side form of (3 - p^2 - pm - m^2)/d^2: (u1^2 + u2^2 + d^2)/(rho1^2 rho2^2 (1 + pm)) + 1/rho1^2 + 1/rho2^2
        const float2 Wsame = fma2(mul2(mul2(fma2(ny, ny, r2s), i12), rden), pps, ssum);
        J0 = sel2(samex, samey, mul2(g, one_pm), mul2(sub2(p, m), rden));
        K2 = mul2(J0, sel2(samex, samey, Wsame, mul2(sub2(f2(3.0f), S2), rden)));
    }
    const float2 K3 = mul2(J1, E3);
    const float2 K4 = mul2(J0, S2);
    const float2 B0 = fma2(a2, K2, J0);
    const float2 A0 = add2(B0, J0);
    const float2 C1 = fma2(nra2, K3, mul2(kn, J1));
    const float2 nrA0 = mul2(nr, A0);
    C.X[0] = fma2(Rpy, S.b[2], mul2(Rpz, S.nb[1]));
    C.X[1] = fma2(Rpz, S.b[0], mul2(Rpx, S.nb[2]));
    C.X[2] = fma2(Rpx, S.b[1], mul2(Rpy, S.nb[0]));
    const float2 Rb = fma2(Rpx, bt[0], fma2(Rpy, bt[1], mul2(Rpz, bt[2])));
    const float2 nRb = neg2(Rb);
    const float2 Rw = fma2(C.X[0], bt[0], fma2(C.X[1], bt[1], mul2(C.X[2], bt[2])));
    const float2 qR = fma2(Rpx, S.q[0], fma2(Rpy, S.q[1], mul2(Rpz, S.q[2])));
    C.cRxb = mul2(nrA0, P.tb);
    C.cq = fma2(P.tb, C1, mul2(J0, nRb));
    C.ct = fma2(nrA0, Rw, fma2(C1, P.qb, mul2(qR, fma2(K3, nRb, mul2(K4, P.tb)))));
    C.cRp = fma2(qR, fma2(K3, P.ntb, mul2(K2, Rb)), mul2(J0, P.nqb));
    C.cb = mul2(qR, B0);
}

// One near-field (Gauss point, source) pair in FP64: (sigma b') of source js
// at Gauss point qp of target seg, from the FP64 records.
__device__ __forceinline__ double3 near_field_fp64(const double* __restrict__ pos, int64_t n,
                                                   const int32_t* __restrict__ nxt, const double* __restrict__ src,
                                                   int64_t seg, int64_t js, int qp, const double* __restrict__ k64)
{
    const double a2 = k64[0], c1 = k64[1], c2 = k64[2];
    const double* tr = src + (int64_t)SRC_STRIDE * seg;
    const int64_t sb = nxt[seg];
    const double xa = pos[seg], ya = pos[n + seg], za = pos[2 * n + seg];
    const double Dx = pos[sb] - xa, Dy = pos[n + sb] - ya, Dz = pos[2 * n + sb] - za;
    const double bt[3] = {tr[8], tr[9], tr[10]};
    const double* r64 = src + (int64_t)SRC_STRIDE * js;
    const double x1d[3] = {r64[0], r64[1], r64[2]};
    const double td[3] = {r64[4], r64[5], r64[6]};
    const double bd[3] = {r64[8], r64[9], r64[10]};
    const double qd[3] = {r64[12], r64[13], r64[14]};
    const double nr = -c1 / c2;
    PairK kd;
    pair_constants(td, qd, bt, nr, kd);
    const double xi = gl4_xi(qp);
    const double xq0 = __dadd_rn(xa, __dmul_rn(xi, Dx));
    const double xq1 = __dadd_rn(ya, __dmul_rn(xi, Dy));
    const double xq2 = __dadd_rn(za, __dmul_rn(xi, Dz));
    double vd[3] = {0.0, 0.0, 0.0};
    seg_sigma_b(xq0 - x1d[0], xq1 - x1d[1], xq2 - x1d[2], td, r64[3], bd, qd, bt, kd, a2, nr, vd);
    return make_double3(c2 * vd[0], c2 * vd[1], c2 * vd[2]);
}

// Near pairs found by a warp wait in a per-warp queue of (source index,
// owner lane << 2 | Gauss point) entries; a full queue is evaluated 32 at a
// time, one entry per lane, so the FP64 work runs with every lane busy.
// Each result goes to its owner's FP64 near sums in queue order, so the
// summation order (and the result) does not depend on scheduling.
constexpr int NEAR_Q = 160;  // <= 31 waiting + 128 added by one source (4 Gauss points x 32 lanes)

template <int TILE, int TPB>
struct MixSmem {
    float2 tile[TILE * MIX_REC];  // source records (MIX_REC float2 each)
    double nacc[12 * TPB];             // FP64 sums: [qp * 3 + e][thread]
    float2 ksum[12 * TPB];             // Kahan sums of the work item: [p * 3 + e][thread], then compensations
    uint2 queue[TPB / 32][NEAR_Q];
};

// Evaluate the first cnt (<= 32) entries of a warp queue; warp-uniform call.
static __device__ __noinline__ void near_flush(const double* __restrict__ pos, int64_t n,
                                               const int32_t* __restrict__ nxt, const double* __restrict__ src,
                                               const double* __restrict__ k64, int64_t seg,
                                               const uint2* __restrict__ q, int cnt, double* __restrict__ nacc,
                                               int tpb)
{
    const int lane = threadIdx.x & 31;
    const uint2 e = lane < cnt ? q[lane] : make_uint2(0u, 0u);
    const int64_t seg_o = __shfl_sync(0xffffffffu, (long long)seg, (int)((e.y >> 2) & 31u));
    double3 d = make_double3(0.0, 0.0, 0.0);
    if (lane < cnt) d = near_field_fp64(pos, n, nxt, src, seg_o, (int64_t)e.x, (int)(e.y & 3u), k64);
    for (int k = 0; k < cnt; ++k) {
        const double dx = __shfl_sync(0xffffffffu, d.x, k);
        const double dy = __shfl_sync(0xffffffffu, d.y, k);
        const double dz = __shfl_sync(0xffffffffu, d.z, k);
        const unsigned tag = __shfl_sync(0xffffffffu, e.y, k);
        if ((int)((tag >> 2) & 31u) == lane) {
            double* acc = nacc + 3 * (int)(tag & 3u) * tpb + threadIdx.x;
            acc[0] += dx;
            acc[tpb] += dy;
            acc[2 * tpb] += dz;
        }
    }
}

// Drop the first 32 entries of a warp queue holding cnt (32 < cnt <= NEAR_Q)
// of them: chunk by chunk, each read before the chunk below it is overwritten.
__device__ __forceinline__ void near_shift(uint2* q, int cnt)
{
    const int lane = threadIdx.x & 31;
    for (int base = 32; base < cnt; base += 32) {
        const uint2 u = base + lane < cnt ? q[base + lane] : make_uint2(0u, 0u);
        __syncwarp();
        if (base + lane < cnt) q[base - 32 + lane] = u;
        __syncwarp();
    }
}

template <int TILE, int TPB>
__device__ __forceinline__ void pair_tile_mixed(const TileArgs& a, const Consts& c, float near2,
                                                MixSmem<TILE, TPB>& sm)
{
    const int64_t n = a.n;
    const bool active = threadIdx.x < a.t_count;
    const int64_t seg = active ? a.tgt[a.t_begin + threadIdx.x] : a.tgt[a.t_begin];
    const double* tr = a.src + (int64_t)SRC_STRIDE * seg;
    const int64_t sb = a.nxt[seg];
    const double xa = a.pos[seg], ya = a.pos[n + seg], za = a.pos[2 * n + seg];
    const double Dx = a.pos[sb] - xa, Dy = a.pos[n + sb] - ya, Dz = a.pos[2 * n + sb] - za;
    const double bt[3] = {tr[8], tr[9], tr[10]};
    float btf[3] = {(float)bt[0], (float)bt[1], (float)bt[2]};
    opaque(btf[0]);
    opaque(btf[1]);
    opaque(btf[2]);
    const float2 bt2[3] = {f2(btf[0]), f2(btf[1]), f2(btf[2])};
    // Gauss points relative to an integer origin Ot near this target (its
    // first Gauss point, rounded, in the frame of the split origin): within a
    // segment length of Ot, so FP32 holds them to ~1e-7 of that length.  A
    // source start x1 = h1 + l1 (integer hi part, |lo| <= 1/2) then moves to
    // this frame as (h1 - Ot) + l1: the integer parts subtract exactly and the
    // fraction rounds once, i.e. to ~1 ulp of |x1 - Ot| ~ |R0| + L.
    // Pair p holds Gauss points 2p, 2p+1.
    float2 XT[2][3];
    float nOt[3];
    {
        double Ot[3];
#pragma unroll
        for (int qp = 0; qp < 4; ++qp) {
            const double xi = gl4_xi(qp);
            const double qd[3] = {__dadd_rn(xa, __dmul_rn(xi, Dx)) - a.origin[0],
                                  __dadd_rn(ya, __dmul_rn(xi, Dy)) - a.origin[1],
                                  __dadd_rn(za, __dmul_rn(xi, Dz)) - a.origin[2]};
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                if (qp == 0) {
                    Ot[e] = rint(qd[e]);
                    nOt[e] = (float)(-Ot[e]);
                    opaque(nOt[e]);
                }
                float xf = (float)(qd[e] - Ot[e]);
                opaque(xf);
                if (qp & 1)
                    XT[qp >> 1][e].y = xf;
                else
                    XT[qp >> 1][e].x = xf;
            }
        }
    }
    // FP64 sums per Gauss point (far-field sums of the work item and
    // near-field values); Kahan sums of the work item and their compensations
#pragma unroll
    for (int k = 0; k < 12; ++k) sm.nacc[k * TPB + threadIdx.x] = 0.0;
#pragma unroll
    for (int k = 0; k < 12; ++k) sm.ksum[k * TPB + threadIdx.x] = f2(0.0f);
    // loop-invariant constants held in registers (not re-derived from FP64 inputs in the loop)
    float kc[4] = {(float)c.a2, (float)(-c.c1 / c.c2), (float)(-c.c1 / c.c2 * c.a2), (float)(1.0 - 2.0 * c.c1 / c.c2)};
#pragma unroll
    for (int k = 0; k < 4; ++k) opaque(kc[k]);
    const float2 a2 = f2(kc[0]), nr = f2(kc[1]), nra2 = f2(kc[2]), kn = f2(kc[3]);
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    uint2* wq = sm.queue[threadIdx.x >> 5];
    int qn = 0;             // entries waiting in this warp's queue (warp-uniform)
    unsigned near_warp = 0;  // near point-pairs of this warp (warp-uniform)

    for (int64_t j0 = a.js; j0 < a.je; j0 += TILE) {
        const int cnt = (int)min((int64_t)TILE, a.je - j0);
        __syncthreads();
        for (int js = threadIdx.x; js < cnt; js += blockDim.x) {
            const float4* g = reinterpret_cast<const float4*>(a.src32 + (int64_t)SRC32_STRIDE * (j0 + js));
            float v[SRC32_STRIDE];
#pragma unroll
            for (int e = 0; e < SRC32_STRIDE / 4; ++e) {
                const float4 u = g[e];
                v[4 * e] = u.x;
                v[4 * e + 1] = u.y;
                v[4 * e + 2] = u.z;
                v[4 * e + 3] = u.w;
            }
            float4* d = reinterpret_cast<float4*>(sm.tile + (int64_t)MIX_REC * js);
#pragma unroll
            for (int e = 0; e < 8; ++e) d[e] = make_float4(v[2 * e], v[2 * e], v[2 * e + 1], v[2 * e + 1]);
            d[8] = make_float4(-v[7], -v[7], -v[8], -v[8]);
            d[9] = make_float4(-v[9], -v[9], -v[10], -v[10]);
            d[10] = make_float4(-v[11], -v[11], -v[12], -v[12]);
            d[11] = make_float4(v[6] * v[6], v[6] * v[6], v[6] + v[6], v[6] + v[6]);
        }
        __syncthreads();
        // plain sums of the current group of SUM_GROUP sources (/ c2); the
        // b' term's coefficient is summed on its own (b' is the target's)
        float2 SG[2][3], SB[2];
        for (int g0 = 0; g0 < cnt; g0 += SUM_GROUP) {
            const int g1 = min(cnt, g0 + SUM_GROUP);
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                SB[p] = f2(0.0f);
#pragma unroll
                for (int e = 0; e < 3; ++e) SG[p][e] = f2(0.0f);
            }
#pragma unroll MIX_UNROLL
            for (int jj = g0; jj < g1; ++jj) {
                const float2* r = sm.tile + jj * MIX_REC;
                if (!(r[6].x > 0.0f)) continue;  // zero-length source (uniform branch)
                Src2 S;
                S.L = r[6];
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    S.t[e] = r[7 + e];
                    S.b[e] = r[10 + e];
                    S.q[e] = r[13 + e];
                    S.nt[e] = r[16 + e];
                    S.nb[e] = r[19 + e];
                }
                S.LL = r[22];
                S.L2 = r[23];
                Pair2 P;
                P.tb = fma2(S.t[0], bt2[0], fma2(S.t[1], bt2[1], mul2(S.t[2], bt2[2])));
                P.qb = fma2(S.q[0], bt2[0], fma2(S.q[1], bt2[1], mul2(S.q[2], bt2[2])));
                P.ntb = neg2(P.tb);
                P.nqb = neg2(P.qb);
                // the source start in this thread's frame
                float x1t[3];
#pragma unroll
                for (int e = 0; e < 3; ++e) x1t[e] = (r[e].x + nOt[e]) + r[3 + e].x;
                // near test of both Gauss-point pairs first (point-to-segment
                // distance), then the coefficients (near lanes give 0)
                Geo2 G[2];
                bool nrq[2][2];
                bool same_all = true;
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    float2 R0[3];
#pragma unroll
                    for (int e = 0; e < 3; ++e) R0[e] = sub2(XT[p][e], f2(x1t[e]));
                    seg_geo2(R0, S, a2, G[p]);
                    const float2 ny = G[p].ny, u2 = G[p].u2;
                    // y < 0: nearest to x1; y > L: nearest to x2; else to the line
                    const float2 dd = sel2(ny.x > 0.0f, ny.y > 0.0f, G[p].r1s,
                                           sel2(u2.x < 0.0f, u2.y < 0.0f, G[p].r2s, G[p].d2));
                    nrq[p][0] = active && dd.x < near2;
                    nrq[p][1] = active && dd.y < near2;
                    same_all = same_all && (ny.x >= 0.0f || u2.x <= 0.0f) && (ny.y >= 0.0f || u2.y <= 0.0f);
                }
                const bool uni = __all_sync(0xffffffffu, same_all);
                // both Gauss-point pairs in one straight block per branch, so
                // that their two chains interleave
                Coef2 C[2];
                if (uni) {
                    seg_coef2<1>(G[0], S, bt2, P, a2, nr, nra2, kn, nrq[0][0], nrq[0][1], C[0]);
                    seg_coef2<1>(G[1], S, bt2, P, a2, nr, nra2, kn, nrq[1][0], nrq[1][1], C[1]);
                } else {
                    seg_coef2<0>(G[0], S, bt2, P, a2, nr, nra2, kn, nrq[0][0], nrq[0][1], C[0]);
                    seg_coef2<0>(G[1], S, bt2, P, a2, nr, nra2, kn, nrq[1][0], nrq[1][1], C[1]);
                }
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    SB[p] = fma2(C[p].Q, C[p].cb, SB[p]);  // (times b' when the group closes)
#pragma unroll
                    for (int e = 0; e < 3; ++e)
                        SG[p][e] = fma2(C[p].Q, fma2(C[p].cRxb, C[p].X[e], fma2(C[p].cq, S.q[e],
                                        fma2(C[p].cRp, G[p].Rp[e], mul2(C[p].ct, S.t[e])))), SG[p][e]);
                }
                if (__any_sync(0xffffffffu, nrq[0][0] || nrq[0][1] || nrq[1][0] || nrq[1][1])) {
                    const unsigned js = (unsigned)(j0 + jj);
#pragma unroll
                    for (int qp = 0; qp < 4; ++qp) {
                        const bool mine = nrq[qp >> 1][qp & 1];
                        const unsigned bal = __ballot_sync(0xffffffffu, mine);
                        if (mine) wq[qn + __popc(bal & lt)] = make_uint2(js, ((unsigned)lane << 2) | (unsigned)qp);
                        qn += __popc(bal);
                        near_warp += (unsigned)__popc(bal);
                    }
                    while (qn >= 32) {
                        __syncwarp();
                        near_flush(a.pos, n, a.nxt, a.src, a.k64, seg, wq, 32, sm.nacc, TPB);
                        near_shift(wq, qn);
                        qn -= 32;
                    }
                }
            }
            // close the group
#pragma unroll
            for (int p = 0; p < 2; ++p)
#pragma unroll
                for (int e = 0; e < 3; ++e) SG[p][e] = fma2(SB[p], bt2[e], SG[p][e]);
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                float2 sk = sm.ksum[k * TPB + threadIdx.x], ck = sm.ksum[(6 + k) * TPB + threadIdx.x];
                kahan_add2(sk, ck, SG[k / 3][k % 3]);
                sm.ksum[k * TPB + threadIdx.x] = sk;
                sm.ksum[(6 + k) * TPB + threadIdx.x] = ck;
            }
        }
    }
    // compensated sums of the work item's sources to FP64, restoring the factor c2
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const float2 sk = sm.ksum[(3 * p + e) * TPB + threadIdx.x];
            const float2 ck = sm.ksum[(6 + 3 * p + e) * TPB + threadIdx.x];
            double* acc = sm.nacc + (6 * p + e) * TPB + threadIdx.x;
            acc[0] = fma(c.c2, (double)sk.x - (double)ck.x, acc[0]);
            acc[3 * TPB] = fma(c.c2, (double)sk.y - (double)ck.y, acc[3 * TPB]);
        }
    if (qn > 0) {
        __syncwarp();
        near_flush(a.pos, n, a.nxt, a.src, a.k64, seg, wq, qn, sm.nacc, TPB);
    }
    // count the FP64 point-pairs (one atomic per warp)
    if (a.near_count && lane == 0 && near_warp) atomicAdd(a.near_count, (unsigned long long)near_warp);
    __syncwarp();
    if (!active) return;
    double acc[4][3];
#pragma unroll
    for (int qp = 0; qp < 4; ++qp)
#pragma unroll
        for (int e = 0; e < 3; ++e) acc[qp][e] = sm.nacc[(3 * qp + e) * TPB + threadIdx.x];
    tile_store(a, seg, Dx, Dy, Dz, bt, acc);
}

}  // namespace ptadd
