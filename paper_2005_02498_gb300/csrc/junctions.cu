// junctions.cu -- junctions between mobile and sessile lines and their
// thermally activated breaking (Sec. 2.2), inside the burst of
// ptadd_advance.
//
// Per step, between the velocity stage and the Euler stage, three kernels:
//   junction_release_kernel (one thread per node): a held node whose break
//     time has come lets go (and remembers the sessile loop it left); every
//     free node that holds nothing goes on the list of nodes looking for a
//     junction, with its best candidate reset;
//   junction_search_kernel (one warp per (looking node, 32 sessile
//     segments), spread over every SM): each lane tests one sessile segment
//     of another loop (not the one the node last left) against the capture
//     radius; the warp's lowest passing position in the sessile list goes
//     into the node's candidate with an atomic minimum, so the lowest-index
//     segment wins whatever the order of the warps;
//   junction_hold_kernel (one thread per node): forms the junction found
//     (breaking after f a), holds the velocity of a held node at 0, and
//     reduces the largest squared speed of the free nodes, the number of
//     held junctions and the earliest break time with 64-bit atomics on the
//     bit patterns of non-negative doubles, whose integer order is their
//     numeric order, so the result does not depend on the order of the
//     atomics.
// after the Euler stage:
//   junction_event_kernel (one thread): t <- t + dt, or, if some junction is
//     held and no free node moved more than the stuck displacement, t <- the
//     earliest break time; the frozen interval adds (the step's line length)
//     x (the interval) to the rho sum, nothing to the Lp sum, and the
//     interval to the time sum.
// Distances and times are formed with explicit round-to-nearest operations,
// no contraction, so a decision depends only on the positions and the clock.
//
// Batched ensembles (ptadd_batch_set_junctions): the same rules per
// realisation, each with its own clock, stuck test and jumps, and break
// fractions drawn from the stream of seed ^ (r * 0x9E3779B97F4A7C15) with the
// realisation-local node number, so realisation r behaves as it would alone
// under ptadd_set_junctions with that seed.  The capture search is one thread
// per free node over its realisation's sessile list, staged through shared
// memory in ascending order: an FP32 distance (positions split into an exact
// integer part and a remainder about the realisation's origin, as in the pair
// kernel's records) rejects the segments that are clearly out of reach, with
// a margin of 4e-6 (|w|_1 + L) that covers its rounding, and the first
// segment that passes the FP64 test of the single-network search is the
// node's junction: the lowest position, as there.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ptadd_internal.cuh"

namespace ptadd {

struct DevJunctions {
    double rc2 = 0;        // capture radius^2, internal length units
    double a = 0;          // maximum break time, s
    double stuck_hat = 0;  // stuck displacement, internal length units
    uint64_t seed = 0;
    int64_t n_sess = 0;
    int32_t* sess = nullptr;     // sessile segments, ascending
    int32_t* seg = nullptr;      // per node: held sessile segment or -1
    int32_t* last = nullptr;     // per node: sessile loop last broken from or -1
    int32_t* count = nullptr;    // per node: junctions formed
    double* brk = nullptr;       // per node: break time, s
    double* clock = nullptr;     // [0] DD time, [1] time jumped (s)
    unsigned long long* red = nullptr;  // [0] max v^2 bits, [1] min break bits, [2] held,
                                        // [3] formed, [4] broken, [5] jumps
    int64_t n_free = 0;          // unpinned nodes (the most that can look in one step)
    int32_t* look = nullptr;     // nodes looking for a junction this step (any order)
    unsigned* look_n = nullptr;  // their number (reset by the event kernel)
    int32_t* found = nullptr;    // per node: lowest passing position in sess, or INT32_MAX
};

namespace {

constexpr int JT = 256;
constexpr unsigned long long INF_BITS = 0x7FF0000000000000ull;

__device__ __forceinline__ uint64_t splitmix64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// f in [0,1) of the k-th junction of `node`: SplitMix64 (Vigna) output k+1
// of the stream seeded with seed ^ (node * 0xD1B54A32D192ED03), top 53 bits
__device__ __forceinline__ double break_fraction(uint64_t seed, int64_t node, int32_t k)
{
    const uint64_t s = seed ^ ((uint64_t)node * 0xD1B54A32D192ED03ull);
    const uint64_t z = splitmix64_mix(s + (uint64_t)(k + 1) * 0x9E3779B97F4A7C15ull);
    return (double)(z >> 11) * 0x1.0p-53;
}

// squared distance from (x, y, z) to the segment p1 -> p2, clamped to it
__device__ __forceinline__ double seg_dist2(double x, double y, double z, const double* p)
{
    const double ex = __dsub_rn(p[3], p[0]), ey = __dsub_rn(p[4], p[1]), ez = __dsub_rn(p[5], p[2]);
    const double wx = __dsub_rn(x, p[0]), wy = __dsub_rn(y, p[1]), wz = __dsub_rn(z, p[2]);
    const double ee = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
    double u = 0.0;
    if (ee > 0.0) {
        u = __ddiv_rn(__dadd_rn(__dadd_rn(__dmul_rn(wx, ex), __dmul_rn(wy, ey)), __dmul_rn(wz, ez)), ee);
        u = u < 0.0 ? 0.0 : (u > 1.0 ? 1.0 : u);
    }
    const double rx = __dsub_rn(wx, __dmul_rn(u, ex)), ry = __dsub_rn(wy, __dmul_rn(u, ey)),
                 rz = __dsub_rn(wz, __dmul_rn(u, ez));
    return __dadd_rn(__dadd_rn(__dmul_rn(rx, rx), __dmul_rn(ry, ry)), __dmul_rn(rz, rz));
}

__global__ void __launch_bounds__(JT) junction_release_kernel(
    int64_t n, const int32_t* __restrict__ loop_of, const uint8_t* __restrict__ pinned, int32_t* __restrict__ jseg,
    int32_t* __restrict__ jlast, const double* __restrict__ jbrk, const double* __restrict__ clock,
    int32_t* __restrict__ look, unsigned* __restrict__ look_n, int32_t* __restrict__ found,
    unsigned long long* __restrict__ red)
{
    const int64_t p = blockIdx.x * (int64_t)JT + threadIdx.x;
    if (p >= n || pinned[p]) return;
    int32_t js = jseg[p];
    if (js >= 0 && jbrk[p] <= clock[0]) {
        jlast[p] = loop_of[js];
        jseg[p] = -1;
        js = -1;
        atomicAdd(&red[4], 1ull);
    }
    if (js < 0) {
        found[p] = INT32_MAX;
        look[atomicAdd(look_n, 1u)] = (int32_t)p;
    }
}

// Block: JSW warps; warp w of block (x, y) tests look[x JSW + w] against the
// sessile positions 32 y .. 32 y + 31, one per lane.
constexpr int JSW = 8;

__global__ void __launch_bounds__(32 * JSW) junction_search_kernel(
    int64_t n, const double* __restrict__ pos, const int32_t* __restrict__ nxt, const int32_t* __restrict__ loop_of,
    const int32_t* __restrict__ sess, int64_t n_sess, const int32_t* __restrict__ jlast,
    const int32_t* __restrict__ look, const unsigned* __restrict__ look_n, int32_t* __restrict__ found, double rc2)
{
    const int li = blockIdx.x * JSW + (threadIdx.x >> 5);
    if (li >= (int)*look_n) return;  // warp-uniform
    const int64_t k = (int64_t)blockIdx.y * 32 + (threadIdx.x & 31);
    const int32_t p = look[li];
    bool hit = false;
    if (k < n_sess) {
        const int32_t sg = sess[k];
        const int32_t sl = loop_of[sg];
        if (sl != loop_of[p] && sl != jlast[p]) {
            const int32_t e = nxt[sg];
            const double sp[6] = {pos[sg], pos[n + sg], pos[2 * n + sg], pos[e], pos[n + e], pos[2 * n + e]};
            hit = seg_dist2(pos[p], pos[n + p], pos[2 * n + p], sp) < rc2;
        }
    }
    const unsigned cand = hit ? (unsigned)k : 0xFFFFFFFFu;
    const unsigned best = __reduce_min_sync(0xffffffffu, cand);
    if ((threadIdx.x & 31) == 0 && best != 0xFFFFFFFFu) atomicMin(&found[p], (int32_t)best);
}

__global__ void __launch_bounds__(JT) junction_hold_kernel(
    int64_t n, const uint8_t* __restrict__ pinned, double* __restrict__ vel, const int32_t* __restrict__ sess,
    int32_t* __restrict__ jseg, int32_t* __restrict__ jcount, double* __restrict__ jbrk,
    const int32_t* __restrict__ found, const double* __restrict__ clock, double a, uint64_t seed,
    unsigned long long* __restrict__ red)
{
    const int64_t p = blockIdx.x * (int64_t)JT + threadIdx.x;
    if (p >= n || pinned[p]) return;
    int32_t js = jseg[p];
    if (js < 0 && found[p] != INT32_MAX) {
        js = sess[found[p]];
        const int32_t k = jcount[p];
        jbrk[p] = __dadd_rn(clock[0], __dmul_rn(a, break_fraction(seed, p, k)));
        jcount[p] = k + 1;
        jseg[p] = js;
        atomicAdd(&red[3], 1ull);
    }
    if (js >= 0) {
        vel[p] = 0.0;
        vel[n + p] = 0.0;
        vel[2 * n + p] = 0.0;
        atomicAdd(&red[2], 1ull);
        atomicMin(&red[1], (unsigned long long)__double_as_longlong(jbrk[p]));
    } else {
        const double v2 = vel[p] * vel[p] + vel[n + p] * vel[n + p] + vel[2 * n + p] * vel[2 * n + p];
        atomicMax(&red[0], (unsigned long long)__double_as_longlong(v2));
    }
}

__global__ void junction_event_kernel(double* __restrict__ clock, unsigned long long* __restrict__ red,
                                      double* __restrict__ acc, unsigned* __restrict__ look_n, double dt_s,
                                      double dt_hat, double stuck_hat, double time_scale)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    *look_n = 0u;
    const double t1 = __dadd_rn(clock[0], dt_s);
    const double vmax = sqrt(__longlong_as_double((long long)red[0]));
    const double tmin = __longlong_as_double((long long)red[1]);
    double tn = t1;
    if (red[2] > 0 && vmax * dt_hat < stuck_hat && tmin > t1) {
        const double jump = __dsub_rn(tmin, t1);
        clock[1] = __dadd_rn(clock[1], jump);
        const double jh = jump * time_scale;
        acc[9] = fma(acc[11], jh, acc[9]);
        acc[12] += jh;
        red[5] += 1;
        tn = tmin;
    }
    clock[0] = tn;
    red[0] = 0;
    red[1] = INF_BITS;
    red[2] = 0;
}

// ------------------------------------------------------ batched ensembles
__global__ void __launch_bounds__(JT) bj_release_kernel(int64_t n, const int32_t* __restrict__ real_of,
                                                        const int32_t* __restrict__ loop_of,
                                                        const uint8_t* __restrict__ pinned, int32_t* __restrict__ jseg,
                                                        int32_t* __restrict__ jlast, const double* __restrict__ jbrk,
                                                        const double* __restrict__ clock,
                                                        unsigned long long* __restrict__ red)
{
    const int64_t p = blockIdx.x * (int64_t)JT + threadIdx.x;
    if (p >= n || pinned[p]) return;
    const int r = real_of[p];
    const int32_t js = jseg[p];
    if (js >= 0 && jbrk[p] <= clock[2 * r]) {
        jlast[p] = loop_of[js];
        jseg[p] = -1;
        atomicAdd(&red[6 * r + 4], 1ull);
    }
}

constexpr int JB = 128;  // free nodes per search block = sessile segments per staged tile
constexpr int JREC = 11; // staged record: x1 integer part (3), remainder (3), L, unit tangent (3), loop

// Block: one item (realisation r, up to JB consecutive entries of its free-node
// list); thread t looks for node free_nodes[f0 + t] if it holds nothing.
__global__ void __launch_bounds__(JB) bj_search_kernel(
    const double* __restrict__ pos, int64_t n, const int32_t* __restrict__ nxt, const int32_t* __restrict__ loop_of,
    const float* __restrict__ src32, const int32_t* __restrict__ sess, const int32_t* __restrict__ sess_off,
    const int32_t* __restrict__ free_nodes, const int32_t* __restrict__ items, const int32_t* __restrict__ jseg,
    const int32_t* __restrict__ jlast, int32_t* __restrict__ found, double rc2, float rc_f)
{
    __shared__ float rec[JB][JREC];
    const int r = items[3 * blockIdx.x], f0 = items[3 * blockIdx.x + 1], fc = items[3 * blockIdx.x + 2];
    const int t = threadIdx.x;
    int32_t p = -1;
    bool look = false;
    if (t < fc) {
        p = free_nodes[f0 + t];
        look = jseg[p] < 0;
    }
    float ph[3] = {0.f, 0.f, 0.f}, pl[3] = {0.f, 0.f, 0.f};
    double px = 0.0, py = 0.0, pz = 0.0;
    int32_t own = -1, left = -1;
    if (look) {
        const float* f = src32 + (int64_t)SRC32_STRIDE * p;  // the record of segment p starts at node p
        for (int c = 0; c < 3; ++c) {
            ph[c] = f[c];
            pl[c] = f[3 + c];
        }
        px = pos[p];
        py = pos[n + p];
        pz = pos[2 * n + p];
        own = loop_of[p];
        left = jlast[p];
    }
    int32_t best = INT32_MAX;
    const int k0 = sess_off[r], k1 = sess_off[r + 1];
    for (int kb = k0; kb < k1; kb += JB) {
        // (also the barrier between the last tile's reads and this tile's writes)
        if (!__syncthreads_or(look && best == INT32_MAX)) break;
        if (kb + t < k1) {
            const int32_t sg = sess[kb + t];
            const float* f = src32 + (int64_t)SRC32_STRIDE * sg;
#pragma unroll
            for (int c = 0; c < 10; ++c) rec[t][c] = f[c];
            rec[t][10] = __int_as_float(loop_of[sg]);
        }
        __syncthreads();
        if (look && best == INT32_MAX) {
            const int m = min(JB, k1 - kb);
            for (int q = 0; q < m; ++q) {
                const int32_t sl = __float_as_int(rec[q][10]);
                if (sl == own || sl == left) continue;
                // w = x_p - x_1: integer parts exactly, then the remainders
                const float wx = (ph[0] - rec[q][0]) + (pl[0] - rec[q][3]);
                const float wy = (ph[1] - rec[q][1]) + (pl[1] - rec[q][4]);
                const float wz = (ph[2] - rec[q][2]) + (pl[2] - rec[q][5]);
                const float L = rec[q][6], tx = rec[q][7], ty = rec[q][8], tz = rec[q][9];
                const float u = fminf(fmaxf(wx * tx + wy * ty + wz * tz, 0.0f), L);
                const float rx = wx - u * tx, ry = wy - u * ty, rz = wz - u * tz;
                const float dl = 4e-6f * (fabsf(wx) + fabsf(wy) + fabsf(wz) + L);
                if (rx * rx + ry * ry + rz * rz >= (rc_f + dl) * (rc_f + dl)) continue;
                const int32_t sg = sess[kb + q], e = nxt[sg];
                const double sp[6] = {pos[sg], pos[n + sg], pos[2 * n + sg], pos[e], pos[n + e], pos[2 * n + e]};
                if (seg_dist2(px, py, pz, sp) < rc2) {
                    best = kb + q;
                    break;
                }
            }
        }
    }
    if (look) found[p] = best;
}

__global__ void __launch_bounds__(JT) bj_hold_kernel(
    int64_t n, const int32_t* __restrict__ real_of, const int64_t* __restrict__ node_off,
    const uint8_t* __restrict__ pinned, double* __restrict__ vel, const int32_t* __restrict__ sess,
    int32_t* __restrict__ jseg, int32_t* __restrict__ jcount, double* __restrict__ jbrk,
    const int32_t* __restrict__ found, const double* __restrict__ clock, double a, uint64_t seed,
    unsigned long long* __restrict__ red)
{
    const int64_t p = blockIdx.x * (int64_t)JT + threadIdx.x;
    if (p >= n || pinned[p]) return;
    const int r = real_of[p];
    unsigned long long* rd = red + 6 * r;
    int32_t js = jseg[p];
    if (js < 0 && found[p] != INT32_MAX) {  // (found is written for every node that looked this step)
        js = sess[found[p]];
        const int32_t k = jcount[p];
        const uint64_t sr = seed ^ ((uint64_t)r * 0x9E3779B97F4A7C15ull);
        jbrk[p] = __dadd_rn(clock[2 * r], __dmul_rn(a, break_fraction(sr, p - node_off[r], k)));
        jcount[p] = k + 1;
        jseg[p] = js;
        atomicAdd(&rd[3], 1ull);
    }
    if (js >= 0) {
        vel[p] = 0.0;
        vel[n + p] = 0.0;
        vel[2 * n + p] = 0.0;
        atomicAdd(&rd[2], 1ull);
        atomicMin(&rd[1], (unsigned long long)__double_as_longlong(jbrk[p]));
    } else {
        const double v2 = vel[p] * vel[p] + vel[n + p] * vel[n + p] + vel[2 * n + p] * vel[2 * n + p];
        atomicMax(&rd[0], (unsigned long long)__double_as_longlong(v2));
    }
}

// one thread per realisation: the clock step or the jump (as junction_event_kernel)
__global__ void bj_event_kernel(int R, double* __restrict__ clock, unsigned long long* __restrict__ red,
                                double* __restrict__ acc, double dt_s, double dt_hat, double stuck_hat,
                                double time_scale)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double* ck = clock + 2 * r;
    unsigned long long* rd = red + 6 * r;
    double* ac = acc + 16 * r;
    const double t1 = __dadd_rn(ck[0], dt_s);
    const double vmax = sqrt(__longlong_as_double((long long)rd[0]));
    const double tmin = __longlong_as_double((long long)rd[1]);
    double tn = t1;
    if (rd[2] > 0 && vmax * dt_hat < stuck_hat && tmin > t1) {
        const double jump = __dsub_rn(tmin, t1);
        ck[1] = __dadd_rn(ck[1], jump);
        const double jh = jump * time_scale;
        ac[9] = fma(ac[11], jh, ac[9]);
        ac[12] += jh;
        rd[5] += 1;
        tn = tmin;
    }
    ck[0] = tn;
    rd[0] = 0;
    rd[1] = INF_BITS;
    rd[2] = 0;
}

}  // namespace

void junctions_free(ptadd_ctx* ctx)
{
    DevJunctions* j = ctx->junc;
    if (!j) return;
    void* ptrs[] = {j->sess, j->seg, j->last, j->count, j->brk, j->clock, j->red, j->look, j->look_n, j->found};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete j;
    ctx->junc = nullptr;
}

cudaError_t launch_junction_update(ptadd_ctx* ctx, cudaStream_t st)
{
    DevJunctions* j = ctx->junc;
    const DevNetwork& net = ctx->net;
    const int64_t n = net.n_nodes;
    const unsigned nb = (unsigned)((n + JT - 1) / JT);
    junction_release_kernel<<<nb, JT, 0, st>>>(n, net.loop_of, net.pinned, j->seg, j->last, j->brk, j->clock,
                                               j->look, j->look_n, j->found, j->red);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (j->n_free > 0 && j->n_sess > 0) {
        const dim3 grid((unsigned)((j->n_free + JSW - 1) / JSW), (unsigned)((j->n_sess + 31) / 32));
        junction_search_kernel<<<grid, 32 * JSW, 0, st>>>(n, net.pos[net.cur], net.nxt, net.loop_of, j->sess,
                                                          j->n_sess, j->last, j->look, j->look_n, j->found, j->rc2);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    junction_hold_kernel<<<nb, JT, 0, st>>>(n, net.pinned, net.vel, j->sess, j->seg, j->count, j->brk, j->found,
                                            j->clock, j->a, j->seed, j->red);
    return cudaGetLastError();
}

cudaError_t launch_junction_event(ptadd_ctx* ctx, double dt_s, double dt_hat, cudaStream_t st)
{
    DevJunctions* j = ctx->junc;
    junction_event_kernel<<<1, 32, 0, st>>>(j->clock, j->red, ctx->net.acc, j->look_n, dt_s, dt_hat, j->stuck_hat,
                                             ctx->mat.mu / ctx->mat.B);
    return cudaGetLastError();
}

// blob part: seg, last, count (int32 x n each), brk (n doubles), clock[2], red[3..5]
size_t junction_state_bytes(const ptadd_ctx* ctx)
{
    const int64_t n = ctx->net.n_nodes;
    return (size_t)n * (3 * sizeof(int32_t) + sizeof(double)) + 2 * sizeof(double) + 3 * sizeof(uint64_t);
}

ptadd_status junction_state_get(ptadd_ctx* ctx, char* dst)
{
    DevJunctions* j = ctx->junc;
    const size_t n = (size_t)ctx->net.n_nodes;
    cudaStream_t s = ctx->stream;
    PTADD_CUDA(cudaMemcpyAsync(dst, j->seg, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PTADD_CUDA(cudaMemcpyAsync(dst + n * 4, j->last, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PTADD_CUDA(cudaMemcpyAsync(dst + n * 8, j->count, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PTADD_CUDA(cudaMemcpyAsync(dst + n * 12, j->brk, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    PTADD_CUDA(cudaMemcpyAsync(dst + n * 20, j->clock, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    PTADD_CUDA(cudaMemcpyAsync(dst + n * 20 + 16, j->red + 3, 3 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    PTADD_CUDA(cudaStreamSynchronize(s));
    return PTADD_OK;
}

ptadd_status junction_state_set(ptadd_ctx* ctx, const char* src)
{
    DevJunctions* j = ctx->junc;
    const size_t n = (size_t)ctx->net.n_nodes;
    cudaStream_t s = ctx->stream;
    PTADD_CUDA(cudaMemcpyAsync(j->seg, src, n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    PTADD_CUDA(cudaMemcpyAsync(j->last, src + n * 4, n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    PTADD_CUDA(cudaMemcpyAsync(j->count, src + n * 8, n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    PTADD_CUDA(cudaMemcpyAsync(j->brk, src + n * 12, n * sizeof(double), cudaMemcpyHostToDevice, s));
    PTADD_CUDA(cudaMemcpyAsync(j->clock, src + n * 20, 2 * sizeof(double), cudaMemcpyHostToDevice, s));
    PTADD_CUDA(cudaMemcpyAsync(j->red + 3, src + n * 20 + 16, 3 * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    PTADD_CUDA(cudaStreamSynchronize(s));
    return PTADD_OK;
}

struct DevBatchJunctions {
    double rc2 = 0, a = 0, stuck_hat = 0;
    float rc_f = 0;
    uint64_t seed = 0;
    int32_t R = 0;
    int64_t n = 0;
    int32_t* sess = nullptr;        // sessile segments, by realisation, ascending
    int32_t* sess_off = nullptr;    // [R + 1]
    int32_t* free_nodes = nullptr;  // unpinned nodes, by realisation, ascending
    int32_t* items = nullptr;       // [3 n_items]: realisation, first free-list entry, count (<= JB)
    int n_items = 0;
    int32_t* seg = nullptr;    // per node: held sessile segment (global node number) or -1
    int32_t* last = nullptr;   // per node: sessile loop last broken from (global loop number) or -1
    int32_t* count = nullptr;  // per node: junctions formed
    int32_t* found = nullptr;  // per node: this step's capture (sessile list position) or INT32_MAX
    double* brk = nullptr;     // per node: break time on its realisation's clock, s
    double* clock = nullptr;   // [2R]: DD time, time jumped (s)
    unsigned long long* red = nullptr;  // [6R]: as DevJunctions::red, per realisation
    std::vector<int64_t> loop_base;     // first loop of each realisation (host)
};

void batch_junctions_free(DevBatchJunctions*& j)
{
    if (!j) return;
    void* ptrs[] = {j->sess, j->sess_off, j->free_nodes, j->items, j->seg, j->last,
                    j->count, j->found, j->brk, j->clock, j->red};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete j;
    j = nullptr;
}

ptadd_status batch_junctions_create(DevBatchJunctions** out, const ptadd_junction_params* p, double len_unit,
                                    int32_t R, const std::vector<int64_t>& node_off, const std::vector<uint8_t>& pin,
                                    const std::vector<int32_t>& nxt, const std::vector<int32_t>& loop_of)
{
    *out = nullptr;
    const int64_t n = node_off[R];
    std::vector<int32_t> sess, sess_off(R + 1, 0), freel, items;
    DevBatchJunctions* j = new DevBatchJunctions;
    j->loop_base.assign(R, 0);
    for (int r = 0; r < R; ++r) {
        sess_off[r] = (int32_t)sess.size();
        const size_t f0 = freel.size();
        j->loop_base[r] = loop_of[node_off[r]];
        for (int64_t i = node_off[r]; i < node_off[r + 1]; ++i) {
            if (pin[i] && pin[nxt[i]]) sess.push_back((int32_t)i);
            if (!pin[i]) freel.push_back((int32_t)i);
        }
        for (size_t f = f0; f < freel.size(); f += JB) {
            items.push_back(r);
            items.push_back((int32_t)f);
            items.push_back((int32_t)std::min<size_t>(JB, freel.size() - f));
        }
    }
    sess_off[R] = (int32_t)sess.size();
    j->rc2 = (p->capture_radius / len_unit) * (p->capture_radius / len_unit);
    j->rc_f = (float)(p->capture_radius / len_unit);
    j->a = p->max_break_time;
    j->stuck_hat = p->stuck_disp / len_unit;
    j->seed = p->seed;
    j->R = R;
    j->n = n;
    j->n_items = (int)(items.size() / 3);
    cudaError_t e = cudaSuccess;
    auto al = [&](void** q, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(q, bytes > 0 ? bytes : 1);
    };
    al((void**)&j->sess, sess.size() * sizeof(int32_t));
    al((void**)&j->sess_off, sess_off.size() * sizeof(int32_t));
    al((void**)&j->free_nodes, freel.size() * sizeof(int32_t));
    al((void**)&j->items, items.size() * sizeof(int32_t));
    al((void**)&j->seg, n * sizeof(int32_t));
    al((void**)&j->last, n * sizeof(int32_t));
    al((void**)&j->count, n * sizeof(int32_t));
    al((void**)&j->found, n * sizeof(int32_t));
    al((void**)&j->brk, n * sizeof(double));
    al((void**)&j->clock, 2 * (size_t)R * sizeof(double));
    al((void**)&j->red, 6 * (size_t)R * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        set_error("ptadd_batch_set_junctions: cudaMalloc failed: %s", cudaGetErrorString(e));
        batch_junctions_free(j);
        return PTADD_ERR_NOMEM;
    }
    std::vector<unsigned long long> red0(6 * (size_t)R, 0ull);
    for (int r = 0; r < R; ++r) red0[6 * r + 1] = INF_BITS;
    auto chk = [&](cudaError_t c) {
        if (e == cudaSuccess) e = c;
    };
    auto up = [&](void* d, const void* h, size_t bytes) {
        if (bytes) chk(cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice));
    };
    up(j->sess, sess.data(), sess.size() * sizeof(int32_t));
    up(j->sess_off, sess_off.data(), sess_off.size() * sizeof(int32_t));
    up(j->free_nodes, freel.data(), freel.size() * sizeof(int32_t));
    up(j->items, items.data(), items.size() * sizeof(int32_t));
    up(j->red, red0.data(), red0.size() * sizeof(unsigned long long));
    chk(cudaMemset(j->seg, 0xFF, n * sizeof(int32_t)));  // -1
    chk(cudaMemset(j->last, 0xFF, n * sizeof(int32_t)));
    chk(cudaMemset(j->count, 0, n * sizeof(int32_t)));
    {
        const std::vector<int32_t> none(n, INT32_MAX);  // no capture
        up(j->found, none.data(), n * sizeof(int32_t));
    }
    chk(cudaMemset(j->brk, 0, n * sizeof(double)));
    chk(cudaMemset(j->clock, 0, 2 * (size_t)R * sizeof(double)));
    if (e != cudaSuccess) {
        set_error("ptadd_batch_set_junctions: initialising the junction state failed: %s", cudaGetErrorString(e));
        batch_junctions_free(j);
        return PTADD_ERR_CUDA;
    }
    *out = j;
    return PTADD_OK;
}

cudaError_t launch_batch_junction_update(DevBatchJunctions* j, const double* pos, const float* src32,
                                         const int32_t* nxt, const int32_t* loop_of, const int32_t* real_of,
                                         const int64_t* node_off_dev, const uint8_t* pinned, double* vel,
                                         cudaStream_t st)
{
    const int64_t n = j->n;
    const unsigned nb = (unsigned)((n + JT - 1) / JT);
    bj_release_kernel<<<nb, JT, 0, st>>>(n, real_of, loop_of, pinned, j->seg, j->last, j->brk, j->clock, j->red);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (j->n_items > 0) {
        bj_search_kernel<<<(unsigned)j->n_items, JB, 0, st>>>(pos, n, nxt, loop_of, src32, j->sess, j->sess_off,
                                                            j->free_nodes, j->items, j->seg, j->last, j->found,
                                                            j->rc2, j->rc_f);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    bj_hold_kernel<<<nb, JT, 0, st>>>(n, real_of, node_off_dev, pinned, vel, j->sess, j->seg, j->count, j->brk,
                                      j->found, j->clock, j->a, j->seed, j->red);
    return cudaGetLastError();
}

cudaError_t launch_batch_junction_event(DevBatchJunctions* j, double* acc, double dt_s, double dt_hat,
                                        double time_scale, cudaStream_t st)
{
    bj_event_kernel<<<(unsigned)((j->R + 127) / 128), 128, 0, st>>>(j->R, j->clock, j->red, acc, dt_s, dt_hat,
                                                                    j->stuck_hat, time_scale);
    return cudaGetLastError();
}

ptadd_status batch_junctions_get(DevBatchJunctions* j, const std::vector<int64_t>& node_off, cudaStream_t s,
                                 ptadd_junction_info* info, int32_t* seg, int32_t* last, int32_t* count,
                                 double* break_time)
{
    const int64_t n = j->n;
    const int R = j->R;
    std::vector<int32_t> sg(n), ls(n);
    std::vector<double> clock(2 * (size_t)R);
    std::vector<unsigned long long> red(6 * (size_t)R);
    PTADD_CUDA(cudaMemcpyAsync(sg.data(), j->seg, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PTADD_CUDA(cudaMemcpyAsync(ls.data(), j->last, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PTADD_CUDA(cudaMemcpyAsync(clock.data(), j->clock, clock.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    PTADD_CUDA(cudaMemcpyAsync(red.data(), j->red, red.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    if (count) PTADD_CUDA(cudaMemcpyAsync(count, j->count, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (break_time) PTADD_CUDA(cudaMemcpyAsync(break_time, j->brk, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    PTADD_CUDA(cudaStreamSynchronize(s));
    for (int r = 0; r < R; ++r) {
        int64_t held = 0;
        for (int64_t i = node_off[r]; i < node_off[r + 1]; ++i) {
            held += sg[i] >= 0;
            if (seg) seg[i] = sg[i] >= 0 ? (int32_t)(sg[i] - node_off[r]) : -1;
            if (last) last[i] = ls[i] >= 0 ? (int32_t)(ls[i] - j->loop_base[r]) : -1;
        }
        if (info) {
            info[r].clock = clock[2 * r];
            info[r].jumped = clock[2 * r + 1];
            info[r].held = held;
            info[r].formed = (int64_t)red[6 * r + 3];
            info[r].broken = (int64_t)red[6 * r + 4];
            info[r].jumps = (int64_t)red[6 * r + 5];
        }
    }
    return PTADD_OK;
}

}  // namespace ptadd

using namespace ptadd;

extern "C" ptadd_status ptadd_set_junctions(ptadd_ctx* ctx, const ptadd_junction_params* p)
{
    if (!ctx) {
        set_error("ptadd_set_junctions: null context");
        return PTADD_ERR_ARG;
    }
    PTADD_CUDA(cudaSetDevice(ctx->device));
    if (!ctx->have_net) {
        set_error("ptadd_set_junctions: no network loaded");
        return PTADD_ERR_STATE;
    }
    if (p && ctx->consistent_mass) {
        set_error("ptadd_set_junctions: junctions need the lumped mobility (ptadd_set_mobility(ctx, 0))");
        return PTADD_ERR_STATE;
    }
    if (p && !(p->capture_radius >= 0.0 && isfinite(p->capture_radius) && p->max_break_time >= 0.0 &&
               isfinite(p->max_break_time) && p->stuck_disp >= 0.0 && isfinite(p->stuck_disp))) {
        set_error("ptadd_set_junctions: parameters must be non-negative and finite");
        return PTADD_ERR_ARG;
    }
    PTADD_CUDA(cudaStreamSynchronize(ctx->stream));
    junctions_free(ctx);
    if (!p) return PTADD_OK;
    const DevNetwork& net = ctx->net;
    const int64_t n = net.n_nodes;
    std::vector<uint8_t> pin(n);
    std::vector<int32_t> nxt(n);
    PTADD_CUDA(cudaMemcpy(pin.data(), net.pinned, n, cudaMemcpyDeviceToHost));
    PTADD_CUDA(cudaMemcpy(nxt.data(), net.nxt, n * sizeof(int32_t), cudaMemcpyDeviceToHost));
    std::vector<int32_t> sess;
    int64_t n_free = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (pin[i] && pin[nxt[i]]) sess.push_back((int32_t)i);
        n_free += pin[i] ? 0 : 1;
    }

    DevJunctions* j = new DevJunctions;
    ctx->junc = j;
    const double l = ctx->len_unit;
    j->rc2 = (p->capture_radius / l) * (p->capture_radius / l);
    j->a = p->max_break_time;
    j->stuck_hat = p->stuck_disp / l;
    j->seed = p->seed;
    j->n_sess = (int64_t)sess.size();
    j->n_free = n_free;
    cudaError_t e = cudaSuccess;
    auto al = [&](void** q, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(q, bytes > 0 ? bytes : 1);
    };
    al((void**)&j->sess, sess.size() * sizeof(int32_t));
    al((void**)&j->seg, n * sizeof(int32_t));
    al((void**)&j->last, n * sizeof(int32_t));
    al((void**)&j->count, n * sizeof(int32_t));
    al((void**)&j->brk, n * sizeof(double));
    al((void**)&j->clock, 2 * sizeof(double));
    al((void**)&j->red, 6 * sizeof(unsigned long long));
    al((void**)&j->look, (size_t)n * sizeof(int32_t));
    al((void**)&j->look_n, sizeof(unsigned));
    al((void**)&j->found, (size_t)n * sizeof(int32_t));
    if (e != cudaSuccess) {
        set_error("ptadd_set_junctions: cudaMalloc failed: %s", cudaGetErrorString(e));
        junctions_free(ctx);
        return PTADD_ERR_NOMEM;
    }
    const unsigned long long red0[6] = {0ull, INF_BITS, 0ull, 0ull, 0ull, 0ull};
    const double clock0[2] = {0.0, 0.0};
    auto chk = [&](cudaError_t r) {
        if (e == cudaSuccess) e = r;
    };
    if (!sess.empty()) chk(cudaMemcpy(j->sess, sess.data(), sess.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    chk(cudaMemset(j->seg, 0xFF, n * sizeof(int32_t)));  // -1
    chk(cudaMemset(j->last, 0xFF, n * sizeof(int32_t)));
    chk(cudaMemset(j->count, 0, n * sizeof(int32_t)));
    chk(cudaMemset(j->brk, 0, n * sizeof(double)));
    chk(cudaMemcpy(j->clock, clock0, sizeof(clock0), cudaMemcpyHostToDevice));
    chk(cudaMemcpy(j->red, red0, sizeof(red0), cudaMemcpyHostToDevice));
    chk(cudaMemset(j->look_n, 0, sizeof(unsigned)));
    if (e != cudaSuccess) {  // leave junctions off rather than half set
        set_error("ptadd_set_junctions: initialising the junction state failed: %s", cudaGetErrorString(e));
        junctions_free(ctx);
        return PTADD_ERR_CUDA;
    }
    return PTADD_OK;
}

extern "C" ptadd_status ptadd_get_junctions(ptadd_ctx* ctx, ptadd_junction_info* info, int32_t* seg, int32_t* last,
                                            int32_t* count, double* break_time)
{
    if (!ctx) {
        set_error("ptadd_get_junctions: null context");
        return PTADD_ERR_ARG;
    }
    PTADD_CUDA(cudaSetDevice(ctx->device));
    DevJunctions* j = ctx->junc;
    if (!ctx->have_net || !j) {
        set_error("ptadd_get_junctions: junctions are off");
        return PTADD_ERR_STATE;
    }
    const size_t n = (size_t)ctx->net.n_nodes;
    cudaStream_t s = ctx->stream;
    std::vector<int32_t> sg(n);
    double clock[2];
    unsigned long long red[6];
    PTADD_CUDA(cudaMemcpyAsync(sg.data(), j->seg, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PTADD_CUDA(cudaMemcpyAsync(clock, j->clock, sizeof(clock), cudaMemcpyDeviceToHost, s));
    PTADD_CUDA(cudaMemcpyAsync(red, j->red, sizeof(red), cudaMemcpyDeviceToHost, s));
    if (last) PTADD_CUDA(cudaMemcpyAsync(last, j->last, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (count) PTADD_CUDA(cudaMemcpyAsync(count, j->count, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (break_time) PTADD_CUDA(cudaMemcpyAsync(break_time, j->brk, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    PTADD_CUDA(cudaStreamSynchronize(s));
    if (seg) memcpy(seg, sg.data(), n * sizeof(int32_t));
    if (info) {
        int64_t held = 0;
        for (size_t i = 0; i < n; ++i) held += sg[i] >= 0;
        info->clock = clock[0];
        info->jumped = clock[1];
        info->held = held;
        info->formed = (int64_t)red[3];
        info->broken = (int64_t)red[4];
        info->jumps = (int64_t)red[5];
    }
    return PTADD_OK;
}
