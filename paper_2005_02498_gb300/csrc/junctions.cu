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
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

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
