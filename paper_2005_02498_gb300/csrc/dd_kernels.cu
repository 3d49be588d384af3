// dd_kernels.cu -- one explicit DD step on the GPU (Sec. 2.1 of the paper):
//   seg_prep      : per-segment source records from the current positions
//   pair_fp64     : O(N^2) stress at the 4 Gauss points of every target
//                   segment, contracted with its Burgers vector, folded into
//                   the two nodal force parts of the segment (PK force, linear
//                   shape functions)
//   node_velocity : nodal force = own part + previous segment's part,
//                   glide-projected lumped mobility
//   lp_euler      : Lp / rho sample of the step-start state (Sec. 2.2, 2.4),
//                   explicit Euler into the other position buffer, block
//                   partial sums; lp_finish sums them in a fixed order into
//                   the running averages of Eq. 2.5.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <math.h>

#include "pair_tile.cuh"
#include "ptadd_internal.cuh"
#include "seg_field.cuh"

namespace ptadd {

// ----------------------------------------------------------- seg_prep
__global__ void seg_prep_kernel(int64_t n, const double* __restrict__ pos, const int32_t* __restrict__ nxt,
                                const int32_t* __restrict__ loop_of, const double* __restrict__ loop_b,
                                double* __restrict__ src, float* __restrict__ src32, double ox, double oy, double oz)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t j = nxt[i];
    const double x1 = pos[i], y1 = pos[n + i], z1 = pos[2 * n + i];
    const double dx = pos[j] - x1, dy = pos[n + j] - y1, dz = pos[2 * n + j] - z1;
    const double L = sqrt(dx * dx + dy * dy + dz * dz);
    const int k = loop_of[i];
    double bx = loop_b[3 * k], by = loop_b[3 * k + 1], bz = loop_b[3 * k + 2];
    double tx = 1.0, ty = 0.0, tz = 0.0;
    if (L > 0.0) {
        tx = dx / L;
        ty = dy / L;
        tz = dz / L;
    }
    double* r = src + (int64_t)SRC_STRIDE * i;
    r[0] = x1; r[1] = y1; r[2] = z1; r[3] = L;
    r[4] = tx; r[5] = ty; r[6] = tz; r[7] = 0.0;
    r[8] = bx; r[9] = by; r[10] = bz; r[11] = 0.0;
    r[12] = by * tz - bz * ty;
    r[13] = bz * tx - bx * tz;
    r[14] = bx * ty - by * tx;
    r[15] = 0.0;
    if (src32) {
        float* f = src32 + (int64_t)SRC32_STRIDE * i;
        const double rx = x1 - ox, ry = y1 - oy, rz = z1 - oz;
        const double hx = rint(rx), hy = rint(ry), hz = rint(rz);
        f[0] = (float)hx; f[1] = (float)hy; f[2] = (float)hz;
        f[3] = (float)(rx - hx); f[4] = (float)(ry - hy); f[5] = (float)(rz - hz);
        f[6] = (float)L;
        f[7] = (float)tx; f[8] = (float)ty; f[9] = (float)tz;
        f[10] = (float)bx; f[11] = (float)by; f[12] = (float)bz;
        f[13] = (float)r[12]; f[14] = (float)r[13]; f[15] = (float)r[14];
    }
}

cudaError_t launch_seg_prep(const DevNetwork& net, cudaStream_t st)
{
    const int64_t n = net.n_nodes;
    if (n == 0) return cudaSuccess;
    seg_prep_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, net.pos[net.cur], net.nxt, net.loop_of,
                                                                  net.loop_b, net.src, net.src32, net.origin[0],
                                                                  net.origin[1], net.origin[2]);
    return cudaGetLastError();
}

// ------------------------------------------------------------ pair stage
// Grid: x = target tiles of PAIR_TPB threads (one target segment each),
//       y = source chunks.  Each block runs one tile (pair_tile.cuh): it
// stages source records through shared memory; every thread walks them in the
// same order (broadcast reads) and accumulates (sigma b') at its 4 Gauss points.
constexpr int PAIR_TPB = 128;
constexpr int PAIR_TILE = 128;
constexpr int MIX_TPB = 128;
constexpr int MIX_TILE = 192;  // sources per staged tile: 3 blocks of 66.5 KB fit one SM's shared memory
constexpr int MIX_MINB = 3;  // resident blocks per SM the register budget is sized for

__global__ void __launch_bounds__(PAIR_TPB) pair_fp64_kernel(TileArgs base, int64_t n_tgt, int64_t chunk_len,
                                                             Consts c)
{
    __shared__ double2 tile[PAIR_TILE * SRC_STRIDE / 2];
    TileArgs a = base;
    a.t_begin = (int64_t)blockIdx.x * PAIR_TPB;
    a.t_count = min((int64_t)PAIR_TPB, n_tgt - a.t_begin);
    a.js = (int64_t)blockIdx.y * chunk_len;
    a.je = min(a.n, a.js + chunk_len);
    a.add_app = blockIdx.y == 0;
    a.fp = base.fp + (int64_t)blockIdx.y * 6 * a.n;
    pair_tile_fp64<PAIR_TILE>(a, c, tile);
}

__global__ void __launch_bounds__(MIX_TPB, MIX_MINB) pair_mixed_kernel(TileArgs base, int64_t n_tgt, int64_t chunk_len,
                                                             Consts c, float near2)
{
    __shared__ MixSmem<MIX_TILE, MIX_TPB> sm;
    TileArgs a = base;
    a.t_begin = (int64_t)blockIdx.x * MIX_TPB;
    a.t_count = min((int64_t)MIX_TPB, n_tgt - a.t_begin);
    a.js = (int64_t)blockIdx.y * chunk_len;
    a.je = min(a.n, a.js + chunk_len);
    a.add_app = blockIdx.y == 0;
    a.fp = base.fp + (int64_t)blockIdx.y * 6 * a.n;
    pair_tile_mixed<MIX_TILE, MIX_TPB>(a, c, near2, sm);
}

int choose_chunks(int64_t n_tgt, int64_t n_src, int max_chunks, int precision)
{
    // About 16 waves of resident blocks, so that the blocks still running
    // when the others have finished (the tail) cost a few per cent; chunks of
    // at least two source tiles, so the per-block set-up and the nodal
    // output stay small next to the pair work, unless that leaves less than
    // one wave (a small network): then chunks down to 32 sources, so that the
    // few targets' work (and their FP64 near pairs) spreads over more SMs.
    // The device queries are made once per device and precision.
    static std::atomic<int> cached[64][2][2];  // [device][mixed] -> {sms, blocks per SM}; 0: not yet
    int dev = 0, sms = 152, per_sm = 2;
    const int mixed = precision == (int)PTADD_MIXED ? 1 : 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 &&
        cached[dev][mixed][0].load(std::memory_order_acquire) > 0) {
        sms = cached[dev][mixed][0].load(std::memory_order_relaxed);
        per_sm = cached[dev][mixed][1].load(std::memory_order_relaxed);
    } else {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (mixed)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pair_mixed_kernel, MIX_TPB, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pair_fp64_kernel, PAIR_TPB, 0);
        if (per_sm < 1) per_sm = 1;
        if (dev >= 0 && dev < 64) {
            cached[dev][mixed][1].store(per_sm, std::memory_order_relaxed);
            cached[dev][mixed][0].store(sms, std::memory_order_release);
        }
    }
    const int64_t tiles_t = (n_tgt + PAIR_TPB - 1) / PAIR_TPB;
    int64_t cap = n_src / (2 * PAIR_TILE);
    if (tiles_t * cap < (int64_t)sms * per_sm) cap = std::max<int64_t>(cap, n_src / 32);
    if (cap > max_chunks) cap = max_chunks;
    if (cap < 1) cap = 1;
    const int64_t want_blocks = (int64_t)sms * per_sm * 16;
    int64_t ch = (want_blocks + tiles_t - 1) / (tiles_t > 0 ? tiles_t : 1);
    if (ch > cap) ch = cap;
    if (ch < 1) ch = 1;
    return (int)ch;
}

cudaError_t launch_pair(const DevNetwork& net, const int32_t* tgt, int64_t n_tgt, int chunks, int precision,
                        const Consts& c, const double sh[6], cudaStream_t st)
{
    const int64_t n = net.n_nodes;
    if (n_tgt == 0 || n == 0) return cudaSuccess;
    const int64_t chunk_len = (n + chunks - 1) / chunks;
    TileArgs a{};
    a.pos = net.pos[net.cur];
    a.n = n;
    a.nxt = net.nxt;
    a.src = net.src;
    a.src32 = net.src32;
    a.tgt = tgt;
    for (int k = 0; k < 6; ++k) a.sh[k] = sh[k];
    for (int k = 0; k < 3; ++k) a.origin[k] = net.origin[k];
    a.fp = net.fpart;
    a.fp_stride = n;
    a.node_base = 0;
    a.near_count = net.near_count;
    a.k64 = net.k64;
    if (precision == (int)PTADD_MIXED) {
        dim3 grid((unsigned)((n_tgt + MIX_TPB - 1) / MIX_TPB), (unsigned)chunks);
        const float near2 = (float)((NEAR_FACTOR * NEAR_FACTOR + 1.0) * c.a2);
        pair_mixed_kernel<<<grid, MIX_TPB, 0, st>>>(a, n_tgt, chunk_len, c, near2);
        return cudaGetLastError();
    }
    dim3 grid((unsigned)((n_tgt + PAIR_TPB - 1) / PAIR_TPB), (unsigned)chunks);
    pair_fp64_kernel<<<grid, PAIR_TPB, 0, st>>>(a, n_tgt, chunk_len, c);
    return cudaGetLastError();
}

// ------------------------------------------------------- node_velocity
__global__ void node_velocity_kernel(int64_t n, const double* __restrict__ pos, const int32_t* __restrict__ nxt,
                                     const int32_t* __restrict__ prv, const int32_t* __restrict__ loop_of,
                                     const double* __restrict__ loop_n, const uint8_t* __restrict__ pinned,
                                     const double* __restrict__ fpart, int chunks, double* __restrict__ force,
                                     double* __restrict__ vel)
{
    const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n) return;
    const int64_t p = prv[a], nx = nxt[a];
    double F[3] = {0, 0, 0};
    for (int ch = 0; ch < chunks; ++ch) {
        const double* fp = fpart + (int64_t)ch * 6 * n;
        F[0] += fp[0 * n + a] + fp[3 * n + p];
        F[1] += fp[1 * n + a] + fp[4 * n + p];
        F[2] += fp[2 * n + a] + fp[5 * n + p];
    }
    const double xa = pos[a], ya = pos[n + a], za = pos[2 * n + a];
    const double px = xa - pos[p], py = ya - pos[n + p], pz = za - pos[2 * n + p];
    const double qx = pos[nx] - xa, qy = pos[n + nx] - ya, qz = pos[2 * n + nx] - za;
    const double M = 0.5 * (sqrt(px * px + py * py + pz * pz) + sqrt(qx * qx + qy * qy + qz * qz));
    const int k = loop_of[a];
    const double nn[3] = {loop_n[3 * k], loop_n[3 * k + 1], loop_n[3 * k + 2]};
    double v[3] = {0, 0, 0};
    if (!(pinned && pinned[a]) && M > 0.0) {
        const double nF = nn[0] * F[0] + nn[1] * F[1] + nn[2] * F[2];
        v[0] = (F[0] - nn[0] * nF) / M;
        v[1] = (F[1] - nn[1] * nF) / M;
        v[2] = (F[2] - nn[2] * nF) / M;
    }
    force[a] = F[0]; force[n + a] = F[1]; force[2 * n + a] = F[2];
    vel[a] = v[0]; vel[n + a] = v[1]; vel[2 * n + a] = v[2];
}

cudaError_t launch_node_velocity(const DevNetwork& net, int chunks, cudaStream_t st)
{
    const int64_t n = net.n_nodes;
    if (n == 0) return cudaSuccess;
    node_velocity_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, net.pos[net.cur], net.nxt, net.prv,
                                                                       net.loop_of, net.loop_n, net.pinned,
                                                                       net.fpart, chunks, net.force, net.vel);
    return cudaGetLastError();
}

// ------------------------------------------------- consistent mobility
// Eq. 2.1's weak form with linear shape functions N_a, per loop (internal
// units, B = 1): sum_b M_ab v_b = P F_a with M_ab = int N_a N_b dl, i.e.
// M_aa = (L_prev + L_next)/3 and M_a,a+1 = L/6 of the segment between them;
// v = 0 at pinned nodes and at a free node whose two segments have zero
// length (held, Dirichlet).  One thread per loop: each chain of free nodes
// between held ones is a tridiagonal system (Thomas elimination); a loop with
// no held node is cyclic (the Sherman-Morrison form of the elimination, with
// the corner terms as a rank-one correction); a two-node loop is solved
// directly.  The matrix is diagonally dominant (M_aa = 2 (M_a,a-1 +
// M_a,a+1)), so no pivoting is needed.  scr: [5 n] per-node factors.
__device__ __forceinline__ double seg_len(const double* __restrict__ pos, int64_t n, int64_t i, int64_t j)
{
    const double dx = pos[j] - pos[i], dy = pos[n + j] - pos[n + i], dz = pos[2 * n + j] - pos[2 * n + i];
    return sqrt(dx * dx + dy * dy + dz * dz);
}

__global__ void consistent_velocity_kernel(int64_t n_loops, const int64_t* __restrict__ loop_off,
                                           const double* __restrict__ pos, int64_t n,
                                           const double* __restrict__ force, const uint8_t* __restrict__ pinned,
                                           const double* __restrict__ loop_n, double* __restrict__ vel,
                                           double* __restrict__ scr)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n_loops) return;
    const int64_t b = loop_off[k], m = loop_off[k + 1] - b;
    const double nn[3] = {loop_n[3 * k], loop_n[3 * k + 1], loop_n[3 * k + 2]};
    // ring helpers: node t of the loop (0 <= t < m) is global b + t
    auto node = [&](int64_t t) { return b + (t % m + m) % m; };
    auto Lseg = [&](int64_t t) { return seg_len(pos, n, node(t), node(t + 1)); };  // segment t -> t+1
    auto held = [&](int64_t t) { return pinned[node(t)] != 0 || !(Lseg(t - 1) + Lseg(t) > 0.0); };
    auto rhs = [&](int64_t t, double d[3]) {  // P F
        const int64_t a = node(t);
        const double F[3] = {force[a], force[n + a], force[2 * n + a]};
        const double nF = nn[0] * F[0] + nn[1] * F[1] + nn[2] * F[2];
        for (int c = 0; c < 3; ++c) d[c] = F[c] - nn[c] * nF;
    };
    auto put = [&](int64_t t, const double v[3]) {
        const int64_t a = node(t);
        vel[a] = v[0];
        vel[n + a] = v[1];
        vel[2 * n + a] = v[2];
    };
    double* cp = scr;          // c' of the elimination
    double* dp = scr + n;      // d' (3 components)
    double* zp = scr + 4 * n;  // d' of the rank-one correction
    int64_t h = -1;
    for (int64_t t = 0; t < m && h < 0; ++t)
        if (held(t)) h = t;
    if (h < 0 && m == 2) {
        const double S = Lseg(0) + Lseg(1), p = S / 3.0, q = S / 6.0, det = p * p - q * q;
        double d0[3], d1[3], v0[3], v1[3];
        rhs(0, d0);
        rhs(1, d1);
        for (int c = 0; c < 3; ++c) {
            v0[c] = (p * d0[c] - q * d1[c]) / det;
            v1[c] = (p * d1[c] - q * d0[c]) / det;
        }
        put(0, v0);
        put(1, v1);
        return;
    }
    if (h < 0) {
        // cyclic: rows a_t x_{t-1} + b_t x_t + c_t x_{t+1} = d_t; corners
        // beta = a_0 (row 0, column m-1) and alpha = c_{m-1} (row m-1, column 0)
        const double L0 = Lseg(0), Lm = Lseg(m - 1);
        const double b0 = (Lm + L0) / 3.0, beta = Lm / 6.0, alpha = Lm / 6.0;
        const double gam = -b0;
        double Lprev = Lm;
        for (int64_t t = 0; t < m; ++t) {
            const double Lt = Lseg(t);
            double bt = (Lprev + Lt) / 3.0;
            if (t == 0) bt -= gam;
            if (t == m - 1) bt -= alpha * beta / gam;
            const double at = t > 0 ? Lprev / 6.0 : 0.0, ct = t < m - 1 ? Lt / 6.0 : 0.0;
            const int64_t a = node(t), ap = node(t - 1);
            const double den = t > 0 ? bt - at * cp[ap] : bt;
            double d[3];
            rhs(t, d);
            const double u = t == 0 ? gam : (t == m - 1 ? alpha : 0.0);
            cp[a] = ct / den;
            for (int c = 0; c < 3; ++c) dp[c * n + a] = (d[c] - (t > 0 ? at * dp[c * n + ap] : 0.0)) / den;
            zp[a] = (u - (t > 0 ? at * zp[ap] : 0.0)) / den;
            Lprev = Lt;
        }
        for (int64_t t = m - 2; t >= 0; --t) {  // back substitution, in place
            const int64_t a = node(t), an = node(t + 1);
            for (int c = 0; c < 3; ++c) dp[c * n + a] -= cp[a] * dp[c * n + an];
            zp[a] -= cp[a] * zp[an];
        }
        const int64_t a0 = node(0), am = node(m - 1);
        const double den = 1.0 + zp[a0] + beta * zp[am] / gam;
        double f[3];
        for (int c = 0; c < 3; ++c) f[c] = (dp[c * n + a0] + beta * dp[c * n + am] / gam) / den;
        for (int64_t t = 0; t < m; ++t) {
            const int64_t a = node(t);
            const double v[3] = {dp[a] - f[0] * zp[a], dp[n + a] - f[1] * zp[a], dp[2 * n + a] - f[2] * zp[a]};
            put(t, v);
        }
        return;
    }
    // chains of free nodes between held ones, walking the ring from h
    const double zero[3] = {0.0, 0.0, 0.0};
    int64_t t = h;
    for (int64_t done = 0; done < m;) {
        if (held(t)) {
            put(t, zero);
            ++t;
            ++done;
            continue;
        }
        // a chain starts at t (its predecessor is held); forward elimination
        int64_t r = 0;
        double Lprev = Lseg(t - 1);
        while (!held(t + r) && done + r < m) {
            const double Lt = Lseg(t + r);
            const double bt = (Lprev + Lt) / 3.0;
            const double at = r > 0 ? Lprev / 6.0 : 0.0;
            const bool last = held(t + r + 1) || done + r + 1 >= m;
            const double ct = last ? 0.0 : Lt / 6.0;
            const int64_t a = node(t + r), ap = node(t + r - 1);
            const double den = r > 0 ? bt - at * cp[ap] : bt;
            double d[3];
            rhs(t + r, d);
            cp[a] = ct / den;
            for (int c = 0; c < 3; ++c) dp[c * n + a] = (d[c] - (r > 0 ? at * dp[c * n + ap] : 0.0)) / den;
            Lprev = Lt;
            ++r;
        }
        // back substitution
        for (int64_t q = r - 1; q >= 0; --q) {
            const int64_t a = node(t + q);
            double v[3];
            for (int c = 0; c < 3; ++c) {
                v[c] = dp[c * n + a];
                if (q < r - 1) v[c] -= cp[a] * dp[c * n + node(t + q + 1)];
                dp[c * n + a] = v[c];
            }
            put(t + q, v);
        }
        t += r;
        done += r;
    }
}

cudaError_t launch_consistent_velocity_raw(int64_t n_loops, const int64_t* loop_off, const double* pos, int64_t n,
                                           const double* force, const uint8_t* pinned, const double* loop_n,
                                           double* vel, double* scr, cudaStream_t st)
{
    if (n_loops == 0) return cudaSuccess;
    consistent_velocity_kernel<<<(unsigned)((n_loops + 127) / 128), 128, 0, st>>>(n_loops, loop_off, pos, n, force,
                                                                                  pinned, loop_n, vel, scr);
    return cudaGetLastError();
}

cudaError_t launch_consistent_velocity(const DevNetwork& net, cudaStream_t st)
{
    return launch_consistent_velocity_raw(net.n_loops, net.loop_off, net.pos[net.cur], net.n_nodes, net.force,
                                          net.pinned, net.loop_n, net.vel, net.cm_scratch, st);
}

// ------------------------------------------------------------ lp_euler
constexpr int RED_TPB = 256;
// per-segment sums of the step-start state: L b (x) (t x vbar) (9), L (1),
// L vbar (3, the polar-velocity sum of Eq. 2.11 without A / |B|)
constexpr int NSUM = 13;

__global__ void __launch_bounds__(RED_TPB) lp_euler_kernel(
    int64_t n, const double* __restrict__ pos, double* __restrict__ pos_next, const int32_t* __restrict__ nxt,
    const int32_t* __restrict__ loop_of, const double* __restrict__ loop_b, const double* __restrict__ vel,
    double dt, double* __restrict__ partial, int* __restrict__ flag)
{
    __shared__ double red[RED_TPB / 32][NSUM];
    const int64_t i = blockIdx.x * (int64_t)RED_TPB + threadIdx.x;
    double v13[NSUM];
#pragma unroll
    for (int m = 0; m < NSUM; ++m) v13[m] = 0.0;
    if (i < n) {
        const int64_t j = nxt[i];
        const double dx = pos[j] - pos[i], dy = pos[n + j] - pos[n + i], dz = pos[2 * n + j] - pos[2 * n + i];
        const double vx = 0.5 * (vel[i] + vel[j]);
        const double vy = 0.5 * (vel[n + i] + vel[n + j]);
        const double vz = 0.5 * (vel[2 * n + i] + vel[2 * n + j]);
        const double cx = dy * vz - dz * vy, cy = dz * vx - dx * vz, cz = dx * vy - dy * vx;  // L t x vbar
        const int k = loop_of[i];
        const double b0 = loop_b[3 * k], b1 = loop_b[3 * k + 1], b2 = loop_b[3 * k + 2];
        const double L = sqrt(dx * dx + dy * dy + dz * dz);
        v13[0] = b0 * cx; v13[1] = b0 * cy; v13[2] = b0 * cz;
        v13[3] = b1 * cx; v13[4] = b1 * cy; v13[5] = b1 * cz;
        v13[6] = b2 * cx; v13[7] = b2 * cy; v13[8] = b2 * cz;
        v13[9] = L;
        v13[10] = L * vx; v13[11] = L * vy; v13[12] = L * vz;
        // explicit Euler (all nodes from the step-start state)
        const double nxp = __dadd_rn(pos[i], __dmul_rn(vel[i], dt));
        const double nyp = __dadd_rn(pos[n + i], __dmul_rn(vel[n + i], dt));
        const double nzp = __dadd_rn(pos[2 * n + i], __dmul_rn(vel[2 * n + i], dt));
        pos_next[i] = nxp;
        pos_next[n + i] = nyp;
        pos_next[2 * n + i] = nzp;
        if (!isfinite(nxp) || !isfinite(nyp) || !isfinite(nzp)) atomicOr(flag, 1);
    }
#pragma unroll
    for (int m = 0; m < NSUM; ++m) {
        double v = v13[m];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][m] = v;
    }
    __syncthreads();
    if (threadIdx.x < NSUM) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < RED_TPB / 32; ++w) s += red[w][threadIdx.x];
        partial[blockIdx.x * NSUM + threadIdx.x] = s;
    }
}

// One block: sum the per-block partials in a fixed order, add dt-weighted
// into acc[0..9] (Lp, rho) and acc[13..15] (polar velocity).
__global__ void lp_finish_kernel(int nblk, const double* __restrict__ partial, double dt, double* __restrict__ acc)
{
    __shared__ double red[256][NSUM];
    double s[NSUM];
#pragma unroll
    for (int m = 0; m < NSUM; ++m) s[m] = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 256)
#pragma unroll
        for (int m = 0; m < NSUM; ++m) s[m] += partial[b * NSUM + m];
#pragma unroll
    for (int m = 0; m < NSUM; ++m) red[threadIdx.x][m] = s[m];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h)
#pragma unroll
            for (int m = 0; m < NSUM; ++m) red[threadIdx.x][m] += red[threadIdx.x + h][m];
        __syncthreads();
    }
    if (threadIdx.x < 10) acc[threadIdx.x] = fma(red[0][threadIdx.x], dt, acc[threadIdx.x]);
    if (threadIdx.x >= 10 && threadIdx.x < NSUM)
        acc[threadIdx.x + 3] = fma(red[0][threadIdx.x], dt, acc[threadIdx.x + 3]);
    if (threadIdx.x == 9) acc[11] = red[0][9];  // the step's line length (junction jumps weight it)
}

cudaError_t launch_lp_euler(DevNetwork& net, double dt_hat, cudaStream_t st)
{
    const int64_t n = net.n_nodes;
    if (n == 0) return cudaSuccess;
    const int nblk = (int)((n + RED_TPB - 1) / RED_TPB);
    lp_euler_kernel<<<nblk, RED_TPB, 0, st>>>(n, net.pos[net.cur], net.pos[1 - net.cur], net.nxt, net.loop_of,
                                               net.loop_b, net.vel, dt_hat, net.partial, net.flag);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    lp_finish_kernel<<<1, 256, 0, st>>>(nblk, net.partial, dt_hat, net.acc);
    net.cur = 1 - net.cur;
    return cudaGetLastError();
}

}  // namespace ptadd
