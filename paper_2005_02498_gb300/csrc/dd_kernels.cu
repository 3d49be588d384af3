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
constexpr int MIX_TILE = 128;
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
