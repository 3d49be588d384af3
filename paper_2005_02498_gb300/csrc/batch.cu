// batch.cu -- batched ensembles: R independent realisations of uneven size
// advanced together (the independent per-block / per-material-point bursts of
// the paper's coupling, Sec. 4.1, run "in parallel").
//
// Layout: the realisations' nodes are concatenated (realisation r owns nodes
// [node_off[r], node_off[r+1])); every per-node table is indexed globally.
// One DD step is five phases, each one launch (nine with junctions: release,
// capture search and hold after the node phase, the clock event at the end):
//   prep     : source records (FP64 + FP32 hi/lo about the realisation's origin)
//   pair     : PERSISTENT kernel (one block per SM slot) that pulls work tiles
//              (realisation, <= TPB targets, source chunk) from a list sorted
//              by cost, largest first, through one atomic counter, so the
//              256x spread of N_r^2 does not leave SMs idle;
//   node     : nodal force = sum of the chunk parts, glide mobility;
//   lp_euler : per-block partial Lp/rho sums (a block never spans two
//              realisations) and the Euler update;
//   finish   : one block per realisation sums its partials in a fixed order.
// Kernel boundaries order the phases (no device-side barrier, nothing to spin
// on).  Two steps (position buffers 0->1->0) are captured once into a CUDA
// graph and replayed, so a 2000-step burst costs 1000 graph launches.
//
// Autotuner: the tile width (threads per block) and the source-chunk length
// are chosen by timing the pair phase of the loaded batch for each candidate;
// results are kept in a JSON-lines cache keyed by GPU, library version, a
// hash of the sources the library was built from, precision and the batch's
// size class.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <sys/stat.h>

#include <algorithm>
#include <string>
#include <vector>

#include "pair_tile.cuh"
#include "ptadd_internal.cuh"

namespace ptadd {

struct WorkItem {
    int32_t r;        // realisation
    int32_t chunk;    // source chunk index within the realisation
    int32_t t_begin;  // first entry in the target list
    int32_t t_count;  // targets in the tile
    int32_t js, je;   // global source range
};

struct BatchConfig {
    int tpb = 128;         // targets per tile (threads per block)
    int chunk_len = 2048;  // sources per chunk
};

struct DevBatch {
    int32_t R = 0;
    int64_t n = 0, n_loops = 0, n_tgt = 0, pairs = 0;
    double* pos[2] = {nullptr, nullptr};
    int cur = 0;
    int32_t *nxt = nullptr, *prv = nullptr, *loop_of = nullptr, *real_of = nullptr, *tgt = nullptr;
    double *loop_b = nullptr, *loop_n = nullptr;
    uint8_t* pinned = nullptr;
    double* src = nullptr;
    float* src32 = nullptr;
    double *fpart = nullptr, *vel = nullptr, *force = nullptr, *partial = nullptr, *acc = nullptr;
    std::vector<double> last_LV;  // [3R] (1/|B|) sum L vbar of the last burst, time-averaged, SI
    int64_t fpart_cap = 0;  // doubles
    // per realisation (device)
    int64_t* d_node_off = nullptr;
    int64_t* d_fp_base = nullptr;
    int32_t* d_chunks = nullptr;
    double* d_origin = nullptr;  // 3R
    double* d_sh = nullptr;      // 6R
    // lp reduction: block b covers nodes [blk_start[b], blk_start[b] + RED) of realisation blk_real[b]
    int32_t* d_blk_real = nullptr;
    int64_t* d_blk_start = nullptr;
    int32_t* d_real_blk = nullptr;  // R+1
    int nblk = 0;
    WorkItem* d_items = nullptr;
    int n_items = 0;
    unsigned* counter = nullptr;
    int* flag = nullptr;
    unsigned long long* near_count = nullptr;
    double* staging = nullptr;
    double* k64 = nullptr;  // {a2, c1, c2} for the near-field path
    // host copies
    std::vector<int64_t> node_off, tgt_off;
    std::vector<double> volume, origin, sh;
    BatchConfig cfg;
    int tuned = 0;
    // graph of two steps
    cudaGraphExec_t graph = nullptr;
    double graph_dt = 0.0;
    int graph_prec = -1;
    int graph_cur = -1;
    bool graph_junc = false;
    bool graph_cons = false;
    bool consistent = false;          // consistent mobility in this burst (the context's setting)
    int64_t* d_loop_off = nullptr;    // [n_loops + 1] (consistent mobility)
    double* cm_scratch = nullptr;     // [5 n] (consistent mobility)
    DevBatchJunctions* junc = nullptr;  // junctions (ptadd_batch_set_junctions), NULL: off
    double dt_s = 0.0;                  // the step of the current burst, s (the junction clock)
    double time_scale = 0.0;            // mu / B: internal time -> s
};

namespace {

constexpr int BRED = 256;   // nodes per reduction block
constexpr int TILE_FP64 = 128;
// sources per staged tile of the mixed kernel: 192 at 128 threads (3 blocks
// of 66.5 KB fit one SM's shared memory), 128 at 64 threads
template <int TPB>
constexpr int tile_mix() { return TPB >= 128 ? 192 : 128; }

// ------------------------------------------------------------ kernels
__global__ void batch_prep_kernel(int64_t n, const double* __restrict__ pos, const int32_t* __restrict__ nxt,
                                  const int32_t* __restrict__ loop_of, const int32_t* __restrict__ real_of,
                                  const double* __restrict__ loop_b, const double* __restrict__ origin,
                                  double* __restrict__ src, float* __restrict__ src32)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t j = nxt[i];
    const double x1 = pos[i], y1 = pos[n + i], z1 = pos[2 * n + i];
    const double dx = pos[j] - x1, dy = pos[n + j] - y1, dz = pos[2 * n + j] - z1;
    const double L = sqrt(dx * dx + dy * dy + dz * dz);
    const int k = loop_of[i];
    const double bx = loop_b[3 * k], by = loop_b[3 * k + 1], bz = loop_b[3 * k + 2];
    double tx = 1.0, ty = 0.0, tz = 0.0;
    if (L > 0.0) {
        tx = dx / L;
        ty = dy / L;
        tz = dz / L;
    }
    const double qx = by * tz - bz * ty, qy = bz * tx - bx * tz, qz = bx * ty - by * tx;
    double* r = src + (int64_t)SRC_STRIDE * i;
    r[0] = x1; r[1] = y1; r[2] = z1; r[3] = L;
    r[4] = tx; r[5] = ty; r[6] = tz; r[7] = 0.0;
    r[8] = bx; r[9] = by; r[10] = bz; r[11] = 0.0;
    r[12] = qx; r[13] = qy; r[14] = qz; r[15] = 0.0;
    const int rr = real_of[i];
    const double rx = x1 - origin[3 * rr], ry = y1 - origin[3 * rr + 1], rz = z1 - origin[3 * rr + 2];
    const double hx = rint(rx), hy = rint(ry), hz = rint(rz);
    float* f = src32 + (int64_t)SRC32_STRIDE * i;
    f[0] = (float)hx; f[1] = (float)hy; f[2] = (float)hz;
    f[3] = (float)(rx - hx); f[4] = (float)(ry - hy); f[5] = (float)(rz - hz);
    f[6] = (float)L;
    f[7] = (float)tx; f[8] = (float)ty; f[9] = (float)tz;
    f[10] = (float)bx; f[11] = (float)by; f[12] = (float)bz;
    f[13] = (float)qx; f[14] = (float)qy; f[15] = (float)qz;
}

struct BatchPairArgs {
    const double* pos;
    int64_t n;
    const int32_t* nxt;
    const double* src;
    const float* src32;
    const int32_t* tgt;
    const int64_t* node_off;
    const int64_t* fp_base;
    const double* origin;
    const double* sh;
    double* fpart;
    const WorkItem* items;
    int n_items;
    unsigned* counter;
    unsigned long long* near_count;
    const double* k64;
};

__device__ __forceinline__ TileArgs tile_from_item(const BatchPairArgs& b, const WorkItem& w)
{
    TileArgs a;
    a.pos = b.pos;
    a.n = b.n;
    a.nxt = b.nxt;
    a.src = b.src;
    a.src32 = b.src32;
    a.tgt = b.tgt;
    a.t_begin = w.t_begin;
    a.t_count = w.t_count;
    a.js = w.js;
    a.je = w.je;
    a.add_app = w.chunk == 0;
    for (int k = 0; k < 6; ++k) a.sh[k] = b.sh[6 * w.r + k];
    for (int k = 0; k < 3; ++k) a.origin[k] = b.origin[3 * w.r + k];
    const int64_t nr = b.node_off[w.r + 1] - b.node_off[w.r];
    a.fp = b.fpart + b.fp_base[w.r] + (int64_t)w.chunk * 6 * nr;
    a.fp_stride = nr;
    a.node_base = b.node_off[w.r];
    a.near_count = b.near_count;
    a.k64 = b.k64;
    return a;
}

// Persistent pair kernel: each block pulls work items until the list is
// exhausted (the counter only grows, so the loop always ends).
template <int TPB, int MINB, bool MIXED>
__global__ void __launch_bounds__(TPB, MINB) batch_pair_kernel(BatchPairArgs b, Consts c, float near2)
{
    constexpr int TILE_MIX = tile_mix<TPB>();
    constexpr int SM_BYTES = MIXED ? (int)sizeof(MixSmem<TILE_MIX, TPB>) : TILE_FP64 * SRC_STRIDE * 8;
    __shared__ __align__(16) unsigned char smem[SM_BYTES];
    __shared__ int item;
    for (;;) {
        if (threadIdx.x == 0) item = (int)atomicAdd(b.counter, 1u);
        __syncthreads();
        const int it = item;
        __syncthreads();
        if (it >= b.n_items) break;
        const WorkItem w = b.items[it];
        const TileArgs a = tile_from_item(b, w);
        if (MIXED)
            pair_tile_mixed<TILE_MIX, TPB>(a, c, near2, *reinterpret_cast<MixSmem<TILE_MIX, TPB>*>(smem));
        else
            pair_tile_fp64<TILE_FP64>(a, c, reinterpret_cast<double2*>(smem));
    }
}

__global__ void batch_node_kernel(int64_t n, const double* __restrict__ pos, const int32_t* __restrict__ nxt,
                                  const int32_t* __restrict__ prv, const int32_t* __restrict__ loop_of,
                                  const int32_t* __restrict__ real_of, const double* __restrict__ loop_n,
                                  const uint8_t* __restrict__ pinned, const int64_t* __restrict__ node_off,
                                  const int64_t* __restrict__ fp_base, const int32_t* __restrict__ chunks,
                                  const double* __restrict__ fpart, double* __restrict__ force,
                                  double* __restrict__ vel)
{
    const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n) return;
    const int r = real_of[a];
    const int64_t base = node_off[r], nr = node_off[r + 1] - base;
    const int64_t la = a - base, lp = prv[a] - base;
    const double* fp0 = fpart + fp_base[r];
    double F[3] = {0, 0, 0};
    const int nch = chunks[r];
    for (int ch = 0; ch < nch; ++ch) {
        const double* fp = fp0 + (int64_t)ch * 6 * nr;
        F[0] += fp[0 * nr + la] + fp[3 * nr + lp];
        F[1] += fp[1 * nr + la] + fp[4 * nr + lp];
        F[2] += fp[2 * nr + la] + fp[5 * nr + lp];
    }
    const int64_t p = prv[a], nx = nxt[a];
    const double xa = pos[a], ya = pos[n + a], za = pos[2 * n + a];
    const double px = xa - pos[p], py = ya - pos[n + p], pz = za - pos[2 * n + p];
    const double qx = pos[nx] - xa, qy = pos[n + nx] - ya, qz = pos[2 * n + nx] - za;
    const double M = 0.5 * (sqrt(px * px + py * py + pz * pz) + sqrt(qx * qx + qy * qy + qz * qz));
    const int k = loop_of[a];
    const double nn[3] = {loop_n[3 * k], loop_n[3 * k + 1], loop_n[3 * k + 2]};
    double v[3] = {0, 0, 0};
    if (!pinned[a] && M > 0.0) {
        const double nF = nn[0] * F[0] + nn[1] * F[1] + nn[2] * F[2];
        v[0] = (F[0] - nn[0] * nF) / M;
        v[1] = (F[1] - nn[1] * nF) / M;
        v[2] = (F[2] - nn[2] * nF) / M;
    }
    force[a] = F[0]; force[n + a] = F[1]; force[2 * n + a] = F[2];
    vel[a] = v[0]; vel[n + a] = v[1]; vel[2 * n + a] = v[2];
}

// per-segment sums of the step-start state: L b (x) (t x vbar) (9), L (1), L vbar (3)
constexpr int BSUM = 13;

__global__ void __launch_bounds__(BRED) batch_lp_euler_kernel(
    int64_t n, const double* __restrict__ pos, double* __restrict__ pos_next, const int32_t* __restrict__ nxt,
    const int32_t* __restrict__ loop_of, const double* __restrict__ loop_b, const double* __restrict__ vel,
    const int32_t* __restrict__ blk_real, const int64_t* __restrict__ blk_start,
    const int64_t* __restrict__ node_off, double dt, double* __restrict__ partial, int* __restrict__ flag)
{
    __shared__ double red[BRED / 32][BSUM];
    const int r = blk_real[blockIdx.x];
    const int64_t i = blk_start[blockIdx.x] + threadIdx.x;
    const bool in = i < node_off[r + 1];
    double v13[BSUM];
#pragma unroll
    for (int m = 0; m < BSUM; ++m) v13[m] = 0.0;
    if (in) {
        const int64_t j = nxt[i];
        const double dx = pos[j] - pos[i], dy = pos[n + j] - pos[n + i], dz = pos[2 * n + j] - pos[2 * n + i];
        const double vx = 0.5 * (vel[i] + vel[j]);
        const double vy = 0.5 * (vel[n + i] + vel[n + j]);
        const double vz = 0.5 * (vel[2 * n + i] + vel[2 * n + j]);
        const double cx = dy * vz - dz * vy, cy = dz * vx - dx * vz, cz = dx * vy - dy * vx;
        const int k = loop_of[i];
        const double b0 = loop_b[3 * k], b1 = loop_b[3 * k + 1], b2 = loop_b[3 * k + 2];
        const double L = sqrt(dx * dx + dy * dy + dz * dz);
        v13[0] = b0 * cx; v13[1] = b0 * cy; v13[2] = b0 * cz;
        v13[3] = b1 * cx; v13[4] = b1 * cy; v13[5] = b1 * cz;
        v13[6] = b2 * cx; v13[7] = b2 * cy; v13[8] = b2 * cz;
        v13[9] = L;
        v13[10] = L * vx; v13[11] = L * vy; v13[12] = L * vz;
        const double nxp = __dadd_rn(pos[i], __dmul_rn(vel[i], dt));
        const double nyp = __dadd_rn(pos[n + i], __dmul_rn(vel[n + i], dt));
        const double nzp = __dadd_rn(pos[2 * n + i], __dmul_rn(vel[2 * n + i], dt));
        pos_next[i] = nxp;
        pos_next[n + i] = nyp;
        pos_next[2 * n + i] = nzp;
        if (!isfinite(nxp) || !isfinite(nyp) || !isfinite(nzp)) atomicOr(flag, 1);
    }
#pragma unroll
    for (int m = 0; m < BSUM; ++m) {
        double v = v13[m];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][m] = v;
    }
    __syncthreads();
    if (threadIdx.x < BSUM) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < BRED / 32; ++w) s += red[w][threadIdx.x];
        partial[(int64_t)blockIdx.x * BSUM + threadIdx.x] = s;
    }
}

// One block per realisation: its partials in order, weighted by dt, into
// acc[16 r + 0..9] (Lp, rho) and acc[16 r + 13..15] (polar velocity); the
// unweighted line length into acc[16 r + 11].
__global__ void batch_finish_kernel(const int32_t* __restrict__ real_blk, const double* __restrict__ partial,
                                    double dt, double* __restrict__ acc)
{
    __shared__ double red[128][BSUM];
    const int r = blockIdx.x;
    const int b0 = real_blk[r], b1 = real_blk[r + 1];
    double s[BSUM];
#pragma unroll
    for (int m = 0; m < BSUM; ++m) s[m] = 0.0;
    for (int b = b0 + threadIdx.x; b < b1; b += 128)
#pragma unroll
        for (int m = 0; m < BSUM; ++m) s[m] += partial[(int64_t)b * BSUM + m];
#pragma unroll
    for (int m = 0; m < BSUM; ++m) red[threadIdx.x][m] = s[m];
    __syncthreads();
    for (int h = 64; h > 0; h >>= 1) {
        if (threadIdx.x < h)
#pragma unroll
            for (int m = 0; m < BSUM; ++m) red[threadIdx.x][m] += red[threadIdx.x + h][m];
        __syncthreads();
    }
    if (threadIdx.x < BSUM) {
        const int slot = threadIdx.x < 10 ? threadIdx.x : threadIdx.x + 3;
        acc[16 * r + slot] = fma(red[0][threadIdx.x], dt, acc[16 * r + slot]);
    }
    if (threadIdx.x == 9) acc[16 * r + 11] = red[0][9];  // the step's line length (junction jumps weight it)
}

__global__ void batch_soa_to_aos(int64_t n, const double* __restrict__ soa, double scale, double* __restrict__ aos)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    aos[i] = soa[(i % 3) * n + i / 3] * scale;
}

// Forces SoA -> AoS in SI, zero at pinned nodes (their segments may be skipped).
__global__ void batch_forces_out(int64_t n, const double* __restrict__ force, const uint8_t* __restrict__ pinned,
                                 double scale, double* __restrict__ aos)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    const int64_t a = i / 3;
    aos[i] = pinned[a] ? 0.0 : force[(i % 3) * n + a] * scale;
}

__global__ void batch_aos_to_soa(int64_t n, const double* __restrict__ aos, double scale, double* __restrict__ soa)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    soa[(i % 3) * n + i / 3] = aos[i] * scale;
}

// ------------------------------------------------------------- helpers
template <typename T>
ptadd_status bd_alloc(T** p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
        *p = nullptr;
        return PTADD_ERR_NOMEM;
    }
    return PTADD_OK;
}

// Work list and fpart layout for a configuration; returns the fpart size needed.
int64_t build_items(const DevBatch& B, const BatchConfig& cfg, std::vector<WorkItem>& items,
                    std::vector<int64_t>& fp_base, std::vector<int32_t>& chunks)
{
    items.clear();
    fp_base.assign(B.R, 0);
    chunks.assign(B.R, 0);
    int64_t off = 0;
    for (int r = 0; r < B.R; ++r) {
        const int64_t s0 = B.node_off[r], nr = B.node_off[r + 1] - s0;
        const int32_t nch = (int32_t)((nr + cfg.chunk_len - 1) / cfg.chunk_len);
        chunks[r] = nch;
        fp_base[r] = off;
        off += (int64_t)nch * 6 * nr;
        const int64_t t0 = B.tgt_off[r], t1 = B.tgt_off[r + 1];
        for (int64_t tb = t0; tb < t1; tb += cfg.tpb)
            for (int32_t ch = 0; ch < nch; ++ch) {
                WorkItem w;
                w.r = r;
                w.chunk = ch;
                w.t_begin = (int32_t)tb;
                w.t_count = (int32_t)std::min<int64_t>(cfg.tpb, t1 - tb);
                w.js = (int32_t)(s0 + (int64_t)ch * cfg.chunk_len);
                w.je = (int32_t)std::min<int64_t>(s0 + nr, w.js + (int64_t)cfg.chunk_len);
                items.push_back(w);
            }
    }
    // largest first (cost ~ targets x sources), ties in a fixed order
    std::stable_sort(items.begin(), items.end(), [](const WorkItem& x, const WorkItem& y) {
        return (int64_t)x.t_count * (x.je - x.js) > (int64_t)y.t_count * (y.je - y.js);
    });
    return off;
}

ptadd_status apply_config(DevBatch& B, const BatchConfig& cfg, cudaStream_t s)
{
    std::vector<WorkItem> items;
    std::vector<int64_t> fp_base;
    std::vector<int32_t> chunks;
    const int64_t need = build_items(B, cfg, items, fp_base, chunks);
    if (need > B.fpart_cap) {
        set_error("internal: partial-force buffer too small for the configuration");
        return PTADD_ERR_STATE;
    }
    if (B.d_items) cudaFree(B.d_items);
    B.d_items = nullptr;
    ptadd_status st = bd_alloc(&B.d_items, items.size());
    if (st != PTADD_OK) return st;
    PTADD_CUDA(cudaMemcpyAsync(B.d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, s));
    PTADD_CUDA(cudaMemcpyAsync(B.d_fp_base, fp_base.data(), B.R * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    PTADD_CUDA(cudaMemcpyAsync(B.d_chunks, chunks.data(), B.R * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    // non-target entries must read as zero
    PTADD_CUDA(cudaMemsetAsync(B.fpart, 0, (size_t)need * sizeof(double), s));
    PTADD_CUDA(cudaStreamSynchronize(s));
    B.n_items = (int)items.size();
    B.cfg = cfg;
    if (B.graph) {
        cudaGraphExecDestroy(B.graph);
        B.graph = nullptr;
    }
    return PTADD_OK;
}

BatchPairArgs pair_args(const DevBatch& B)
{
    BatchPairArgs a;
    a.pos = B.pos[B.cur];
    a.n = B.n;
    a.nxt = B.nxt;
    a.src = B.src;
    a.src32 = B.src32;
    a.tgt = B.tgt;
    a.node_off = B.d_node_off;
    a.fp_base = B.d_fp_base;
    a.origin = B.d_origin;
    a.sh = B.d_sh;
    a.fpart = B.fpart;
    a.items = B.d_items;
    a.n_items = B.n_items;
    a.counter = B.counter;
    a.near_count = B.near_count;
    a.k64 = B.k64;
    return a;
}

template <int TPB, int MINB, bool MIXED>
cudaError_t launch_batch_pair_t(const DevBatch& B, const Consts& c, float near2, cudaStream_t s)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_pair_kernel<TPB, MINB, MIXED>, TPB, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int grid = std::min(sms * per_sm, std::max(1, B.n_items));
    batch_pair_kernel<TPB, MINB, MIXED><<<grid, TPB, 0, s>>>(pair_args(B), c, near2);
    return cudaGetLastError();
}

cudaError_t launch_batch_pair(const DevBatch& B, int prec, const Consts& c, cudaStream_t s)
{
    const float near2 = (float)((NEAR_FACTOR * NEAR_FACTOR + 1.0) * c.a2);
    const bool mixed = prec == (int)PTADD_MIXED;
    if (B.cfg.tpb == 64)
        return mixed ? launch_batch_pair_t<64, 6, true>(B, c, near2, s) : launch_batch_pair_t<64, 6, false>(B, c, near2, s);
    return mixed ? launch_batch_pair_t<128, 3, true>(B, c, near2, s) : launch_batch_pair_t<128, 3, false>(B, c, near2, s);
}

// One DD step of the whole batch on stream s (pos[cur] -> pos[1-cur]).
cudaError_t batch_step(DevBatch& B, int prec, const Consts& c, double dt_hat, cudaStream_t s)
{
    const unsigned nb = (unsigned)((B.n + 255) / 256);
    batch_prep_kernel<<<nb, 256, 0, s>>>(B.n, B.pos[B.cur], B.nxt, B.loop_of, B.real_of, B.loop_b, B.d_origin, B.src,
                                         B.src32);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(B.counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    if (B.n_items > 0) {
        e = launch_batch_pair(B, prec, c, s);
        if (e != cudaSuccess) return e;
    }
    batch_node_kernel<<<nb, 256, 0, s>>>(B.n, B.pos[B.cur], B.nxt, B.prv, B.loop_of, B.real_of, B.loop_n, B.pinned,
                                         B.d_node_off, B.d_fp_base, B.d_chunks, B.fpart, B.force, B.vel);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (B.consistent) {
        e = launch_consistent_velocity_raw(B.n_loops, B.d_loop_off, B.pos[B.cur], B.n, B.force, B.pinned, B.loop_n,
                                           B.vel, B.cm_scratch, s);
        if (e != cudaSuccess) return e;
    }
    if (B.junc) {
        e = launch_batch_junction_update(B.junc, B.pos[B.cur], B.src32, B.nxt, B.loop_of, B.real_of, B.d_node_off,
                                         B.pinned, B.vel, s);
        if (e != cudaSuccess) return e;
    }
    batch_lp_euler_kernel<<<B.nblk, BRED, 0, s>>>(B.n, B.pos[B.cur], B.pos[1 - B.cur], B.nxt, B.loop_of, B.loop_b,
                                                  B.vel, B.d_blk_real, B.d_blk_start, B.d_node_off, dt_hat, B.partial,
                                                  B.flag);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    batch_finish_kernel<<<B.R, 128, 0, s>>>(B.d_real_blk, B.partial, dt_hat, B.acc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (B.junc) {
        e = launch_batch_junction_event(B.junc, B.acc, B.dt_s, dt_hat, B.time_scale, s);
        if (e != cudaSuccess) return e;
    }
    B.cur = 1 - B.cur;
    return cudaSuccess;
}

void free_batch(DevBatch& B)
{
    if (B.graph) cudaGraphExecDestroy(B.graph);
    batch_junctions_free(B.junc);
    if (B.d_loop_off) cudaFree(B.d_loop_off);
    if (B.cm_scratch) cudaFree(B.cm_scratch);
    void* ptrs[] = {B.pos[0],   B.pos[1],    B.nxt,       B.prv,        B.loop_of,  B.real_of, B.tgt,
                    B.loop_b,   B.loop_n,    B.pinned,    B.src,        B.src32,    B.fpart,   B.vel,
                    B.force,    B.partial,   B.acc,       B.d_node_off, B.d_fp_base, B.d_chunks, B.d_origin,
                    B.d_sh,     B.d_blk_real, B.d_blk_start, B.d_real_blk, B.d_items, B.counter, B.flag,
                    B.near_count, B.staging, B.k64};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    B = DevBatch{};
}

Consts batch_consts(const ptadd_ctx* ctx)
{
    Consts c;
    const double r = ctx->mat.a / ctx->len_unit;
    c.a2 = r * r;
    c.c1 = 1.0 / (8.0 * M_PI);
    c.c2 = 1.0 / (4.0 * M_PI * (1.0 - ctx->mat.nu));
    return c;
}

// ----------------------------------------------------------- tune cache
#ifndef PTADD_BUILD_HASH
#define PTADD_BUILD_HASH 0ull  // a build that passes no source hash (build.py passes one)
#endif
std::string tune_key(const ptadd_ctx* ctx, const DevBatch& B, int prec)
{
    cudaDeviceProp p;
    cudaGetDeviceProperties(&p, ctx->device);
    const double mean_n = (double)B.n / std::max(1, B.R);
    char buf[512];
    snprintf(buf, sizeof(buf), "%.200s|sm%d|v%d|h%016llx|%s|n2^%d|R2^%d", p.name, p.multiProcessorCount,
             ptadd_version(), (unsigned long long)PTADD_BUILD_HASH, prec == (int)PTADD_MIXED ? "mixed" : "fp64",
             (int)lround(log2(std::max(1.0, mean_n))), (int)lround(log2((double)std::max(1, B.R))));
    for (char* q = buf; *q; ++q)
        if (*q == '"' || *q == '\n') *q = '_';
    return buf;
}

std::string tune_path(const char* path)
{
    if (path && *path) return path;
    const char* env = getenv("PTADD_TUNE_CACHE");
    if (env && *env) return env;
    const char* home = getenv("HOME");
    return std::string(home ? home : "/tmp") + "/.cache/ptadd_tune.jsonl";
}

bool tune_lookup(const std::string& file, const std::string& key, BatchConfig& cfg)
{
    FILE* f = fopen(file.c_str(), "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        char k[512];
        int tpb = 0, chunk = 0;
        // {"key": "...", "tpb": N, "chunk": N, ...}
        if (sscanf(line, " {\"key\": \"%511[^\"]\", \"tpb\": %d, \"chunk\": %d", k, &tpb, &chunk) == 3 &&
            key == k && (tpb == 64 || tpb == 128) && chunk >= 256 && chunk % 256 == 0) {
            cfg.tpb = tpb;
            cfg.chunk_len = chunk;
            found = true;  // the last entry for a key wins
        }
    }
    fclose(f);
    return found;
}

void tune_store(const std::string& file, const std::string& key, const BatchConfig& cfg, double ms)
{
    const size_t slash = file.rfind('/');
    if (slash != std::string::npos && slash > 0) {
        const std::string dir = file.substr(0, slash);
        for (size_t i = 1; i <= dir.size(); ++i)  // mkdir -p, ignoring "exists"
            if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
    }
    FILE* f = fopen(file.c_str(), "a");
    if (!f) return;
    fprintf(f, "{\"key\": \"%s\", \"tpb\": %d, \"chunk\": %d, \"pair_ms\": %.6f}\n", key.c_str(), cfg.tpb,
            cfg.chunk_len, ms);
    fclose(f);
}

}  // namespace

bool batch_has_junctions(const ptadd_ctx* ctx) { return ctx && ctx->batch && ctx->batch->junc; }

void batch_free(ptadd_ctx* ctx)
{
    if (ctx && ctx->batch) {
        free_batch(*ctx->batch);
        delete ctx->batch;
        ctx->batch = nullptr;
    }
}

}  // namespace ptadd

using namespace ptadd;

static ptadd_status barg(const char* m)
{
    set_error("%s", m);
    return PTADD_ERR_ARG;
}

extern "C" {

ptadd_status ptadd_batch_set(ptadd_ctx* ctx, int32_t R, const int64_t* node_off, int64_t n_loops,
                             const int64_t* loop_off, const double* xyz, const double* burgers, const double* normal,
                             const uint8_t* pinned, const double* sig6, const double* volume)
{
    if (!ctx) return barg("null context");
    PTADD_CUDA(cudaSetDevice(ctx->device));
    if (R < 1) return barg("R must be >= 1");
    if (!node_off || !loop_off || !xyz || !burgers || !normal || !sig6 || !volume) return barg("null array");
    if (node_off[0] != 0) return barg("node_off[0] must be 0");
    for (int r = 0; r < R; ++r)
        if (node_off[r + 1] - node_off[r] < 2) return barg("every realisation needs >= 2 nodes");
    const int64_t n = node_off[R];
    if (n > ((int64_t)1 << 31) - 1) return barg("too many nodes in the batch (max 2^31 - 1)");
    if (n_loops < R || loop_off[0] != 0 || loop_off[n_loops] != n) return barg("loop_off must run from 0 to n_nodes");
    // loops: >= 2 nodes, inside one realisation
    {
        int r = 0;
        for (int64_t k = 0; k < n_loops; ++k) {
            const int64_t a = loop_off[k], b = loop_off[k + 1];
            if (b - a < 2) return barg("every loop needs >= 2 nodes");
            while (r < R && a >= node_off[r + 1]) ++r;
            if (r >= R || b > node_off[r + 1]) return barg("a loop straddles two realisations");
        }
    }
    const double bmag = ctx->mat.b;
    const int ie = -ctx->len_exp;
    std::vector<double> origin(3 * R), sh(6 * R), vol(R);
    for (int r = 0; r < R; ++r) {
        if (!(volume[r] > 0) || !isfinite(volume[r])) return barg("volumes must be positive and finite");
        vol[r] = volume[r];
        for (int c = 0; c < 6; ++c) {
            if (!isfinite(sig6[6 * r + c])) return barg("non-finite applied stress");
            sh[6 * r + c] = sig6[6 * r + c] / ctx->mat.mu;
        }
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t i = node_off[r]; i < node_off[r + 1]; ++i)
            for (int c = 0; c < 3; ++c) {
                const double v = xyz[3 * i + c];
                if (!isfinite(v)) return barg("non-finite node position");
                lo[c] = fmin(lo[c], v);
                hi[c] = fmax(hi[c], v);
            }
        for (int c = 0; c < 3; ++c) {
            if ((hi[c] - lo[c]) / bmag > 1.0e6) return barg("a realisation's extent exceeds 1e6 Burgers vectors");
            origin[3 * r + c] = rint(ldexp(0.5 * (lo[c] + hi[c]), ie));
        }
    }
    for (int64_t k = 0; k < n_loops; ++k) {
        const double* nn = normal + 3 * k;
        if (!(fabs(sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]) - 1.0) <= 1e-9))
            return barg("glide normals must be unit vectors");
        for (int c = 0; c < 3; ++c)
            if (!isfinite(burgers[3 * k + c])) return barg("non-finite Burgers vector");
    }

    if (ctx->batch) {
        free_batch(*ctx->batch);
    } else {
        ctx->batch = new (std::nothrow) DevBatch();
        if (!ctx->batch) return barg("host allocation failed");
    }
    DevBatch& B = *ctx->batch;
    B.R = R;
    B.n = n;
    B.n_loops = n_loops;
    B.node_off.assign(node_off, node_off + R + 1);
    B.volume = vol;
    B.origin = origin;
    B.sh = sh;

    std::vector<double> pos(3 * n), lb(3 * n_loops), ln(3 * n_loops);
    std::vector<int32_t> nxt(n), prv(n), lof(n), rof(n), tgt;
    std::vector<uint8_t> pin(n, 0);
    for (int64_t i = 0; i < n; ++i) {
        pos[i] = ldexp(xyz[3 * i], ie);
        pos[n + i] = ldexp(xyz[3 * i + 1], ie);
        pos[2 * n + i] = ldexp(xyz[3 * i + 2], ie);
        if (pinned) pin[i] = pinned[i] ? 1 : 0;
    }
    for (int64_t k = 0; k < n_loops; ++k) {
        const int64_t a = loop_off[k], b = loop_off[k + 1];
        for (int64_t i = a; i < b; ++i) {
            nxt[i] = (int32_t)((i + 1 < b) ? i + 1 : a);
            prv[i] = (int32_t)((i > a) ? i - 1 : b - 1);
            lof[i] = (int32_t)k;
        }
        for (int c = 0; c < 3; ++c) {
            lb[3 * k + c] = burgers[3 * k + c] / ctx->len_unit;
            ln[3 * k + c] = normal[3 * k + c];
        }
    }
    B.tgt_off.assign(R + 1, 0);
    std::vector<int32_t> blk_real;
    std::vector<int64_t> blk_start;
    std::vector<int32_t> real_blk(R + 1, 0);
    B.pairs = 0;
    for (int r = 0; r < R; ++r) {
        const int64_t a = node_off[r], b = node_off[r + 1];
        B.tgt_off[r] = (int64_t)tgt.size();
        for (int64_t i = a; i < b; ++i) {
            rof[i] = r;
            if (!(pin[i] && pin[nxt[i]])) tgt.push_back((int32_t)i);
        }
        B.pairs += ((int64_t)tgt.size() - B.tgt_off[r]) * (b - a);
        real_blk[r] = (int32_t)blk_real.size();
        for (int64_t s0 = a; s0 < b; s0 += BRED) {
            blk_real.push_back(r);
            blk_start.push_back(s0);
        }
    }
    B.tgt_off[R] = (int64_t)tgt.size();
    real_blk[R] = (int32_t)blk_real.size();
    B.n_tgt = (int64_t)tgt.size();
    B.nblk = (int)blk_real.size();

    // partial-force capacity: the smallest chunk length any configuration uses
    {
        std::vector<WorkItem> items;
        std::vector<int64_t> fb;
        std::vector<int32_t> ch;
        BatchConfig smallest;
        smallest.chunk_len = 1024;
        B.fpart_cap = build_items(B, smallest, items, fb, ch);
    }

    ptadd_status st = PTADD_OK;
#define BALLOC(p, cnt) \
    if (st == PTADD_OK) st = bd_alloc(&(p), (size_t)(cnt));
    BALLOC(B.pos[0], 3 * n);
    BALLOC(B.pos[1], 3 * n);
    BALLOC(B.nxt, n);
    BALLOC(B.prv, n);
    BALLOC(B.loop_of, n);
    BALLOC(B.real_of, n);
    BALLOC(B.tgt, tgt.size());
    BALLOC(B.loop_b, 3 * n_loops);
    BALLOC(B.loop_n, 3 * n_loops);
    BALLOC(B.pinned, n);
    BALLOC(B.src, SRC_STRIDE * n);
    BALLOC(B.src32, SRC32_STRIDE * n);
    BALLOC(B.fpart, B.fpart_cap);
    BALLOC(B.vel, 3 * n);
    BALLOC(B.force, 3 * n);
    BALLOC(B.partial, (int64_t)BSUM * B.nblk);
    BALLOC(B.acc, 16 * (int64_t)R);
    BALLOC(B.d_node_off, R + 1);
    BALLOC(B.d_fp_base, R);
    BALLOC(B.d_chunks, R);
    BALLOC(B.d_origin, 3 * R);
    BALLOC(B.d_sh, 6 * R);
    BALLOC(B.d_blk_real, B.nblk);
    BALLOC(B.d_blk_start, B.nblk);
    BALLOC(B.d_real_blk, R + 1);
    BALLOC(B.counter, 1);
    BALLOC(B.flag, 1);
    BALLOC(B.near_count, 1);
    BALLOC(B.staging, 3 * n);
    BALLOC(B.k64, 4);
    BALLOC(B.d_loop_off, n_loops + 1);
    BALLOC(B.cm_scratch, 5 * n);
#undef BALLOC
    if (st != PTADD_OK) {
        free_batch(B);
        delete ctx->batch;
        ctx->batch = nullptr;
        return st;
    }
    cudaStream_t s = ctx->own_stream;
    PTADD_CUDA(cudaStreamSynchronize(ctx->stream));
#define H2D(dst, srcv, cnt) PTADD_CUDA(cudaMemcpyAsync(dst, srcv, (size_t)(cnt) * sizeof(*(dst)), cudaMemcpyHostToDevice, s))
    H2D(B.pos[0], pos.data(), 3 * n);
    H2D(B.nxt, nxt.data(), n);
    H2D(B.prv, prv.data(), n);
    H2D(B.loop_of, lof.data(), n);
    H2D(B.real_of, rof.data(), n);
    if (!tgt.empty()) H2D(B.tgt, tgt.data(), tgt.size());
    H2D(B.loop_b, lb.data(), 3 * n_loops);
    H2D(B.loop_n, ln.data(), 3 * n_loops);
    H2D(B.pinned, pin.data(), n);
    H2D(B.d_node_off, node_off, R + 1);
    H2D(B.d_loop_off, loop_off, n_loops + 1);
    H2D(B.d_origin, origin.data(), 3 * R);
    H2D(B.d_sh, sh.data(), 6 * R);
    H2D(B.d_blk_real, blk_real.data(), B.nblk);
    H2D(B.d_blk_start, blk_start.data(), B.nblk);
    H2D(B.d_real_blk, real_blk.data(), R + 1);
#undef H2D
    PTADD_CUDA(cudaMemsetAsync(B.acc, 0, 16 * (size_t)R * sizeof(double), s));
    PTADD_CUDA(cudaMemsetAsync(B.flag, 0, sizeof(int), s));
    PTADD_CUDA(cudaMemsetAsync(B.near_count, 0, sizeof(unsigned long long), s));
    {
        const Consts kc = batch_consts(ctx);
        const double k64[4] = {kc.a2, kc.c1, kc.c2, 0.0};
        PTADD_CUDA(cudaMemcpyAsync(B.k64, k64, sizeof(k64), cudaMemcpyHostToDevice, s));
    }
    PTADD_CUDA(cudaStreamSynchronize(s));
    BatchConfig cfg;
    B.tuned = tune_lookup(tune_path(nullptr), tune_key(ctx, B, (int)ctx->prec), cfg) ? 1 : 0;
    return apply_config(B, cfg, s);
}

ptadd_status ptadd_batch_set_stress(ptadd_ctx* ctx, const double* sig6)
{
    if (!ctx || !ctx->batch) {
        set_error("no batch loaded");
        return PTADD_ERR_STATE;
    }
    if (!sig6) return barg("sig6 is NULL");
    DevBatch& B = *ctx->batch;
    for (int64_t k = 0; k < 6 * (int64_t)B.R; ++k) {
        if (!isfinite(sig6[k])) return barg("non-finite applied stress");
        B.sh[k] = sig6[k] / ctx->mat.mu;
    }
    PTADD_CUDA(cudaSetDevice(ctx->device));
    PTADD_CUDA(cudaMemcpyAsync(B.d_sh, B.sh.data(), 6 * B.R * sizeof(double), cudaMemcpyHostToDevice, ctx->own_stream));
    PTADD_CUDA(cudaStreamSynchronize(ctx->own_stream));
    return PTADD_OK;
}

ptadd_status ptadd_batch_advance(ptadd_ctx* ctx, int64_t n_steps, double dt, double* Lp_avg, double* rho_avg)
{
    if (!ctx || !ctx->batch) {
        set_error("no batch loaded");
        return PTADD_ERR_STATE;
    }
    if (n_steps < 0) return barg("n_steps < 0");
    if (!(dt > 0) || !isfinite(dt)) return barg("dt must be positive and finite");
    PTADD_CUDA(cudaSetDevice(ctx->device));
    DevBatch& B = *ctx->batch;
    cudaStream_t s = ctx->own_stream;
    PTADD_CUDA(cudaStreamSynchronize(ctx->stream));  // order after the caller's work
    const Consts c = batch_consts(ctx);
    const double dt_hat = dt * ctx->mat.mu / ctx->mat.B;
    const int prec = (int)ctx->prec;
    PTADD_CUDA(cudaMemsetAsync(B.acc, 0, 16 * (size_t)B.R * sizeof(double), s));
    PTADD_CUDA(cudaMemsetAsync(B.flag, 0, sizeof(int), s));
    B.dt_s = dt;
    B.time_scale = ctx->mat.mu / ctx->mat.B;
    const bool junc = B.junc != nullptr;
    B.consistent = ctx->consistent_mass;
    const int per_step = (junc ? 9 : 5) + (B.consistent ? 1 : 0);
    int64_t left = n_steps;
    if (left >= 2) {
        if (!B.graph || B.graph_dt != dt_hat || B.graph_prec != prec || B.graph_cur != B.cur || B.graph_junc != junc ||
            B.graph_cons != B.consistent) {
            if (B.graph) cudaGraphExecDestroy(B.graph);
            B.graph = nullptr;
            const int cur0 = B.cur;
            cudaGraph_t g = nullptr;
            PTADD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = batch_step(B, prec, c, dt_hat, s);
            if (e == cudaSuccess) e = batch_step(B, prec, c, dt_hat, s);
            cudaError_t e2 = cudaStreamEndCapture(s, &g);
            B.cur = cur0;
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                set_error("capturing the batch step graph failed: %s",
                          cudaGetErrorString(e != cudaSuccess ? e : e2));
                return PTADD_ERR_CUDA;
            }
            e = cudaGraphInstantiate(&B.graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                B.graph = nullptr;
                set_error("instantiating the batch step graph failed: %s", cudaGetErrorString(e));
                return PTADD_ERR_CUDA;
            }
            B.graph_dt = dt_hat;
            B.graph_prec = prec;
            B.graph_cur = B.cur;
            B.graph_junc = junc;
            B.graph_cons = B.consistent;
        }
        while (left >= 2) {
            PTADD_CUDA(cudaGraphLaunch(B.graph, s));
            left -= 2;
            ctx->kernel_launches += 2 * per_step;
        }
    }
    if (left == 1) {
        PTADD_CUDA(batch_step(B, prec, c, dt_hat, s));
        ctx->kernel_launches += per_step;
    }
    std::vector<double> acc(16 * (size_t)B.R);
    int flag = 0;
    PTADD_CUDA(cudaMemcpyAsync(acc.data(), B.acc, acc.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    PTADD_CUDA(cudaMemcpyAsync(&flag, B.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    PTADD_CUDA(cudaStreamSynchronize(s));
    const double l = ctx->len_unit;
    bool finite = flag == 0;
    B.last_LV.assign(3 * (size_t)B.R, 0.0);
    for (int r = 0; r < B.R; ++r) {
        // Eq. 2.5; the time a realisation jumped over while stuck counts with Lp = 0 and the step's rho
        const double St = dt_hat * (double)n_steps + (junc ? acc[16 * r + 12] : 0.0);
        const double lp_scale = l * l * l * ctx->mat.mu / (ctx->mat.B * B.volume[r]);
        const double rho_scale = l / B.volume[r];
        const double v_scale = l * l * ctx->mat.mu / (ctx->mat.B * B.volume[r]);
        for (int m = 0; m < 10; ++m) finite = finite && isfinite(acc[16 * r + m]);
        for (int m = 0; m < 3; ++m) {
            finite = finite && isfinite(acc[16 * r + 13 + m]);
            B.last_LV[3 * r + m] = n_steps > 0 ? acc[16 * r + 13 + m] / St * v_scale : 0.0;
        }
        if (Lp_avg)
            for (int m = 0; m < 9; ++m) Lp_avg[9 * r + m] = n_steps > 0 ? acc[16 * r + m] / St * lp_scale : 0.0;
        if (rho_avg) rho_avg[r] = n_steps > 0 ? acc[16 * r + 9] / St * rho_scale : 0.0;
    }
    if (!finite) {
        set_error("batch burst produced a non-finite position or average");
        return PTADD_ERR_NONFINITE;
    }
    return PTADD_OK;
}

ptadd_status ptadd_batch_set_junctions(ptadd_ctx* ctx, const ptadd_junction_params* p)
{
    if (!ctx || !ctx->batch) {
        set_error("ptadd_batch_set_junctions: no batch loaded");
        return PTADD_ERR_STATE;
    }
    if (p && !(p->capture_radius >= 0.0 && isfinite(p->capture_radius) && p->max_break_time >= 0.0 &&
               isfinite(p->max_break_time) && p->stuck_disp >= 0.0 && isfinite(p->stuck_disp)))
        return barg("ptadd_batch_set_junctions: parameters must be non-negative and finite");
    if (p && ctx->consistent_mass) {
        set_error("ptadd_batch_set_junctions: junctions need the lumped mobility (ptadd_set_mobility(ctx, 0))");
        return PTADD_ERR_STATE;
    }
    PTADD_CUDA(cudaSetDevice(ctx->device));
    DevBatch& B = *ctx->batch;
    PTADD_CUDA(cudaStreamSynchronize(ctx->own_stream));
    batch_junctions_free(B.junc);
    if (B.graph) {  // it holds the old junction state's pointers
        cudaGraphExecDestroy(B.graph);
        B.graph = nullptr;
    }
    if (!p) return PTADD_OK;
    const int64_t n = B.n;
    std::vector<uint8_t> pin(n);
    std::vector<int32_t> nxt(n), lof(n);
    PTADD_CUDA(cudaMemcpy(pin.data(), B.pinned, n, cudaMemcpyDeviceToHost));
    PTADD_CUDA(cudaMemcpy(nxt.data(), B.nxt, n * sizeof(int32_t), cudaMemcpyDeviceToHost));
    PTADD_CUDA(cudaMemcpy(lof.data(), B.loop_of, n * sizeof(int32_t), cudaMemcpyDeviceToHost));
    return batch_junctions_create(&B.junc, p, ctx->len_unit, B.R, B.node_off, pin, nxt, lof);
}

ptadd_status ptadd_batch_get_junctions(ptadd_ctx* ctx, ptadd_junction_info* info, int32_t* seg, int32_t* last,
                                       int32_t* count, double* break_time)
{
    if (!ctx || !ctx->batch || !ctx->batch->junc) {
        set_error("ptadd_batch_get_junctions: junctions of the batch are off");
        return PTADD_ERR_STATE;
    }
    PTADD_CUDA(cudaSetDevice(ctx->device));
    DevBatch& B = *ctx->batch;
    return batch_junctions_get(B.junc, B.node_off, ctx->own_stream, info, seg, last, count, break_time);
}

ptadd_status ptadd_batch_get_polar_velocity(ptadd_ctx* ctx, double core_area, double* V_avg)
{
    if (!ctx || !ctx->batch) {
        set_error("no batch loaded");
        return PTADD_ERR_STATE;
    }
    if (!V_avg) return barg("V_avg is NULL");
    if (!(core_area > 0) || !isfinite(core_area)) return barg("core_area must be positive and finite");
    const DevBatch& B = *ctx->batch;
    if (B.last_LV.size() != 3 * (size_t)B.R) {
        set_error("no batch burst has run since the batch was set");
        return PTADD_ERR_STATE;
    }
    for (size_t k = 0; k < B.last_LV.size(); ++k) V_avg[k] = core_area * B.last_LV[k];
    return PTADD_OK;
}

ptadd_status ptadd_batch_get_nodes(ptadd_ctx* ctx, double* xyz)
{
    if (!ctx || !ctx->batch) {
        set_error("no batch loaded");
        return PTADD_ERR_STATE;
    }
    if (!xyz) return barg("xyz is NULL");
    PTADD_CUDA(cudaSetDevice(ctx->device));
    DevBatch& B = *ctx->batch;
    cudaStream_t s = ctx->own_stream;
    batch_soa_to_aos<<<(unsigned)((3 * B.n + 255) / 256), 256, 0, s>>>(B.n, B.pos[B.cur], ctx->len_unit, B.staging);
    PTADD_CUDA(cudaGetLastError());
    PTADD_CUDA(cudaMemcpyAsync(xyz, B.staging, 3 * B.n * sizeof(double), cudaMemcpyDeviceToHost, s));
    PTADD_CUDA(cudaStreamSynchronize(s));
    return PTADD_OK;
}

ptadd_status ptadd_batch_set_nodes(ptadd_ctx* ctx, const double* xyz)
{
    if (!ctx || !ctx->batch) {
        set_error("no batch loaded");
        return PTADD_ERR_STATE;
    }
    if (!xyz) return barg("xyz is NULL");
    PTADD_CUDA(cudaSetDevice(ctx->device));
    DevBatch& B = *ctx->batch;
    for (int r = 0; r < B.R; ++r) {
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t i = B.node_off[r]; i < B.node_off[r + 1]; ++i)
            for (int c = 0; c < 3; ++c) {
                const double v = xyz[3 * i + c];
                if (!isfinite(v)) return barg("non-finite node position");
                lo[c] = fmin(lo[c], v);
                hi[c] = fmax(hi[c], v);
            }
        for (int c = 0; c < 3; ++c) {
            if ((hi[c] - lo[c]) / ctx->mat.b > 1.0e6) return barg("a realisation's extent exceeds 1e6 Burgers vectors");
            B.origin[3 * r + c] = rint(ldexp(0.5 * (lo[c] + hi[c]), -ctx->len_exp));
        }
    }
    cudaStream_t s = ctx->own_stream;
    PTADD_CUDA(cudaMemcpyAsync(B.d_origin, B.origin.data(), 3 * B.R * sizeof(double), cudaMemcpyHostToDevice, s));
    PTADD_CUDA(cudaMemcpyAsync(B.staging, xyz, 3 * B.n * sizeof(double), cudaMemcpyHostToDevice, s));
    batch_aos_to_soa<<<(unsigned)((3 * B.n + 255) / 256), 256, 0, s>>>(B.n, B.staging, 1.0 / ctx->len_unit,
                                                                         B.pos[B.cur]);
    PTADD_CUDA(cudaGetLastError());
    PTADD_CUDA(cudaStreamSynchronize(s));
    return PTADD_OK;
}

ptadd_status ptadd_batch_configure(ptadd_ctx* ctx, int32_t tile_targets, int32_t chunk_sources)
{
    if (!ctx || !ctx->batch) {
        set_error("no batch loaded");
        return PTADD_ERR_STATE;
    }
    if (tile_targets != 64 && tile_targets != 128) return barg("tile_targets must be 64 or 128");
    if (chunk_sources < 1024 || chunk_sources > (1 << 24) || chunk_sources % 128 != 0)
        return barg("chunk_sources must be a multiple of 128 in [1024, 2^24]");
    PTADD_CUDA(cudaSetDevice(ctx->device));
    PTADD_CUDA(cudaStreamSynchronize(ctx->stream));
    BatchConfig cfg;
    cfg.tpb = tile_targets;
    cfg.chunk_len = chunk_sources;
    ptadd_status st = apply_config(*ctx->batch, cfg, ctx->own_stream);
    if (st == PTADD_OK) ctx->batch->tuned = 0;
    return st;
}

ptadd_status ptadd_batch_get_forces(ptadd_ctx* ctx, double* F)
{
    if (!ctx || !ctx->batch) {
        set_error("no batch loaded");
        return PTADD_ERR_STATE;
    }
    if (!F) return barg("F is NULL");
    PTADD_CUDA(cudaSetDevice(ctx->device));
    DevBatch& B = *ctx->batch;
    cudaStream_t s = ctx->own_stream;
    PTADD_CUDA(cudaStreamSynchronize(ctx->stream));
    const Consts c = batch_consts(ctx);
    const unsigned nb = (unsigned)((B.n + 255) / 256);
    batch_prep_kernel<<<nb, 256, 0, s>>>(B.n, B.pos[B.cur], B.nxt, B.loop_of, B.real_of, B.loop_b, B.d_origin, B.src,
                                         B.src32);
    PTADD_CUDA(cudaGetLastError());
    PTADD_CUDA(cudaMemsetAsync(B.counter, 0, sizeof(unsigned), s));
    if (B.n_items > 0) PTADD_CUDA(launch_batch_pair(B, (int)ctx->prec, c, s));
    batch_node_kernel<<<nb, 256, 0, s>>>(B.n, B.pos[B.cur], B.nxt, B.prv, B.loop_of, B.real_of, B.loop_n, B.pinned,
                                         B.d_node_off, B.d_fp_base, B.d_chunks, B.fpart, B.force, B.vel);
    PTADD_CUDA(cudaGetLastError());
    batch_forces_out<<<(unsigned)((3 * B.n + 255) / 256), 256, 0, s>>>(
        B.n, B.force, B.pinned, ctx->mat.mu * ctx->len_unit * ctx->len_unit, B.staging);
    PTADD_CUDA(cudaGetLastError());
    ctx->kernel_launches += 4;
    PTADD_CUDA(cudaMemcpyAsync(F, B.staging, 3 * B.n * sizeof(double), cudaMemcpyDeviceToHost, s));
    PTADD_CUDA(cudaStreamSynchronize(s));
    return PTADD_OK;
}

ptadd_status ptadd_batch_get_info(ptadd_ctx* ctx, ptadd_batch_info* info)
{
    if (!ctx || !ctx->batch) {
        set_error("no batch loaded");
        return PTADD_ERR_STATE;
    }
    if (!info) return barg("info is NULL");
    const DevBatch& B = *ctx->batch;
    info->R = B.R;
    info->n_nodes = B.n;
    info->n_loops = B.n_loops;
    info->n_targets = B.n_tgt;
    info->pairs_per_step = B.pairs;
    info->work_items = B.n_items;
    info->tile_targets = B.cfg.tpb;
    info->chunk_sources = B.cfg.chunk_len;
    info->tuned = B.tuned;
    return PTADD_OK;
}

ptadd_status ptadd_batch_autotune(ptadd_ctx* ctx, const char* cache_path, int force)
{
    if (!ctx || !ctx->batch) {
        set_error("no batch loaded");
        return PTADD_ERR_STATE;
    }
    PTADD_CUDA(cudaSetDevice(ctx->device));
    DevBatch& B = *ctx->batch;
    const int prec = (int)ctx->prec;
    const std::string path = tune_path(cache_path);
    const std::string key = tune_key(ctx, B, prec);
    BatchConfig cached;
    if (!force && tune_lookup(path, key, cached)) {
        B.tuned = 1;
        return apply_config(B, cached, ctx->own_stream);
    }
    cudaStream_t s = ctx->own_stream;
    PTADD_CUDA(cudaStreamSynchronize(ctx->stream));
    const Consts c = batch_consts(ctx);
    cudaEvent_t e0, e1;
    PTADD_CUDA(cudaEventCreate(&e0));
    PTADD_CUDA(cudaEventCreate(&e1));
    const int tpbs[2] = {64, 128};
    const int chunks[3] = {1024, 2048, 4096};
    BatchConfig best;
    double best_ms = INFINITY;
    ptadd_status st = PTADD_OK;
    const unsigned nb = (unsigned)((B.n + 255) / 256);
    for (int ti = 0; ti < 2 && st == PTADD_OK; ++ti)
        for (int ci = 0; ci < 3 && st == PTADD_OK; ++ci) {
            BatchConfig cfg;
            cfg.tpb = tpbs[ti];
            cfg.chunk_len = chunks[ci];
            st = apply_config(B, cfg, s);
            if (st != PTADD_OK) break;
            float best_rep = INFINITY;
            for (int rep = 0; rep < 3; ++rep) {  // first repetition is a warm-up
                batch_prep_kernel<<<nb, 256, 0, s>>>(B.n, B.pos[B.cur], B.nxt, B.loop_of, B.real_of, B.loop_b,
                                                     B.d_origin, B.src, B.src32);
                cudaError_t e = cudaMemsetAsync(B.counter, 0, sizeof(unsigned), s);
                if (e == cudaSuccess) e = cudaEventRecord(e0, s);
                if (e == cudaSuccess && B.n_items > 0) e = launch_batch_pair(B, prec, c, s);
                if (e == cudaSuccess) e = cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) {
                    set_error("autotune run failed: %s", cudaGetErrorString(e));
                    st = PTADD_ERR_CUDA;
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0 && ms < best_rep) best_rep = ms;
            }
            if (st == PTADD_OK && best_rep < best_ms) {
                best_ms = best_rep;
                best = cfg;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PTADD_OK) return st;
    tune_store(path, key, best, best_ms);
    B.tuned = 1;
    return apply_config(B, best, s);
}

ptadd_status ptadd_batch_run(ptadd_ctx* ctx, int32_t R, const int64_t* node_off, int64_t n_loops,
                             const int64_t* loop_off, const double* xyz, const double* burgers, const double* normal,
                             const uint8_t* pinned, const double* sig6, const double* volume, int64_t n_steps,
                             double dt, double* Lp_avg, double* rho_avg)
{
    ptadd_status st = ptadd_batch_set(ctx, R, node_off, n_loops, loop_off, xyz, burgers, normal, pinned, sig6, volume);
    if (st != PTADD_OK) return st;
    return ptadd_batch_advance(ctx, n_steps, dt, Lp_avg, rho_avg);
}

}  // extern "C"
