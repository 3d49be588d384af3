// ptadd_internal.cuh -- shared declarations of the CUDA implementation of ptadd.h.
//
// Internal units (all kernels): lengths in l = 2^e metres with e the integer
// nearest log2(b) (so converting positions is an exact scaling: the kernels
// see the caller's geometry without rounding -- the nodal forces of a loop
// network change by ~3e-11 relative under a 1-ulp change of the positions),
// stresses in mu, time in B/mu.  Then a nodal velocity is the projected nodal
// force divided by the lumped length, v = P F / M, and the Euler step uses
// dt_hat = dt mu / B.  Conversion to SI happens only in the host entry points.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ptadd.h"

struct ptadd_ctx;

namespace ptadd {

// --------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
const char* cuda_msg(cudaError_t e);

#define PTADD_CUDA(call)                                                          \
    do {                                                                          \
        cudaError_t _e = (call);                                                  \
        if (_e != cudaSuccess) {                                                  \
            ::ptadd::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(_e), \
                               __FILE__, __LINE__);                               \
            return PTADD_ERR_CUDA;                                                \
        }                                                                         \
    } while (0)

// ------------------------------------------------------- source records
// Every segment i (node i -> nxt[i]) is described to the pair kernels by a
// 16-double record, rebuilt at the start of each step:
//   [0..2] x1 (start node)   [3] L      [4..6] unit tangent t   [7] 0
//   [8..10] Burgers vector b [11] 0     [12..14] q = b x t      [15] 0
constexpr int SRC_STRIDE = 16;
// FP32 record of the mixed path (16 floats):
//   [0..2] x1_hi  [3..5] x1_lo  [6] L  [7..9] t  [10..12] b  [13..15] q
// with x1 - origin = x1_hi + x1_lo, x1_hi integer-valued (exact in FP32 for
// |x1 - origin| < 2^24 l), so that a target can move x1 into a frame of its
// own (integer origin Ot nearby) as (x1_hi - Ot) + x1_lo with one rounding,
// and R0 = x - x1 keeps ~1e-7 relative accuracy for every pair.
constexpr int SRC32_STRIDE = 16;
// Near field of the mixed path: point-to-segment distance below 10 a, with a
// 1 % margin in favour of FP64 on the FP32 estimate of that distance.
constexpr double NEAR_FACTOR = 10.1;

// Device-side state of one realisation.
struct DevNetwork {
    int64_t n_nodes = 0, n_loops = 0;
    double* pos[2] = {nullptr, nullptr};  // SoA x|y|z (3*n), double-buffered
    int cur = 0;
    int32_t* nxt = nullptr;
    int32_t* prv = nullptr;
    int32_t* loop_of = nullptr;
    double* loop_b = nullptr;  // [n_loops*3] Burgers vectors in units of l
    double* loop_n = nullptr;  // [n_loops*3] unit normals
    uint8_t* pinned = nullptr;
    int32_t* tgt_burst = nullptr;  // segments with >= 1 unpinned node
    int64_t n_tgt_burst = 0;
    int32_t* tgt_all = nullptr;    // every segment
    double* src = nullptr;         // [n*SRC_STRIDE]
    float* src32 = nullptr;        // [n*SRC32_STRIDE] FP32 records of the mixed path
    double origin[3] = {0, 0, 0};  // integer-valued origin of the FP32 hi/lo split
    unsigned long long* near_count = nullptr;  // FP64 point-pairs of the mixed path
    double* k64 = nullptr;         // {a2, c1, c2} for the near-field path of the mixed kernel
    double* fpart = nullptr;       // [max_chunks*6*n] partial nodal-force parts
    int max_chunks = 0;
    double* vel = nullptr;         // SoA [3*n]
    double* force = nullptr;       // SoA [3*n] (last evaluated nodal force)
    double* partial = nullptr;     // [max_blocks*13]
    int max_red_blocks = 0;
    double* acc = nullptr;         // [16]: 0..8 sum Lp dt, 9 sum rho dt, 11 line length of the last
                                   // step, 12 time jumped over while stuck (junctions), 13..15 sum
                                   // (sum_s L vbar) dt (polar velocity)
    int* flag = nullptr;           // non-finite flag
    double* staging = nullptr;     // [3*n] AoS SI positions in / out
    int64_t* loop_off = nullptr;   // [n_loops + 1] first node of each loop (consistent mobility)
    double* cm_scratch = nullptr;  // [5*n] elimination factors of the consistent mobility
    double volume = 0;             // m^3
};

struct Consts {
    double a2;   // (a/l)^2
    double c1;   // 1/(8 pi)
    double c2;   // 1/(4 pi (1 - nu))
};

// ------------------------------------------------------------ launchers
// All return cudaGetLastError() of their launches.
cudaError_t launch_seg_prep(const DevNetwork& net, cudaStream_t st);
// pair stage: writes fpart[chunk][6][seg] for the listed targets
cudaError_t launch_pair(const DevNetwork& net, const int32_t* tgt, int64_t n_tgt, int chunks,
                        int precision, const Consts& c, const double sig_hat[6], cudaStream_t st);
// node stage: F = sum of parts, v = P F / M (0 if pinned); writes net.force / net.vel
cudaError_t launch_node_velocity(const DevNetwork& net, int chunks, cudaStream_t st);
// consistent mobility (Eq. 2.1 with its Galerkin mass matrix): M v = P F per
// loop, v = 0 at pinned nodes; replaces net.vel from net.force
cudaError_t launch_consistent_velocity(const DevNetwork& net, cudaStream_t st);
// the same on raw arrays (loops [loop_off[k], loop_off[k+1]) of n nodes, SoA
// positions, forces and velocities; scr: 5 n doubles), for the batch
cudaError_t launch_consistent_velocity_raw(int64_t n_loops, const int64_t* loop_off, const double* pos, int64_t n,
                                           const double* force, const uint8_t* pinned, const double* loop_n,
                                           double* vel, double* scr, cudaStream_t st);
// Lp/rho sample of the step-start state, Euler update into the other buffer,
// and the fixed-order reduction into net.acc (weighted by dt_hat)
cudaError_t launch_lp_euler(DevNetwork& net, double dt_hat, cudaStream_t st);
int choose_chunks(int64_t n_tgt, int64_t n_src, int max_chunks, int precision);

// peak microbenchmark
cudaError_t launch_fma_chains(int fp64, int blocks, int threads, long iters, double* sink, cudaStream_t st);

// junctions and thermally activated breaking (junctions.cu)
struct DevJunctions;
void junctions_free(ptadd_ctx* ctx);
// before the Euler stage of a step: release due junctions, form new ones,
// hold the velocities of held nodes, reduce the stuck test's inputs
cudaError_t launch_junction_update(ptadd_ctx* ctx, cudaStream_t st);
// after it: advance the DD clock by dt_s, or to the next break when stuck
// (adding the frozen interval to the rho and time sums in net.acc)
cudaError_t launch_junction_event(ptadd_ctx* ctx, double dt_s, double dt_hat, cudaStream_t st);
// junction part of the state blob
size_t junction_state_bytes(const ptadd_ctx* ctx);
ptadd_status junction_state_get(ptadd_ctx* ctx, char* dst);
ptadd_status junction_state_set(ptadd_ctx* ctx, const char* src);

struct DevBatch;
void batch_free(ptadd_ctx* ctx);
bool batch_has_junctions(const ptadd_ctx* ctx);
// junctions of a batched ensemble (junctions.cu)
struct DevBatchJunctions;
void batch_junctions_free(DevBatchJunctions*& j);
ptadd_status batch_junctions_create(DevBatchJunctions** out, const ptadd_junction_params* p, double len_unit,
                                    int32_t R, const std::vector<int64_t>& node_off, const std::vector<uint8_t>& pin,
                                    const std::vector<int32_t>& nxt, const std::vector<int32_t>& loop_of);
// release, capture search and hold of one step (after the velocity stage)
cudaError_t launch_batch_junction_update(DevBatchJunctions* j, const double* pos, const float* src32,
                                         const int32_t* nxt, const int32_t* loop_of, const int32_t* real_of,
                                         const int64_t* node_off_dev, const uint8_t* pinned, double* vel,
                                         cudaStream_t st);
// the per-realisation clock step or jump (after the reduction of the step into acc[16 r ..])
cudaError_t launch_batch_junction_event(DevBatchJunctions* j, double* acc, double dt_s, double dt_hat,
                                        double time_scale, cudaStream_t st);
// junction state with realisation-local node and loop numbers; info[R]
ptadd_status batch_junctions_get(DevBatchJunctions* j, const std::vector<int64_t>& node_off, cudaStream_t s,
                                 ptadd_junction_info* info, int32_t* seg, int32_t* last, int32_t* count,
                                 double* break_time);
struct MlpDev;
void mlp_free(ptadd_ctx* ctx);

}  // namespace ptadd

struct ptadd_ctx {
    int device = 0;
    ptadd_material mat{};
    int len_exp = 0;       // internal length unit l = 2^len_exp m
    double len_unit = 1.0; // l in metres
    ptadd_precision prec = PTADD_FP64;
    bool consistent_mass = false;  // ptadd_set_mobility
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    ptadd::DevNetwork net;
    bool have_net = false;
    ptadd::DevBatch* batch = nullptr;  // batched ensemble (ptadd_batch_*)
    ptadd::MlpDev* mlp = nullptr;      // surrogate (ptadd_mlp_* / ptadd_surrogate_*)
    ptadd::DevJunctions* junc = nullptr;  // junctions (ptadd_set_junctions), NULL: off
    double sig_app[6] = {0, 0, 0, 0, 0, 0};  // Pa
    // (1/|B|) sum_s L vbar of the last burst, time-averaged, SI (the polar velocity
    // of Eq. 2.11 divided by the core area)
    double last_LV[3] = {0, 0, 0};
    bool have_LV = false;
    // profiling (ptadd_profile_*)
    bool timing = false;
    int64_t kernel_launches = 0, pair_launches = 0, pair_evals = 0;
    double pair_ms = 0.0;
    unsigned long long near_base = 0;  // near_count at the last profile reset
    std::vector<cudaEvent_t> ev_pool;     // reusable events
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_open;  // recorded, not yet read
};
