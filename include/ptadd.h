/*
 * ptadd.h -- C ABI of the GPU discrete-dislocation-dynamics (DD) burst used
 * by Practical Time Averaging (PTA) to close mesoscale plasticity
 * (arXiv:2005.02498, "Plasticity without phenomenology: a first step").
 *
 * The problem the calls follow (Sec. 2.1, 2.3, 2.4): given a network of
 * closed dislocation loops (straight segments between nodes), their Burgers
 * vectors and glide normals, and an applied stress held fixed (the load l_t
 * of Eq. 2.4), run the fast DD dynamics for a burst of explicit Euler steps
 * and return the running time averages (Eq. 2.5) of the plastic distortion
 * rate Lp (Sec. 2.2, Eq. 2.9) and of the line density rho (Sec. 2.4).
 *
 * One DD step (Sec. 2.1):
 *   1. sigma(x_q) = sigma_app + sum over ALL segments of the nonsingular
 *      isotropic stress of a straight segment (sigma = S R * alpha, Sec. 2.1;
 *      R replaced by R_a = sqrt(R.R + a^2)), at the 4 Gauss-Legendre points
 *      x_q of every target segment;
 *   2. Peach-Koehler force per length f_q = (sigma(x_q) b) x t (Sec. 2.1),
 *      assembled to nodes with linear shape functions;
 *   3. lumped glide mobility v_a = (I - n n) F_a / (B M_a),
 *      M_a = (L_prev + L_next)/2, v_a = 0 at pinned nodes (Eq. 2.1);
 *   4. Lp_i = (1/V) sum_s L_s b_s (x) (t_s x vbar_s), rho_i = (1/V) sum_s L_s,
 *      evaluated on the step-start state and accumulated with weight dt;
 *   5. x_a <- x_a + v_a dt for all nodes at once.
 *
 * Conventions
 *   - SI units at the boundary: m, Pa, s, N.  Stresses are Voigt 6-vectors in
 *     the order xx, yy, zz, yz, xz, xy.  Lp is a row-major 3x3 matrix (1/s).
 *   - Every call returns a ptadd_status.  Nothing aborts the process.  After
 *     an error the message is available from ptadd_last_error(); the context
 *     stays usable unless the status is PTADD_ERR_CUDA from a sticky device
 *     error.
 *   - Host arrays passed in are copied; the caller keeps ownership.  Device
 *     pointers ("_dev" calls) must stay valid until the call's work on the
 *     context's stream has completed.
 *   - A context is not thread-safe; use one context per host thread.
 *   - All device memory a context needs is allocated by the calls that
 *     create it or load data into it (ptadd_create, ptadd_set_network,
 *     ptadd_batch_set / ptadd_batch_run, the ptadd_mlp_* and
 *     ptadd_surrogate_* calls) and freed by ptadd_destroy.  ptadd_gemm_bf16
 *     allocates and frees its own buffers; ptadd_forces_noalloc allocates
 *     nothing.
 */
#ifndef PTADD_H
#define PTADD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PTADD_VERSION_MAJOR 0
#define PTADD_VERSION_MINOR 2

typedef struct ptadd_ctx ptadd_ctx; /* opaque; owns its device memory and stream */

typedef enum {
    PTADD_OK = 0,
    PTADD_ERR_ARG = 1,       /* invalid argument (size, pointer, non-unit normal, ...) */
    PTADD_ERR_CUDA = 2,      /* a CUDA runtime call failed                              */
    PTADD_ERR_NONFINITE = 3, /* a burst produced NaN/Inf (positions or averages)        */
    PTADD_ERR_TIMEOUT = 4,   /* a bounded device-side wait gave up                      */
    PTADD_ERR_STATE = 5,     /* call out of order (e.g. advance before set_network)     */
    PTADD_ERR_NOMEM = 6      /* device allocation failed                                */
} ptadd_status;

/* Isotropic material and the drag law (SI).  a is the core width of the
 * nonsingular field; b the reference Burgers-vector magnitude (the unit of
 * length inside the kernels); B the scalar drag coefficient of Eq. 2.1. */
typedef struct {
    double mu; /* shear modulus, Pa */
    double nu; /* Poisson ratio     */
    double b;  /* |b|, m            */
    double a;  /* core width, m     */
    double B;  /* drag, Pa s        */
} ptadd_material;

typedef enum {
    PTADD_FP64 = 0, /* every pair interaction in FP64                                  */
    PTADD_MIXED = 1 /* pairs farther than 10a in FP32 (compensated), nearer in FP64;   *
                     * positions, forces and averages always FP64                      */
} ptadd_precision;

/* Static description of the loaded network and of the work of one step. */
typedef struct {
    int64_t n_nodes;
    int64_t n_loops;
    int64_t n_targets;      /* segments whose force is evaluated (>= 1 unpinned node) */
    int64_t pairs_per_step; /* n_targets * n_nodes: segment-pair evaluations per step */
    int32_t precision;      /* ptadd_precision                                        */
    int32_t device;
} ptadd_info;

/* ---------------------------------------------------------------- lifetime */
/* Library version as major*1000 + minor. */
int ptadd_version(void);

/* Create a context on CUDA device `device` (it is made current).  mat must
 * have mu > 0, -1 < nu < 0.5, b > 0, a > 0, B > 0. */
ptadd_status ptadd_create(ptadd_ctx** out, const ptadd_material* mat, ptadd_precision prec, int device);
/* Synchronise the context's stream, then free everything the context owns
 * (device buffers, graphs, events, its own stream; a caller's stream set by
 * ptadd_set_stream is left alone).  NULL is a no-op. */
void ptadd_destroy(ptadd_ctx* ctx);

/* Message of the last failed call on this host thread (never NULL). */
const char* ptadd_last_error(void);

/* Switch precision of later bursts. */
ptadd_status ptadd_set_precision(ptadd_ctx* ctx, ptadd_precision prec);

/* Run the context's work on a caller-owned stream (a cudaStream_t passed as
 * void*; NULL restores the context's own stream). */
ptadd_status ptadd_set_stream(ptadd_ctx* ctx, void* stream);

/* ----------------------------------------------------------------- network */
/* Load one realisation (host arrays, copied).  Loops are closed rings: loop k
 * owns nodes [loop_off[k], loop_off[k+1]) in order (line sense = node order,
 * segment i runs from node i to the next node of its loop, wrapping).
 *   xyz[n_nodes*3]       node positions, m
 *   loop_off[n_loops+1]  loop_off[0] = 0, increasing, loop_off[n_loops] = n_nodes,
 *                        every loop has >= 2 nodes
 *   burgers[n_loops*3]   Burgers vector per loop, m
 *   normal[n_loops*3]    glide normal per loop, | |n| - 1 | <= 1e-9
 *   pinned[n_nodes]      1 = sessile node (never moves); NULL = none pinned.
 *                        Segments whose two nodes are pinned act as sources
 *                        only: their own force is not evaluated.
 *   volume               averaging volume |B_x| of Sec. 2.2, m^3, > 0
 * Resets the running averages and the applied stress to zero. */
ptadd_status ptadd_set_network(ptadd_ctx* ctx, int64_t n_nodes, const double* xyz,
                               int64_t n_loops, const int64_t* loop_off,
                               const double* burgers, const double* normal,
                               const uint8_t* pinned, double volume);

/* Applied stress sigma_app (Pa, Voigt order), uniform over the box. */
ptadd_status ptadd_set_applied_stress(ptadd_ctx* ctx, const double sig[6]);

/* Sizes of the loaded network into *info (caller-owned): nodes, loops,
 * target segments (those with an unpinned node), segment pairs per DD step
 * (targets x sources), precision and device.  PTADD_ERR_STATE without a
 * network; PTADD_ERR_ARG for NULL arguments. */
ptadd_status ptadd_get_info(const ptadd_ctx* ctx, ptadd_info* info);

/* ------------------------------------------------------------------- burst */
/* Advance the loaded network by n_steps >= 0 Euler steps of dt > 0 s and
 * return R^Lp (row-major 3x3, 1/s) and R^rho (1/m^2), the averages of Eq. 2.5
 * over the n_steps step-start states of this call.  Either output may be
 * NULL.  Positions stay on the device.  Returns PTADD_ERR_NONFINITE if a
 * position or an average is not finite (the positions are then undefined). */
ptadd_status ptadd_advance(ptadd_ctx* ctx, int64_t n_steps, double dt,
                           double Lp_avg[9], double* rho_avg);

/* Polar dislocation velocity of the last burst (Sec. 2.4, Eq. 2.11; Eq. 2.5
 * for its running average): the volume-averaged dislocation velocity
 *   V = (1/|B|) sum_s vbar_s l_s A_s,
 * with vbar_s the velocity of segment s (the mean of its two nodal
 * velocities, the one that gives Lp = alpha x V segment by segment), l_s its
 * length, |B| the network's volume and A_s = core_area (m^2) the core
 * cross-section of every segment, which the paper takes as |b|^2 up to a
 * constant and leaves to the caller.  The burst sums l_s vbar_s in the same
 * reduction as Lp and rho, so the call only scales them: V_avg[3] (m/s).
 * PTADD_ERR_STATE before the first ptadd_advance after ptadd_set_network;
 * PTADD_ERR_ARG for a non-positive core_area. */
ptadd_status ptadd_get_polar_velocity(ptadd_ctx* ctx, double core_area, double V_avg[3]);

/* Current node positions (m) into host xyz[n_nodes*3] (caller-owned, node
 * order of ptadd_set_network); synchronises the stream.  PTADD_ERR_STATE
 * without a network; PTADD_ERR_ARG for a NULL array. */
ptadd_status ptadd_get_nodes(ptadd_ctx* ctx, double* xyz);

/* Replace the positions of the loaded network (host xyz[n_nodes*3], m; same
 * topology).  The array is copied to the device as is (pinned host memory
 * gives a direct DMA) and converted there.  Resets nothing else. */
ptadd_status ptadd_set_nodes(ptadd_ctx* ctx, const double* xyz);

/* Nodal forces (N) at the current positions into host F[n_nodes*3]: the
 * Peach-Koehler force (Sec. 2.1) of the nonsingular stress of every segment
 * plus the applied stress, integrated against the linear shape functions
 * with the 4-point Gauss rule, in the context's precision; every segment is
 * evaluated (pinned ones included).  PTADD_ERR_STATE without a network;
 * PTADD_ERR_ARG for a NULL array. */
ptadd_status ptadd_get_forces(ptadd_ctx* ctx, double* F);

/* Same as ptadd_get_forces into a device buffer F_dev[n_nodes*3] (N),
 * enqueued on the context's stream; returns without synchronising. */
ptadd_status ptadd_get_forces_dev(ptadd_ctx* ctx, double* F_dev);

/* Serialise the positions (so a burst can resume where the last ended, the
 * PTA carry-over of Sec. 2.5) into buf.  Call with buf = NULL to get the size
 * in *bytes; otherwise *bytes must hold the buffer size. */
ptadd_status ptadd_get_state(ptadd_ctx* ctx, void* buf, size_t* bytes);
/* Restore positions (and, while junctions are on, the junction state) from a
 * blob of ptadd_get_state taken on the same network.  PTADD_ERR_ARG if the
 * size or the header does not match (another network, or junctions on in
 * one and off in the other); PTADD_ERR_STATE without a network.  The blob
 * stays the caller's. */
ptadd_status ptadd_set_state(ptadd_ctx* ctx, const void* buf, size_t bytes);

/* ------------------------------------------------------------------ batched */
/* R independent realisations advanced together (the independent bursts of
 * the blocks / material points of the paper's coupling, Sec. 4.1, which it
 * runs "in parallel").  Realisation r owns nodes [node_off[r], node_off[r+1])
 * of the concatenated arrays; loops use GLOBAL node indices and must not
 * straddle realisations.  Per realisation: its applied stress sig6[6r..6r+5]
 * (Pa) and averaging volume volume[r] (m^3).  The precision of the context
 * applies.  The pair stage is one persistent kernel that pulls (realisation,
 * target tile, source chunk) work items, largest first, from an atomic
 * counter; two steps are captured once into a CUDA graph and replayed.
 * A batch lives beside (not instead of) the single network of the context. */
typedef struct {
    int32_t R;
    int64_t n_nodes, n_loops, n_targets;
    int64_t pairs_per_step; /* sum over realisations of n_targets_r * n_nodes_r */
    int64_t work_items;     /* tiles of the persistent pair kernel per step    */
    int32_t tile_targets;   /* autotuned: targets per tile (threads per block)  */
    int32_t chunk_sources;  /* autotuned: sources per work item                 */
    int32_t tuned;          /* 1 if the configuration came from the tuner/cache */
} ptadd_batch_info;

/* Load a batch (host arrays, copied; layout as above): node_off[R+1] with
 * node_off[0] = 0 and >= 2 nodes per realisation, loop_off[n_loops+1],
 * xyz[n*3] (m), burgers and normal [n_loops*3], pinned[n] (NULL: none),
 * sig6[R*6] (Pa), volume[R] (m^3).  Replaces any earlier batch and resets
 * its running averages.  PTADD_ERR_ARG on NULL arrays, R < 1, offset
 * tables that do not run from 0 to n_nodes, a loop or realisation of fewer
 * than 2 nodes, a loop that straddles realisations, a volume that is not
 * positive and finite, or more than 2^31 - 1 nodes. */
ptadd_status ptadd_batch_set(ptadd_ctx* ctx, int32_t R, const int64_t* node_off, int64_t n_loops,
                             const int64_t* loop_off, const double* xyz, const double* burgers,
                             const double* normal, const uint8_t* pinned, const double* sig6,
                             const double* volume);
/* New applied stresses sig6[R*6] (Pa) for the loaded batch; positions kept. */
ptadd_status ptadd_batch_set_stress(ptadd_ctx* ctx, const double* sig6);
/* Burst of n_steps for every realisation: Lp_avg[R*9] (row-major, 1/s) and
 * rho_avg[R] (1/m^2), the averages of Eq. 2.5; either may be NULL. */
ptadd_status ptadd_batch_advance(ptadd_ctx* ctx, int64_t n_steps, double dt, double* Lp_avg, double* rho_avg);
/* R^V of the last batch burst per realisation (as ptadd_get_polar_velocity,
 * with each realisation's own volume): V_avg[R*3] (m/s). */
ptadd_status ptadd_batch_get_polar_velocity(ptadd_ctx* ctx, double core_area, double* V_avg);
/* Positions of every realisation (concatenated, m) into / from host
 * xyz[n_nodes*3] (caller-owned); set_nodes keeps the topology, stresses and
 * junctions.  PTADD_ERR_STATE without a batch; PTADD_ERR_ARG for NULL. */
ptadd_status ptadd_batch_get_nodes(ptadd_ctx* ctx, double* xyz);
ptadd_status ptadd_batch_set_nodes(ptadd_ctx* ctx, const double* xyz);
/* Sizes and the pair-stage configuration of the loaded batch into *info.
 * PTADD_ERR_STATE without a batch; PTADD_ERR_ARG for NULL. */
ptadd_status ptadd_batch_get_info(ptadd_ctx* ctx, ptadd_batch_info* info);
/* Time the pair stage of the loaded batch for every candidate (tile of 64 or
 * 128 targets x chunks of 1024/2048/4096 sources), keep the fastest, and
 * append it to a JSON-lines cache (cache_path, else $PTADD_TUNE_CACHE, else
 * $HOME/.cache/ptadd_tune.jsonl) keyed by GPU, library version, a hash of
 * the sources the library was built from, precision and the batch's size
 * class.  A cached entry is reused unless force != 0.
 * ptadd_batch_set applies a cached entry when one exists. */
ptadd_status ptadd_batch_autotune(ptadd_ctx* ctx, const char* cache_path, int force);
/* Set the pair-stage configuration by hand: tile_targets (threads per
 * block) 64 or 128, chunk_sources a multiple of 128 in [1024, 2^24].  A
 * realisation of N nodes is then split into ceil(N / chunk_sources) source
 * chunks, each a separate work item whose nodal-force parts the node stage
 * sums in chunk order.  Results equal those of any other configuration up to
 * the summation order.  Marks the batch untuned (info.tuned = 0).
 * PTADD_ERR_ARG outside those values, PTADD_ERR_STATE without a batch. */
ptadd_status ptadd_batch_configure(ptadd_ctx* ctx, int32_t tile_targets, int32_t chunk_sources);
/* Nodal forces F[n_nodes*3] (N) of every realisation at the current
 * positions, as the burst's step would evaluate them (Sec. 2.1: the
 * Peach-Koehler force of the nonsingular stress of all segments of the
 * realisation plus its applied stress, integrated against the linear shape
 * functions with the 4-point Gauss rule), in the context's precision.  The
 * burst does not evaluate segments whose nodes are all pinned (sessile
 * obstacles, sources only), so the entries of pinned nodes are 0; the
 * entries of every other node are complete.  Positions are not changed. */
ptadd_status ptadd_batch_get_forces(ptadd_ctx* ctx, double* F);
/* ptadd_batch_set followed by ptadd_batch_advance. */
ptadd_status ptadd_batch_run(ptadd_ctx* ctx, int32_t R, const int64_t* node_off, int64_t n_loops,
                             const int64_t* loop_off, const double* xyz, const double* burgers,
                             const double* normal, const uint8_t* pinned, const double* sig6,
                             const double* volume, int64_t n_steps, double dt, double* Lp_avg,
                             double* rho_avg);

/* ---------------------------------------------------------- tensor cores */
/* C[M x N] = A[M x K] * B[N x K]^T on the tensor cores (tcgen05.mma, FP32
 * accumulation in tensor memory).  Host arrays: A and B hold BF16 bit
 * patterns (uint16), K contiguous; C is FP32 row-major.  N a multiple of 16
 * in [16, 256], K a multiple of 16.  Allocates its own device buffers; the
 * surrogate's training uses the same GEMM kernel.  Returns PTADD_ERR_TIMEOUT
 * if a bounded wait for the tensor core gave up. */
ptadd_status ptadd_gemm_bf16(int device, int64_t M, int32_t N, int32_t K, const uint16_t* A, const uint16_t* B,
                             float* C);
/* Self-test of the bounded tensor-core waits; it has no counterpart in the
 * paper.  Runs the GEMM kernel above once (M = 128, N = K = 64, zero
 * operands) with the MMAs and their commit withheld, so the mbarrier phase
 * that every thread waits on never completes: each wait gives up after its
 * iteration limit (about 2 s of SM clocks), the kernel sets its error word,
 * frees its tensor memory and returns, and the call reports
 * PTADD_ERR_TIMEOUT -- the expected result.  PTADD_OK would mean a wait
 * completed without its arrival.  The device and the library stay usable
 * afterwards. */
ptadd_status ptadd_gemm_timeout_selftest(int device);

/* -------------------------------------------------------------- surrogate */
/* A learned stand-in for the PTA closure (not in the paper): an MLP
 * 30 -> 256 -> 256 -> 256 -> 6 with GELU hidden layers, BF16 weights and
 * activations and FP32 accumulation on the tensor cores, FP32 master weights,
 * trained with Adam (beta 0.9/0.999, eps 1e-8) on the mean-square error.
 * Parameters are exchanged packed per layer as W (out x in, row-major) then b,
 * FP32, ptadd_mlp_param_count() values in all. */
int64_t ptadd_mlp_param_count(void);
/* Glorot-uniform weights from a splitmix64 stream of `seed`, zero biases. */
ptadd_status ptadd_mlp_init(ptadd_ctx* ctx, uint64_t seed);
/* Copy all parameters in (set: also resets Adam's moments) or out, packed
 * as above; params[count] is host memory of the caller, count must equal
 * ptadd_mlp_param_count() (else PTADD_ERR_ARG).  get before init or set:
 * PTADD_ERR_STATE. */
ptadd_status ptadd_mlp_set_params(ptadd_ctx* ctx, const float* params, int64_t count);
ptadd_status ptadd_mlp_get_params(ptadd_ctx* ctx, float* params, int64_t count);
/* Loss and gradient (packed like the parameters) of one forward/backward pass
 * over n normalised samples (host xn[n*30], yn[n*6]); no update. */
ptadd_status ptadd_mlp_loss_grad(ptadd_ctx* ctx, int64_t n, const float* xn, const float* yn, float* grad,
                                 float* loss);
/* Adam training on normalised samples: `epochs` passes over a seeded
 * shuffle, full batches of `batch` (a multiple of 16) only.  loss_per_epoch
 * (or NULL) receives the mean batch loss of each epoch. */
ptadd_status ptadd_mlp_train(ptadd_ctx* ctx, int64_t n, const float* xn, const float* yn, int epochs, int batch,
                             float lr, uint64_t seed, float* loss_per_epoch);
/* Forward pass on normalised inputs (host arrays xn[n*30] -> yn[n*6]). */
ptadd_status ptadd_mlp_forward(ptadd_ctx* ctx, int64_t n, const float* xn, float* yn);

/* Closure level.  Raw features per point, feat[n*30]: the 6 applied-stress
 * components (Pa, Voigt order), the 12 mobile then the 12 sessile line
 * densities per FCC slip system (1/m^2); labels lp6[n*6]: sym(Lp) in Voigt
 * order (1/s).  Inputs are mapped to [sigma/200 MPa, log10(rho + 1e10)] and
 * standardised, labels standardised, with the training set's moments.  The
 * trust region of a point: inside the per-feature [min, max] box of the
 * training inputs, and a Mahalanobis distance (training covariance) within the
 * training set's 99th percentile.  fit (re)trains from the
 * current weights (initialised from `seed` if none). */
ptadd_status ptadd_surrogate_fit(ptadd_ctx* ctx, int64_t n, const double* feat, const double* lp6, int epochs,
                                 int batch, float lr, uint64_t seed, float* loss_per_epoch);
/* Host arrays; in_region (or NULL) receives 1 inside the trust region.
 * Prediction runs one fused kernel (input map, trust region, the four layers,
 * output map) on the tensor cores with FP16 operands (the BF16 weights
 * convert to FP16 exactly in its normal range; inputs and activations are
 * rounded to FP16) and FP32 accumulation.  Its GELU evaluates erf through
 * tanh(x (A + B x^2)), a fit with |error| <= 2.8e-4, in f16x2 arithmetic, at
 * the size of the FP16 rounding of the stored activations; so its answers
 * can differ from ptadd_mlp_forward (BF16 activations, exact erf) at the
 * level of those roundings (4.9e-4 relative against the FP64 reference in
 * the tests). */
ptadd_status ptadd_surrogate_predict(ptadd_ctx* ctx, int64_t n, const double* feat, double* lp6, uint8_t* in_region);
/* Device arrays, enqueued on the context's stream without synchronising. */
ptadd_status ptadd_surrogate_predict_dev(ptadd_ctx* ctx, int64_t n, const double* feat_dev, double* lp6_dev,
                                         uint8_t* in_region_dev);

/* Closure sweep: one closure per point of a mesoscale load path (the PTA
 * closure of Sec. 3 asked for at many material points).  Per point i:
 * sig6[6i..] (Pa, Voigt order) and rho24[24i..] (12 mobile then 12 sessile
 * line densities per FCC slip system, 1/m^2, systems in the order of
 * ptadd_closure_realisation).  Points inside the fitted surrogate's trust
 * region take its answer; the others fall back to DD: the mean of sym(R^Lp)
 * (Eq. 2.5, Voigt order) over `ens` realisations from
 * ptadd_closure_realisation (segments/32 loops; realisation q of the sweep
 * uses seed ^ (q * 0x9E3779B97F4A7C15), q = index among the fallback points
 * * ens + member), all run as batched bursts of `steps` steps of dt (s) in
 * the context's precision.  Outputs: Lp_sym6[6 n_pts] (1/s) and
 * used_fallback[n_pts] (1 where DD answered; may be NULL).  Needs a fitted
 * surrogate (PTADD_ERR_STATE otherwise); segments a multiple of 32, >= 64.
 * Replaces the context's loaded batch; allocates device memory through the
 * surrogate and batch calls. */
ptadd_status ptadd_closure_sweep(ptadd_ctx* ctx, int64_t n_pts, const double* sig6, const double* rho24, int32_t ens,
                                 int64_t segments, int64_t steps, double dt, uint64_t seed, double* Lp_sym6,
                                 uint8_t* used_fallback);

/* One realisation for a closure input (host only, no GPU): n_loops circular
 * glide loops of 32 nodes following the 24 densities rho24 (1/m^2; 12
 * mobile then 12 sessile, FCC systems in the order: planes (111), (-111),
 * (1-11), (11-1), in each the <110> directions [01-1], [10-1], [1-10],
 * [011], [101], [110] that lie in it).  Class counts are the floor of
 * n_loops x share, plus one for the classes picked by systematic sampling of
 * the remainders; radii are stratified over (0.05, 0.2) um and line senses
 * balanced within each class; centres uniform in a cube whose volume makes
 * the total density exact; sessile loops pinned.  Random numbers: xoshiro256**
 * seeded by SplitMix64 from `seed`.  Outputs (caller-owned host arrays):
 * xyz[n_loops*32*3] (m), burgers[n_loops*3] (m, |b| = mat->b),
 * normal[n_loops*3], pinned[n_loops*32], *volume (m^3).  Loop l owns nodes
 * 32l .. 32l+31. */
ptadd_status ptadd_closure_realisation(const ptadd_material* mat, uint64_t seed, const double* rho24,
                                       int32_t n_loops, double* xyz, double* burgers, double* normal,
                                       uint8_t* pinned, double* volume);

/* Line density per slip system of one realisation (host only, no GPU): the
 * observable the closure inputs are made of (mobile and sessile density per
 * FCC {111}<110> system, Sec. 3.2.1, Sec. 2.4).  rho24[i] (i < 12) =
 * (1/V) x length of the segments of loops on system i with at least one
 * free node; rho24[12 + i] the same for segments whose two nodes are
 * pinned.  Systems in the order of ptadd_closure_realisation; a loop's
 * system is the one whose Burgers direction and plane normal are parallel
 * (to 1e-9) to its Burgers vector and glide normal.  Network arrays as in
 * ptadd_set_network (host, m).  PTADD_ERR_ARG on bad sizes, NULL arrays, a
 * non-positive volume, non-finite positions or a loop on no FCC system. */
ptadd_status ptadd_system_densities(int64_t n_nodes, const double* xyz, int64_t n_loops, const int64_t* loop_off,
                                    const double* burgers, const double* normal, const uint8_t* pinned, double volume,
                                    double* rho24);

/* Non-negative dissipation at a material point (Sec. 4, "Ensuring
 * non-negative dissipation"; host only, no GPU).  T6: Cauchy stress in
 * Voigt order xx, yy, zz, yz, xz, xy (any unit); Lp[9]: plastic distortion rate, row-major, corrected in
 * place: if T : Lp < 0 its component along T is removed (Lp -= (T:Lp) T /
 * |T|^2).  V[3] (or NULL): polar dislocation velocity, corrected in place
 * with alpha[9] (dislocation density tensor, row-major): if
 * beta = V . X(T alpha) < 0, V -= beta X(T alpha) / |X(T alpha)|^2, where
 * (X A)_i = e_ijk A_jk.  Zero T (or zero X(T alpha)) leaves the input as is.
 * PTADD_ERR_ARG on NULL T/Lp, V without alpha, or non-finite values. */
ptadd_status ptadd_dissipation_projection(const double T6[6], const double alpha[9], double Lp[9], double V[3]);
/* The same correction at n_points material points on the device (the Gauss
 * points of a mesh, the realisations of a batch), one thread per point.
 * Caller-owned DEVICE arrays: T6_dev[n*6], Lp_dev[n*9] (corrected in place),
 * alpha_dev[n*9] and V_dev[n*3] (both NULL, or both given; V corrected in
 * place).  A point with a non-finite value is left unchanged and counted in
 * *n_bad_dev (a device int the call zeroes first; NULL to skip the count).
 * Work is enqueued on `stream` (cudaStream_t as void*, NULL = legacy default
 * stream) without synchronising; allocates nothing.  PTADD_ERR_ARG on
 * n_points < 0 or a missing array. */
ptadd_status ptadd_dissipation_projection_dev(int64_t n_points, const double* T6_dev, const double* alpha_dev,
                                              double* Lp_dev, double* V_dev, int* n_bad_dev, void* stream);

/* Glide mobility of Eq. 2.1 (Sec. 2.1) for ptadd_advance and
 * ptadd_batch_advance on this context.
 * consistent = 0 (the default): the lumped form, v_a = (I - n n) F_a / (B M_a)
 * with M_a = (L_prev + L_next)/2.  consistent = 1: the consistent (Galerkin)
 * form with the linear shape functions, per loop sum_b B M_ab v_b = (I - n n)
 * F_a with M_aa = (L_prev + L_next)/3 and M_a,a+-1 = L/6 of the segment
 * between them, v = 0 at pinned nodes (and at a free node whose two segments
 * have zero length); n is the loop's glide normal.  The setting stays with
 * the context across networks and batches (ptadd_forces_noalloc computes
 * forces only).  PTADD_ERR_ARG for another value; PTADD_ERR_STATE for
 * consistent = 1 while junctions are on, single or batched (they hold nodes
 * at rest by the lumped form's rule). */
ptadd_status ptadd_set_mobility(ptadd_ctx* ctx, int32_t consistent);

/* Junctions and thermally activated breaking in the burst (Sec. 2.2).
 * Sessile segments are those whose two nodes are pinned.  In every step of
 * ptadd_advance, before the Euler update, each free node:
 *   - releases its junction when the DD clock has reached its break time;
 *   - if it holds none, forms one with the lowest-index sessile segment of
 *     another loop within capture_radius, except segments of the sessile
 *     loop it last broke away from; the junction breaks after t_b = f a
 *     (Eq. 2.2), a = max_break_time, f in [0,1) the top 53 bits of
 *     SplitMix64 output k+1 of the stream seeded with
 *     seed ^ (node * 0xD1B54A32D192ED03) for the node's k-th junction;
 *   - holds still (velocity 0) while it holds a junction.
 * After the update the clock advances by dt; when some junction is held and
 * no free node moved more than stuck_disp in the step, the clock instead
 * jumps to the earliest break time.  Over a jump the network is frozen: Lp
 * is 0 and rho keeps the step's value, and the averages of ptadd_advance
 * divide by the steps' time plus the jumps (Eq. 2.5).
 * p = NULL switches junctions off.  Setting them (again) clears every
 * junction and sets the clock to 0.  ptadd_set_network switches them off;
 * ptadd_set_nodes moves nodes and leaves the junctions as they are (a held
 * node stays held where it was put).
 * The state blob of ptadd_get_state carries the junction state while they
 * are on.  Single-realisation API (ptadd_batch_set_junctions below is the
 * batch's).  PTADD_ERR_ARG on negative or non-finite parameters;
 * PTADD_ERR_STATE without a network or with the consistent mobility on. */
typedef struct {
    double capture_radius;  /* m */
    double max_break_time;  /* a, s */
    double stuck_disp;      /* m per step */
    uint64_t seed;
} ptadd_junction_params;
ptadd_status ptadd_set_junctions(ptadd_ctx* ctx, const ptadd_junction_params* p);

typedef struct {
    double clock;     /* DD time since ptadd_set_junctions, s */
    double jumped;    /* time skipped while stuck, s */
    int64_t held;     /* junctions held now */
    int64_t formed;   /* junctions formed since ptadd_set_junctions */
    int64_t broken;
    int64_t jumps;
} ptadd_junction_info;
/* Junction state (Sec. 2.2, Eq. 2.2); the per-node arrays (caller-owned,
 * n_nodes each, any may be NULL): seg = held sessile segment or -1, last = sessile loop last
 * broken from or -1, count = junctions formed, break_time (s).
 * PTADD_ERR_STATE when junctions are off. */
ptadd_status ptadd_get_junctions(ptadd_ctx* ctx, ptadd_junction_info* info, int32_t* seg, int32_t* last,
                                 int32_t* count, double* break_time);

/* Junctions in a batched ensemble (Sec. 2.2, in each of the independent
 * bursts of Sec. 4.1): the rules of ptadd_set_junctions in every realisation
 * r, each with its own DD clock, stuck test and jumps; the break fractions of
 * realisation r come from the stream of seed ^ (r * 0x9E3779B97F4A7C15)
 * (unsigned 64-bit product) with the realisation-local node number, so that
 * realisation r behaves as it would alone under ptadd_set_junctions with
 * that seed (the capture search reaches the same segment: the lowest
 * position among the realisation's sessile segments, in node order).
 * ptadd_batch_advance's averages of realisation r divide by the steps' time
 * plus that realisation's jumps.  p = NULL switches them off; setting them
 * again clears every junction and every clock.  ptadd_batch_set switches
 * them off; ptadd_batch_set_nodes and ptadd_batch_set_stress leave them.
 * PTADD_ERR_STATE without a batch; PTADD_ERR_ARG on negative or non-finite
 * parameters. */
ptadd_status ptadd_batch_set_junctions(ptadd_ctx* ctx, const ptadd_junction_params* p);
/* The batch's junction state (Sec. 2.2, per realisation): info[R] (one per
 * realisation, caller-owned); the per-node arrays (n nodes
 * of the batch each, any may be NULL) in realisation-local numbers: seg =
 * start node of the held sessile segment within its realisation or -1, last
 * = loop (numbered from 0 within the realisation) last broken from or -1,
 * count = junctions formed, break_time (s, on the realisation's clock).
 * PTADD_ERR_STATE when the batch's junctions are off. */
ptadd_status ptadd_batch_get_junctions(ptadd_ctx* ctx, ptadd_junction_info* info, int32_t* seg, int32_t* last,
                                       int32_t* count, double* break_time);

/* Block stress average of the coupling (Sec. 4.2, the stress-averaging
 * block; host only, no GPU): <T>_r = sum_{g in r} w_g T_g / sum_{g in r} w_g
 * over the Gauss points g of block r.  T6[6g..]: stress at point g (Voigt
 * order, any unit); w[g] > 0: its volume weight (quadrature weight times
 * Jacobian, so that the weights of a block add up to its volume);
 * block[g] in [0, n_blocks).  T6_avg[6r..] (caller-owned) receives <T>_r.
 * Sums run in point order.  PTADD_ERR_ARG on NULL arrays, bad sizes, a block
 * index out of range, a weight that is not positive and finite, a
 * non-finite stress, or a block that holds no point. */
ptadd_status ptadd_block_average(int64_t n_gp, const double* T6, const double* w, const int32_t* block,
                                 int32_t n_blocks, double* T6_avg);

/* The two stresses one coupling increment k hands to PTA at each block
 * (Sec. 4.2.1, stress extrapolation and the minimum stress gap; host only):
 *   T6_prev[r] = <T>^k_r                                  (T^_{r,t-Delta})
 *   T6_t[r]    = <T>^k_r + (delta_star/dt_prev)(<T>^k_r - <T>^{k-1}_r)
 * and, when the gap |T6_t - T6_prev| (Frobenius norm of the full tensor) is
 * below gap_min, T6_t = T6_prev + mag (T6_t - T6_prev) with
 * mag[r] = gap_min / gap > 1, so that the gap is gap_min; otherwise mag = 1.
 * The rates PTA returns for block r are to be divided by mag[r].  A zero gap
 * leaves T6_t = T6_prev with mag = +inf (rates 0).  T6_km1 = NULL or
 * dt_prev <= 0 means no extrapolation (T6_t = <T>^k before the gap rule).
 * Arrays [n_blocks][6] (Voigt, any unit) and mag[n_blocks], caller-owned.
 * PTADD_ERR_ARG on NULL arrays, delta_star <= 0, gap_min < 0, or
 * non-finite values. */
ptadd_status ptadd_block_stress_pair(int32_t n_blocks, const double* T6_k, const double* T6_km1, double delta_star,
                                     double dt_prev, double gap_min, double* T6_prev, double* T6_t, double* mag);

/* Save / restore a fitted surrogate (weights, input/output maps, trust
 * region) as one blob; buf = NULL asks for the size. */
ptadd_status ptadd_surrogate_get_state(ptadd_ctx* ctx, void* buf, size_t* bytes);
/* Restore a blob of ptadd_surrogate_get_state (any context, same library
 * version); PTADD_ERR_ARG if its size or header does not match. */
ptadd_status ptadd_surrogate_set_state(ptadd_ctx* ctx, const void* buf, size_t bytes);

/* ------------------------------------------------------------- measurement */
/* Launch counters and CUDA-event timing of the pair-stress kernels, recorded
 * on the stream they are launched on.  Timing costs two event records per
 * pair launch and is off by default. */
typedef struct {
    int64_t kernel_launches; /* kernels this context launched since the last reset */
    int64_t pair_launches;   /* of which pair-stress kernels                         */
    int64_t pair_evals;      /* segment-pair evaluations those launches performed    */
    double pair_ms;          /* summed event time of the pair launches (timing on)   */
    int64_t near_point_pairs;/* PTADD_MIXED: (Gauss point, source) pairs evaluated   *
                              * in FP64 because nearer than 10a (4 per pair eval)    */
} ptadd_profile;

/* Reset the counters; enable (1) or disable (0) the event timing. */
ptadd_status ptadd_profile_reset(ptadd_ctx* ctx, int timing);
/* Read the counters (synchronises the context's stream). */
ptadd_status ptadd_profile_read(ptadd_ctx* ctx, ptadd_profile* out);

/* Throughput of dependent fused multiply-add chains on every SM of `device`
 * (fp64 = 1: FP64; 0: FP32; 2: packed FP32 pairs, two FMAs per
 * instruction), run for about `seconds`; *flops receives FLOP/s counting an
 * FMA as 2.  The non-tensor arithmetic peak the pair kernels are compared
 * against. */
ptadd_status ptadd_fma_peak(int device, int fp64, double seconds, double* flops);

/* ------------------------------------------------------ no device allocation */
/* Largest network ptadd_forces_noalloc accepts. */
#define PTADD_NOALLOC_MAX_SEGMENTS 16384

/* Nodal forces (N) of a network whose arrays are already on the device,
 * computed without allocating any device memory.  This call has no
 * counterpart in the paper; it exists for callers that cannot call
 * cudaMalloc: code running under another framework's memory pool, which owns
 * the device memory budget (a hidden cudaMalloc can fail there, or fragment
 * the pool), and latency-critical loops where cudaMalloc's implicit device
 * synchronisation would stall other streams.
 *
 * Same forces as ptadd_get_forces (FP64; every segment is a target).
 * Inputs and output are caller-owned DEVICE arrays:
 *   xyz_dev[n*3]      node positions, m
 *   nxt_dev[n]        index of the node after node i on its loop (segment i
 *                     runs i -> nxt[i]); prv_dev[n] the node before i.
 *                     Required: 0 <= nxt[i], prv[i] < n_nodes and
 *                     prv[nxt[i]] == nxt[prv[i]] == i for every i.  The
 *                     tables are checked on the device before any kernel
 *                     indexes with them; if an entry breaks the rule, no
 *                     out-of-range access happens and every output force
 *                     is NaN (the status, returned before the GPU ran, is
 *                     still PTADD_OK).
 *   burgers_dev[n*3]  Burgers vector of segment i, m
 *   sig_app[6]        HOST array, applied stress, Pa (Voigt order)
 *   F_dev[n*3]        output nodal forces, N
 *   stream            cudaStream_t as void* (NULL = legacy default stream)
 * 2 <= n_nodes <= PTADD_NOALLOC_MAX_SEGMENTS, else PTADD_ERR_ARG.
 * Call it with the device that owns `stream` and the arrays current
 * (cudaSetDevice): the scratch used is that device's.
 *
 * Scratch: one fixed array of about 7 MB in the library's device memory.
 * With lazy module loading (the CUDA default) the library's module, and with
 * it the array, is loaded on a device at the first call there: that first
 * call allocates device memory outside the caller's pool and may
 * synchronise the device, so make one warm-up call on each device before
 * entering a pool-managed region or a stream capture.  The array then stays
 * until the process exits.  Outside stream capture every call looks up the
 * array's device address (cudaGetSymbolAddress) afresh; a call under
 * capture reuses the address of the last uncaptured call on that device
 * (PTADD_ERR_STATE if there was none).  Every call on a device shares the
 * array: calls whose work overlaps on the GPU (other streams, other host
 * threads) race and corrupt each other's results -- serialise them.  The
 * call writes every scratch entry it reads, so nothing carries over from the
 * previous call.  Work is enqueued on `stream`; the call returns without
 * synchronising. */
ptadd_status ptadd_forces_noalloc(const ptadd_material* mat, int64_t n_nodes, const double* xyz_dev,
                                  const int32_t* nxt_dev, const int32_t* prv_dev, const double* burgers_dev,
                                  const double sig_app[6], double* F_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PTADD_H */
