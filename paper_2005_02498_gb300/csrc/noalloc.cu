// noalloc.cu -- ptadd_forces_noalloc: nodal forces of a loop network whose
// arrays already live on the device, computed without any device allocation.
//
// The scratch the force evaluation needs (internal-unit positions, source
// records, per-chunk partial nodal forces, ...) lives in one file-scope
// __device__ array sized for at most PTADD_NOALLOC_MAX_SEGMENTS segments.
// Every GPU on which the library's module is loaded holds that array (about
// 7 MB) until the process exits; with lazy module loading (the CUDA default)
// that happens at the first call on the device.  Host code cannot use the
// array's name as a device address: every call made outside stream capture
// looks the address up with cudaGetSymbolAddress (with the caller's device
// current) and caches it per device; a call under capture uses the cache.
//
// The caller's loop tables are checked on the device before anything indexes
// with them: na_prepare copies them into the scratch, replacing every entry
// that is out of range or breaks prv[nxt[i]] == i, nxt[prv[i]] == i by i (a
// zero-length segment) and setting an error word; every later kernel uses
// the copies, so a bad table never leads to an out-of-bounds access, and
// na_finish then writes NaN to every output force.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "ptadd_internal.cuh"

namespace ptadd {
namespace {

constexpr int64_t NA_MAX = PTADD_NOALLOC_MAX_SEGMENTS;
constexpr int NA_CHUNKS = 4;
// doubles per segment: positions 3, source record 16, partial forces 6 per
// chunk, force 3, velocity 3, Burgers vector 3, normal 3; then four int32
// tables (loop index, target list, checked nxt and prv copies) and the error
// word packed into the same array.
constexpr int64_t NA_DOUBLES_PER_SEG = 3 + SRC_STRIDE + 6 * NA_CHUNKS + 3 + 3 + 3 + 3;
// + 4*NA_MAX int32 (= 2*NA_MAX doubles) + slack for the 256-byte alignment of
// the regions (each pad < 32 doubles) and the error word
constexpr int64_t NA_DOUBLES = NA_DOUBLES_PER_SEG * NA_MAX + 2 * NA_MAX + 512;

static __device__ __align__(256) double g_noalloc_scratch[NA_DOUBLES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
double* g_na_ptr[NA_MAX_DEVICES] = {nullptr};

// Address of the scratch array on the current device.  Outside stream
// capture it is looked up on every call (a new primary context after a
// device reset reloads the module, and the array may move); under capture the
// address cached by the last uncaptured call on this device is used.
ptadd_status scratch_for_current_device(cudaStream_t s, double** out)
{
    int dev = 0;
    PTADD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEVICES) {
        set_error("device index %d out of range for ptadd_forces_noalloc", dev);
        return PTADD_ERR_ARG;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();  // e.g. the legacy stream while another stream captures: treat as capturing
        cs = cudaStreamCaptureStatusActive;
    }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (cs == cudaStreamCaptureStatusNone) {
        double* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress of the no-allocation scratch failed: %s", cudaGetErrorString(e));
            return PTADD_ERR_CUDA;
        }
        g_na_ptr[dev] = p;
    } else if (!g_na_ptr[dev]) {
        set_error("ptadd_forces_noalloc: the first call on a device must come before any stream capture");
        return PTADD_ERR_STATE;
    }
    *out = g_na_ptr[dev];
    return PTADD_OK;
}

// Also copies the loop tables, checked: an entry outside [0, n) is never
// used as an index, and an entry that breaks prv[nxt[i]] == i or
// nxt[prv[i]] == i is replaced by i and flagged in *err.
__global__ void na_prepare(int64_t n, const double* __restrict__ xyz, const double* __restrict__ burgers,
                           const int32_t* __restrict__ nxt_in, const int32_t* __restrict__ prv_in,
                           double pos_scale, double len_unit, double* __restrict__ pos, double* __restrict__ bseg,
                           double* __restrict__ nseg, int32_t* __restrict__ loop_of, int32_t* __restrict__ tgt,
                           int32_t* __restrict__ nxt, int32_t* __restrict__ prv, int* __restrict__ err)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t nx = nxt_in[i], pv = prv_in[i];
    const bool nx_in = nx >= 0 && nx < n, pv_in = pv >= 0 && pv < n;
    const bool ok = nx_in && pv_in && prv_in[nx] == (int32_t)i && nxt_in[pv] == (int32_t)i;
    nxt[i] = ok ? nx : (int32_t)i;
    prv[i] = ok ? pv : (int32_t)i;
    if (!ok) atomicOr(err, 1);
    for (int c = 0; c < 3; ++c) {
        pos[c * n + i] = xyz[3 * i + c] * pos_scale;  // power of two: exact
        bseg[3 * i + c] = burgers[3 * i + c] / len_unit;
        nseg[3 * i + c] = 0.0;
    }
    loop_of[i] = (int32_t)i;  // one Burgers vector per segment
    tgt[i] = (int32_t)i;
}

// NaN everywhere if the loop tables were rejected.
__global__ void na_finish(int64_t n, const double* __restrict__ force, double scale, const int* __restrict__ err,
                          double* __restrict__ F)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    F[i] = *err ? __longlong_as_double(0x7ff8000000000000ll) : force[(i % 3) * n + i / 3] * scale;
}

}  // namespace
}  // namespace ptadd

using namespace ptadd;

extern "C" ptadd_status ptadd_forces_noalloc(const ptadd_material* mat, int64_t n_nodes, const double* xyz_dev,
                                             const int32_t* nxt_dev, const int32_t* prv_dev,
                                             const double* burgers_dev, const double sig_app[6], double* F_dev,
                                             void* stream)
{
    if (!mat || !xyz_dev || !nxt_dev || !prv_dev || !burgers_dev || !sig_app || !F_dev) {
        set_error("ptadd_forces_noalloc: null argument");
        return PTADD_ERR_ARG;
    }
    if (!(mat->mu > 0) || !(mat->nu > -1.0 && mat->nu < 0.5) || !(mat->b > 0) || !(mat->a > 0) || !(mat->B > 0)) {
        set_error("ptadd_forces_noalloc: material out of range");
        return PTADD_ERR_ARG;
    }
    if (n_nodes < 2 || n_nodes > NA_MAX) {
        set_error("ptadd_forces_noalloc: n_nodes = %lld outside [2, %lld] (the size of its fixed scratch array)",
                  (long long)n_nodes, (long long)NA_MAX);
        return PTADD_ERR_ARG;
    }
    for (int c = 0; c < 6; ++c)
        if (!isfinite(sig_app[c])) {
            set_error("ptadd_forces_noalloc: non-finite applied stress");
            return PTADD_ERR_ARG;
        }
    cudaStream_t s = (cudaStream_t)stream;
    double* base = nullptr;
    ptadd_status st = scratch_for_current_device(s, &base);
    if (st != PTADD_OK) return st;

    const int64_t n = n_nodes;
    const int len_exp = (int)lround(log2(mat->b));
    const double len_unit = ldexp(1.0, len_exp);

    // carve the scratch (offsets in doubles; every region 256-byte aligned)
    auto align32 = [](int64_t x) { return (x + 31) & ~(int64_t)31; };
    int64_t off = 0;
    DevNetwork net;
    net.n_nodes = n;
    net.n_loops = n;
    net.pos[0] = base + off; off = align32(off + 3 * n);
    net.src = base + off;    off = align32(off + SRC_STRIDE * n);
    net.fpart = base + off;  off = align32(off + 6 * NA_CHUNKS * n);
    net.force = base + off;  off = align32(off + 3 * n);
    net.vel = base + off;    off = align32(off + 3 * n);
    net.loop_b = base + off; off = align32(off + 3 * n);
    net.loop_n = base + off; off = align32(off + 3 * n);
    int32_t* ints = reinterpret_cast<int32_t*>(base + off);
    net.loop_of = ints;
    int32_t* tgt = ints + align32(n);
    net.nxt = tgt + align32(n);
    net.prv = net.nxt + align32(n);
    int* err = reinterpret_cast<int*>(net.prv + align32(n));
    net.pinned = nullptr;
    net.cur = 0;
    net.max_chunks = NA_CHUNKS;

    const unsigned blk = (unsigned)((n + 255) / 256);
    PTADD_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    na_prepare<<<blk, 256, 0, s>>>(n, xyz_dev, burgers_dev, nxt_dev, prv_dev, ldexp(1.0, -len_exp), len_unit,
                                   net.pos[0], net.loop_b, net.loop_n, net.loop_of, tgt, net.nxt, net.prv, err);
    PTADD_CUDA(cudaGetLastError());
    Consts c;
    const double r = mat->a / len_unit;
    c.a2 = r * r;
    c.c1 = 1.0 / (8.0 * M_PI);
    c.c2 = 1.0 / (4.0 * M_PI * (1.0 - mat->nu));
    double sh[6];
    for (int k = 0; k < 6; ++k) sh[k] = sig_app[k] / mat->mu;
    const int chunks = choose_chunks(n, n, NA_CHUNKS, (int)PTADD_FP64);
    PTADD_CUDA(launch_seg_prep(net, s));
    PTADD_CUDA(launch_pair(net, tgt, n, chunks, (int)PTADD_FP64, c, sh, s));
    PTADD_CUDA(launch_node_velocity(net, chunks, s));
    na_finish<<<(unsigned)((3 * n + 255) / 256), 256, 0, s>>>(n, net.force, mat->mu * len_unit * len_unit, err,
                                                              F_dev);
    PTADD_CUDA(cudaGetLastError());
    return PTADD_OK;
}
