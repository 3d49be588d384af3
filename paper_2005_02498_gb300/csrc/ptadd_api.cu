// ptadd_api.cu -- host entry points of ptadd.h (argument checks, device
// memory, unit conversion SI <-> internal units, kernel sequencing).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "ptadd_internal.cuh"

namespace ptadd {

static thread_local char g_err[1024] = "no error";

void set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

static ptadd_status arg_error(const char* msg)
{
    set_error("%s", msg);
    return PTADD_ERR_ARG;
}

template <typename T>
static ptadd_status dalloc(T** p, size_t count)
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

static void free_network(DevNetwork& n)
{
    void* ptrs[] = {n.pos[0], n.pos[1], n.nxt,   n.prv,   n.loop_of, n.loop_b,  n.loop_n, n.pinned, n.tgt_burst,
                    n.tgt_all, n.src,    n.fpart, n.vel,   n.force,   n.partial, n.acc,    n.flag,   n.staging,
                    n.src32,   n.near_count, n.k64, n.loop_off, n.cm_scratch};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    n = DevNetwork{};
}

static Consts make_consts(const ptadd_ctx* ctx)
{
    const ptadd_material& m = ctx->mat;
    Consts c;
    const double r = m.a / ctx->len_unit;
    c.a2 = r * r;
    c.c1 = 1.0 / (8.0 * M_PI);
    c.c2 = 1.0 / (4.0 * M_PI * (1.0 - m.nu));
    return c;
}

}  // namespace ptadd

using namespace ptadd;

#define CHECK_CTX(ctx)                                   \
    do {                                                 \
        if (!(ctx)) return arg_error("null context");    \
        PTADD_CUDA(cudaSetDevice((ctx)->device));        \
    } while (0)

extern "C" {

int ptadd_version(void) { return PTADD_VERSION_MAJOR * 1000 + PTADD_VERSION_MINOR; }

const char* ptadd_last_error(void) { return g_err; }

ptadd_status ptadd_create(ptadd_ctx** out, const ptadd_material* mat, ptadd_precision prec, int device)
{
    if (!out) return arg_error("out is NULL");
    *out = nullptr;
    if (!mat) return arg_error("material is NULL");
    if (!(mat->mu > 0) || !(mat->nu > -1.0 && mat->nu < 0.5) || !(mat->b > 0) || !(mat->a > 0) || !(mat->B > 0))
        return arg_error("material out of range (mu, b, a, B > 0; -1 < nu < 0.5)");
    if (prec != PTADD_FP64 && prec != PTADD_MIXED) return arg_error("unknown precision");
    int ndev = 0;
    PTADD_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return arg_error("device index out of range");
    PTADD_CUDA(cudaSetDevice(device));
    ptadd_ctx* c = new (std::nothrow) ptadd_ctx();
    if (!c) return arg_error("host allocation failed");
    c->device = device;
    c->mat = *mat;
    c->len_exp = (int)lround(log2(mat->b));
    c->len_unit = ldexp(1.0, c->len_exp);
    c->prec = prec;
    cudaError_t e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete c;
        set_error("cudaStreamCreate failed: %s", cudaGetErrorString(e));
        return PTADD_ERR_CUDA;
    }
    c->stream = c->own_stream;
    *out = c;
    return PTADD_OK;
}

void ptadd_destroy(ptadd_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    free_network(ctx->net);
    batch_free(ctx);
    mlp_free(ctx);
    junctions_free(ctx);
    for (auto& e : ctx->ev_open) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    for (auto e : ctx->ev_pool) cudaEventDestroy(e);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    delete ctx;
}

ptadd_status ptadd_set_precision(ptadd_ctx* ctx, ptadd_precision prec)
{
    if (!ctx) return arg_error("null context");
    if (prec != PTADD_FP64 && prec != PTADD_MIXED) return arg_error("unknown precision");
    ctx->prec = prec;
    return PTADD_OK;
}

ptadd_status ptadd_set_stream(ptadd_ctx* ctx, void* stream)
{
    if (!ctx) return arg_error("null context");
    ctx->stream = stream ? (cudaStream_t)stream : ctx->own_stream;
    return PTADD_OK;
}

ptadd_status ptadd_set_network(ptadd_ctx* ctx, int64_t n_nodes, const double* xyz, int64_t n_loops,
                               const int64_t* loop_off, const double* burgers, const double* normal,
                               const uint8_t* pinned, double volume)
{
    CHECK_CTX(ctx);
    if (n_nodes < 2 || n_loops < 1) return arg_error("need n_nodes >= 2 and n_loops >= 1");
    if (n_nodes > (int64_t)1 << 30) return arg_error("n_nodes too large (max 2^30)");
    if (!xyz || !loop_off || !burgers || !normal) return arg_error("null array");
    if (!(volume > 0) || !isfinite(volume)) return arg_error("volume must be positive and finite");
    if (loop_off[0] != 0 || loop_off[n_loops] != n_nodes) return arg_error("loop_off must start at 0 and end at n_nodes");
    for (int64_t k = 0; k < n_loops; ++k)
        if (loop_off[k + 1] - loop_off[k] < 2) return arg_error("every loop needs >= 2 nodes");
    const double b = ctx->mat.b;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < n_nodes; ++i)
        for (int c = 0; c < 3; ++c) {
            const double v = xyz[3 * i + c];
            if (!isfinite(v)) return arg_error("non-finite node position");
            lo[c] = fmin(lo[c], v);
            hi[c] = fmax(hi[c], v);
        }
    for (int c = 0; c < 3; ++c)
        if ((hi[c] - lo[c]) / b > 1.0e6) return arg_error("network extent exceeds 1e6 Burgers vectors");
    double origin[3];
    for (int c = 0; c < 3; ++c) origin[c] = rint(ldexp(0.5 * (lo[c] + hi[c]), -ctx->len_exp));
    for (int64_t k = 0; k < n_loops; ++k) {
        const double* nn = normal + 3 * k;
        const double nrm = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
        if (!(fabs(nrm - 1.0) <= 1e-9)) return arg_error("glide normals must be unit vectors");
        for (int c = 0; c < 3; ++c)
            if (!isfinite(burgers[3 * k + c])) return arg_error("non-finite Burgers vector");
    }

    junctions_free(ctx);
    free_network(ctx->net);
    ctx->have_net = false;
    DevNetwork& net = ctx->net;
    const int64_t n = n_nodes;
    net.n_nodes = n;
    net.n_loops = n_loops;
    net.volume = volume;
    for (int c = 0; c < 3; ++c) net.origin[c] = origin[c];

    // host-side tables
    std::vector<double> pos(3 * n);
    std::vector<int32_t> nxt(n), prv(n), lof(n), tb, ta(n);
    std::vector<double> lb(3 * n_loops), ln(3 * n_loops);
    const int ie = -ctx->len_exp;  // exact scaling to internal units
    for (int64_t i = 0; i < n; ++i) {
        pos[i] = ldexp(xyz[3 * i], ie);
        pos[n + i] = ldexp(xyz[3 * i + 1], ie);
        pos[2 * n + i] = ldexp(xyz[3 * i + 2], ie);
    }
    for (int64_t k = 0; k < n_loops; ++k) {
        const int64_t s = loop_off[k], e = loop_off[k + 1];
        for (int64_t i = s; i < e; ++i) {
            nxt[i] = (int32_t)((i + 1 < e) ? i + 1 : s);
            prv[i] = (int32_t)((i > s) ? i - 1 : e - 1);
            lof[i] = (int32_t)k;
        }
        for (int c = 0; c < 3; ++c) {
            lb[3 * k + c] = burgers[3 * k + c] / ctx->len_unit;
            ln[3 * k + c] = normal[3 * k + c];
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        ta[i] = (int32_t)i;
        if (!(pinned && pinned[i] && pinned[nxt[i]])) tb.push_back((int32_t)i);
    }
    net.n_tgt_burst = (int64_t)tb.size();
    net.max_chunks = 64;
    net.max_red_blocks = (int)((n + 255) / 256);

    ptadd_status st = PTADD_OK;
#define ALLOC(p, cnt)                              \
    if (st == PTADD_OK) st = dalloc(&(p), (cnt));
    ALLOC(net.pos[0], 3 * n);
    ALLOC(net.pos[1], 3 * n);
    ALLOC(net.nxt, n);
    ALLOC(net.prv, n);
    ALLOC(net.loop_of, n);
    ALLOC(net.loop_b, 3 * n_loops);
    ALLOC(net.loop_n, 3 * n_loops);
    ALLOC(net.pinned, n);
    ALLOC(net.tgt_burst, tb.size());
    ALLOC(net.tgt_all, n);
    ALLOC(net.src, SRC_STRIDE * n);
    ALLOC(net.fpart, (size_t)net.max_chunks * 6 * n);
    ALLOC(net.vel, 3 * n);
    ALLOC(net.force, 3 * n);
    ALLOC(net.partial, (size_t)net.max_red_blocks * 13);
    ALLOC(net.acc, 16);
    ALLOC(net.flag, 1);
    ALLOC(net.staging, 3 * n);
    ALLOC(net.src32, SRC32_STRIDE * n);
    ALLOC(net.near_count, 1);
    ALLOC(net.k64, 4);
    ALLOC(net.loop_off, n_loops + 1);
    ALLOC(net.cm_scratch, 5 * n);
#undef ALLOC
    if (st != PTADD_OK) {
        free_network(net);
        return st;
    }
    std::vector<uint8_t> pin(n, 0);
    if (pinned)
        for (int64_t i = 0; i < n; ++i) pin[i] = pinned[i] ? 1 : 0;
    cudaStream_t s = ctx->stream;
    PTADD_CUDA(cudaMemcpyAsync(net.pos[0], pos.data(), 3 * n * sizeof(double), cudaMemcpyHostToDevice, s));
    PTADD_CUDA(cudaMemcpyAsync(net.nxt, nxt.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    PTADD_CUDA(cudaMemcpyAsync(net.prv, prv.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    PTADD_CUDA(cudaMemcpyAsync(net.loop_of, lof.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    PTADD_CUDA(cudaMemcpyAsync(net.loop_b, lb.data(), 3 * n_loops * sizeof(double), cudaMemcpyHostToDevice, s));
    PTADD_CUDA(cudaMemcpyAsync(net.loop_n, ln.data(), 3 * n_loops * sizeof(double), cudaMemcpyHostToDevice, s));
    PTADD_CUDA(cudaMemcpyAsync(net.pinned, pin.data(), n, cudaMemcpyHostToDevice, s));
    PTADD_CUDA(cudaMemcpyAsync(net.loop_off, loop_off, (n_loops + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    if (!tb.empty())
        PTADD_CUDA(cudaMemcpyAsync(net.tgt_burst, tb.data(), tb.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    PTADD_CUDA(cudaMemcpyAsync(net.tgt_all, ta.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    PTADD_CUDA(cudaMemsetAsync(net.fpart, 0, (size_t)net.max_chunks * 6 * n * sizeof(double), s));
    PTADD_CUDA(cudaMemsetAsync(net.acc, 0, 16 * sizeof(double), s));
    PTADD_CUDA(cudaMemsetAsync(net.flag, 0, sizeof(int), s));
    PTADD_CUDA(cudaMemsetAsync(net.near_count, 0, sizeof(unsigned long long), s));
    const Consts kc = make_consts(ctx);
    const double k64[4] = {kc.a2, kc.c1, kc.c2, 0.0};
    PTADD_CUDA(cudaMemcpyAsync(net.k64, k64, sizeof(k64), cudaMemcpyHostToDevice, s));
    // host vectors die at return: make the copies complete first
    PTADD_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < 6; ++c) ctx->sig_app[c] = 0.0;
    ctx->have_net = true;
    ctx->have_LV = false;
    return PTADD_OK;
}

ptadd_status ptadd_set_applied_stress(ptadd_ctx* ctx, const double sig[6])
{
    if (!ctx) return arg_error("null context");
    if (!sig) return arg_error("sig is NULL");
    for (int c = 0; c < 6; ++c) {
        if (!isfinite(sig[c])) return arg_error("non-finite applied stress");
        ctx->sig_app[c] = sig[c];
    }
    return PTADD_OK;
}

ptadd_status ptadd_get_info(const ptadd_ctx* ctx, ptadd_info* info)
{
    if (!ctx || !info) return arg_error("null argument");
    if (!ctx->have_net) {
        set_error("no network loaded");
        return PTADD_ERR_STATE;
    }
    info->n_nodes = ctx->net.n_nodes;
    info->n_loops = ctx->net.n_loops;
    info->n_targets = ctx->net.n_tgt_burst;
    info->pairs_per_step = ctx->net.n_tgt_burst * ctx->net.n_nodes;
    info->precision = (int32_t)ctx->prec;
    info->device = ctx->device;
    return PTADD_OK;
}

static ptadd_status take_events(ptadd_ctx* ctx, std::pair<cudaEvent_t, cudaEvent_t>& ev)
{
    while (ctx->ev_pool.size() < 2) {
        cudaEvent_t e;
        PTADD_CUDA(cudaEventCreate(&e));
        ctx->ev_pool.push_back(e);
    }
    ev.first = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
    ev.second = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
    return PTADD_OK;
}

// forces at the current positions for a target list (into net.force, net.vel)
static ptadd_status eval_forces(ptadd_ctx* ctx, const int32_t* tgt, int64_t n_tgt)
{
    DevNetwork& net = ctx->net;
    const Consts c = make_consts(ctx);
    double sh[6];
    for (int k = 0; k < 6; ++k) sh[k] = ctx->sig_app[k] / ctx->mat.mu;
    const int chunks = choose_chunks(n_tgt, net.n_nodes, net.max_chunks, (int)ctx->prec);
    cudaStream_t s = ctx->stream;
    if (n_tgt < net.n_nodes)
        PTADD_CUDA(cudaMemsetAsync(net.fpart, 0, (size_t)chunks * 6 * net.n_nodes * sizeof(double), s));
    PTADD_CUDA(launch_seg_prep(net, s));
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (ctx->timing && n_tgt > 0) {
        ptadd_status st = take_events(ctx, ev);
        if (st != PTADD_OK) return st;
        PTADD_CUDA(cudaEventRecord(ev.first, s));
    }
    PTADD_CUDA(launch_pair(net, tgt, n_tgt, chunks, (int)ctx->prec, c, sh, s));
    if (ev.first) {
        PTADD_CUDA(cudaEventRecord(ev.second, s));
        ctx->ev_open.push_back(ev);
    }
    PTADD_CUDA(launch_node_velocity(net, chunks, s));
    ctx->kernel_launches += 2 + (n_tgt > 0 ? 1 : 0);
    if (n_tgt > 0) {
        ctx->pair_launches += 1;
        ctx->pair_evals += n_tgt * net.n_nodes;
    }
    return PTADD_OK;
}

// read and recycle the recorded event pairs (caller has synchronised)
static ptadd_status drain_events(ptadd_ctx* ctx)
{
    for (auto& e : ctx->ev_open) {
        float ms = 0.f;
        PTADD_CUDA(cudaEventElapsedTime(&ms, e.first, e.second));
        ctx->pair_ms += ms;
        ctx->ev_pool.push_back(e.first);
        ctx->ev_pool.push_back(e.second);
    }
    ctx->ev_open.clear();
    return PTADD_OK;
}

ptadd_status ptadd_set_mobility(ptadd_ctx* ctx, int32_t consistent)
{
    CHECK_CTX(ctx);
    if (consistent != 0 && consistent != 1) return arg_error("ptadd_set_mobility: consistent must be 0 or 1");
    if (consistent && (ctx->junc || batch_has_junctions(ctx))) {
        set_error("ptadd_set_mobility: the consistent mobility does not combine with junctions (switch them off first)");
        return PTADD_ERR_STATE;
    }
    ctx->consistent_mass = consistent == 1;
    return PTADD_OK;
}

ptadd_status ptadd_advance(ptadd_ctx* ctx, int64_t n_steps, double dt, double Lp_avg[9], double* rho_avg)
{
    CHECK_CTX(ctx);
    if (!ctx->have_net) {
        set_error("advance before set_network");
        return PTADD_ERR_STATE;
    }
    if (n_steps < 0) return arg_error("n_steps < 0");
    if (!(dt > 0) || !isfinite(dt)) return arg_error("dt must be positive and finite");
    DevNetwork& net = ctx->net;
    cudaStream_t s = ctx->stream;
    const double dt_hat = dt * ctx->mat.mu / ctx->mat.B;
    PTADD_CUDA(cudaMemsetAsync(net.acc, 0, 16 * sizeof(double), s));
    PTADD_CUDA(cudaMemsetAsync(net.flag, 0, sizeof(int), s));
    for (int64_t it = 0; it < n_steps; ++it) {
        ptadd_status st = eval_forces(ctx, net.tgt_burst, net.n_tgt_burst);
        if (st != PTADD_OK) return st;
        if (ctx->consistent_mass) {
            PTADD_CUDA(launch_consistent_velocity(net, s));
            ctx->kernel_launches += 1;
        }
        if (ctx->junc) {
            PTADD_CUDA(launch_junction_update(ctx, s));
            ctx->kernel_launches += 3;
        }
        PTADD_CUDA(launch_lp_euler(net, dt_hat, s));
        ctx->kernel_launches += 2;
        if (ctx->junc) {
            PTADD_CUDA(launch_junction_event(ctx, dt, dt_hat, s));
            ctx->kernel_launches += 1;
        }
    }
    double acc[16];
    int flag = 0;
    PTADD_CUDA(cudaMemcpyAsync(acc, net.acc, 16 * sizeof(double), cudaMemcpyDeviceToHost, s));
    PTADD_CUDA(cudaMemcpyAsync(&flag, net.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    PTADD_CUDA(cudaStreamSynchronize(s));
    {
        ptadd_status st = drain_events(ctx);
        if (st != PTADD_OK) return st;
    }
    // Eq. 2.5 with internal sums: R = (sum Lambda_hat dt_hat) / (sum dt_hat), then SI scale; the
    // time jumped over while stuck (junctions) counts with Lp = 0 and the step's rho
    const double l = ctx->len_unit;
    const double St = dt_hat * (double)n_steps + (ctx->junc ? acc[12] : 0.0);
    const double lp_scale = l * l * l * ctx->mat.mu / (ctx->mat.B * net.volume);
    const double rho_scale = l / net.volume;
    bool finite = (flag == 0);
    for (int m = 0; m < 10; ++m) finite = finite && isfinite(acc[m]);
    if (Lp_avg)
        for (int m = 0; m < 9; ++m) Lp_avg[m] = n_steps > 0 ? acc[m] / St * lp_scale : 0.0;
    if (rho_avg) *rho_avg = n_steps > 0 ? acc[9] / St * rho_scale : 0.0;
    // R^V of Eq. 2.11 without the factor A (applied by ptadd_get_polar_velocity):
    // (1/|B|) sum L vbar, in SI (L in l, v in l mu / B)
    const double v_scale = l * l * ctx->mat.mu / (ctx->mat.B * net.volume);
    for (int m = 0; m < 3; ++m) ctx->last_LV[m] = n_steps > 0 ? acc[13 + m] / St * v_scale : 0.0;
    ctx->have_LV = true;
    for (int m = 13; m < 16; ++m) finite = finite && isfinite(acc[m]);
    if (!finite) {
        set_error("burst produced a non-finite position or average");
        return PTADD_ERR_NONFINITE;
    }
    return PTADD_OK;
}

ptadd_status ptadd_get_polar_velocity(ptadd_ctx* ctx, double core_area, double V_avg[3])
{
    if (!ctx) return arg_error("null context");
    if (!V_avg) return arg_error("V_avg is NULL");
    if (!(core_area > 0) || !isfinite(core_area)) return arg_error("core_area must be positive and finite");
    if (!ctx->have_LV) {
        set_error("no burst has run since the network was set");
        return PTADD_ERR_STATE;
    }
    for (int m = 0; m < 3; ++m) V_avg[m] = core_area * ctx->last_LV[m];
    return PTADD_OK;
}

__global__ void soa_to_aos_scaled(int64_t n, const double* __restrict__ soa, double scale, double* __restrict__ aos)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    const int64_t node = i / 3, c = i % 3;
    aos[i] = soa[c * n + node] * scale;
}

__global__ void aos_to_soa_scaled(int64_t n, const double* __restrict__ aos, double scale, double* __restrict__ soa)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    const int64_t node = i / 3, c = i % 3;
    soa[c * n + node] = aos[i] * scale;
}

// SoA device array (internal units) -> host AoS (SI) via the staging buffer
static ptadd_status read_soa(ptadd_ctx* ctx, const double* dev, double scale, double* out)
{
    const int64_t n = ctx->net.n_nodes;
    soa_to_aos_scaled<<<(unsigned)((3 * n + 255) / 256), 256, 0, ctx->stream>>>(n, dev, scale, ctx->net.staging);
    PTADD_CUDA(cudaGetLastError());
    ctx->kernel_launches += 1;
    PTADD_CUDA(cudaMemcpyAsync(out, ctx->net.staging, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    PTADD_CUDA(cudaStreamSynchronize(ctx->stream));
    return PTADD_OK;
}

ptadd_status ptadd_get_nodes(ptadd_ctx* ctx, double* xyz)
{
    CHECK_CTX(ctx);
    if (!ctx->have_net) {
        set_error("no network loaded");
        return PTADD_ERR_STATE;
    }
    if (!xyz) return arg_error("xyz is NULL");
    return read_soa(ctx, ctx->net.pos[ctx->net.cur], ctx->len_unit, xyz);
}

ptadd_status ptadd_set_nodes(ptadd_ctx* ctx, const double* xyz)
{
    CHECK_CTX(ctx);
    if (!ctx->have_net) {
        set_error("no network loaded");
        return PTADD_ERR_STATE;
    }
    if (!xyz) return arg_error("xyz is NULL");
    const int64_t n = ctx->net.n_nodes;
    // new origin of the FP32 hi/lo split; the extent limit of set_network holds
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < 3; ++c) {
            const double v = xyz[3 * i + c];
            if (!isfinite(v)) return arg_error("non-finite node position");
            lo[c] = fmin(lo[c], v);
            hi[c] = fmax(hi[c], v);
        }
    for (int c = 0; c < 3; ++c) {
        if ((hi[c] - lo[c]) / ctx->mat.b > 1.0e6) return arg_error("network extent exceeds 1e6 Burgers vectors");
        ctx->net.origin[c] = rint(ldexp(0.5 * (lo[c] + hi[c]), -ctx->len_exp));
    }
    PTADD_CUDA(cudaMemcpyAsync(ctx->net.staging, xyz, 3 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    aos_to_soa_scaled<<<(unsigned)((3 * n + 255) / 256), 256, 0, ctx->stream>>>(n, ctx->net.staging, 1.0 / ctx->len_unit,
                                                                                ctx->net.pos[ctx->net.cur]);
    PTADD_CUDA(cudaGetLastError());
    ctx->kernel_launches += 1;
    // the caller may reuse xyz on return
    PTADD_CUDA(cudaStreamSynchronize(ctx->stream));
    return PTADD_OK;
}

ptadd_status ptadd_profile_reset(ptadd_ctx* ctx, int timing)
{
    CHECK_CTX(ctx);
    PTADD_CUDA(cudaStreamSynchronize(ctx->stream));
    ptadd_status st = drain_events(ctx);
    if (st != PTADD_OK) return st;
    ctx->timing = timing != 0;
    ctx->kernel_launches = ctx->pair_launches = ctx->pair_evals = 0;
    ctx->pair_ms = 0.0;
    ctx->near_base = 0;
    if (ctx->have_net)
        PTADD_CUDA(cudaMemcpy(&ctx->near_base, ctx->net.near_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    return PTADD_OK;
}

ptadd_status ptadd_profile_read(ptadd_ctx* ctx, ptadd_profile* out)
{
    CHECK_CTX(ctx);
    if (!out) return arg_error("out is NULL");
    PTADD_CUDA(cudaStreamSynchronize(ctx->stream));
    ptadd_status st = drain_events(ctx);
    if (st != PTADD_OK) return st;
    out->kernel_launches = ctx->kernel_launches;
    out->pair_launches = ctx->pair_launches;
    out->pair_evals = ctx->pair_evals;
    out->pair_ms = ctx->pair_ms;
    out->near_point_pairs = 0;
    if (ctx->have_net) {
        unsigned long long nc = 0;
        PTADD_CUDA(cudaMemcpy(&nc, ctx->net.near_count, sizeof(nc), cudaMemcpyDeviceToHost));
        out->near_point_pairs = (int64_t)(nc - ctx->near_base);
    }
    return PTADD_OK;
}

ptadd_status ptadd_get_forces(ptadd_ctx* ctx, double* F)
{
    CHECK_CTX(ctx);
    if (!ctx->have_net) {
        set_error("no network loaded");
        return PTADD_ERR_STATE;
    }
    if (!F) return arg_error("F is NULL");
    ptadd_status st = eval_forces(ctx, ctx->net.tgt_all, ctx->net.n_nodes);
    if (st != PTADD_OK) return st;
    return read_soa(ctx, ctx->net.force, ctx->mat.mu * ctx->len_unit * ctx->len_unit, F);
}

ptadd_status ptadd_get_forces_dev(ptadd_ctx* ctx, double* F_dev)
{
    CHECK_CTX(ctx);
    if (!ctx->have_net) {
        set_error("no network loaded");
        return PTADD_ERR_STATE;
    }
    if (!F_dev) return arg_error("F_dev is NULL");
    ptadd_status st = eval_forces(ctx, ctx->net.tgt_all, ctx->net.n_nodes);
    if (st != PTADD_OK) return st;
    const int64_t n = ctx->net.n_nodes;
    soa_to_aos_scaled<<<(unsigned)((3 * n + 255) / 256), 256, 0, ctx->stream>>>(
        n, ctx->net.force, ctx->mat.mu * ctx->len_unit * ctx->len_unit, F_dev);
    PTADD_CUDA(cudaGetLastError());
    ctx->kernel_launches += 1;
    return PTADD_OK;
}

// state blob: magic, n_nodes, then 3n doubles (internal units, SoA); with
// junctions on, a second magic and the junction state follow
static const uint64_t STATE_MAGIC = 0x5054414444535431ull;  // "PTADDST1"
static const uint64_t JUNC_MAGIC = 0x5054414444534A31ull;   // "PTADDSJ1"

ptadd_status ptadd_get_state(ptadd_ctx* ctx, void* buf, size_t* bytes)
{
    CHECK_CTX(ctx);
    if (!ctx->have_net) {
        set_error("no network loaded");
        return PTADD_ERR_STATE;
    }
    if (!bytes) return arg_error("bytes is NULL");
    const int64_t n = ctx->net.n_nodes;
    const size_t base = 2 * sizeof(uint64_t) + 3 * n * sizeof(double);
    const size_t need = base + (ctx->junc ? sizeof(uint64_t) + junction_state_bytes(ctx) : 0);
    if (!buf) {
        *bytes = need;
        return PTADD_OK;
    }
    if (*bytes < need) return arg_error("state buffer too small");
    uint64_t hdr[2] = {STATE_MAGIC, (uint64_t)n};
    memcpy(buf, hdr, sizeof(hdr));
    PTADD_CUDA(cudaMemcpyAsync((char*)buf + sizeof(hdr), ctx->net.pos[ctx->net.cur], 3 * n * sizeof(double),
                               cudaMemcpyDeviceToHost, ctx->stream));
    PTADD_CUDA(cudaStreamSynchronize(ctx->stream));
    if (ctx->junc) {
        memcpy((char*)buf + base, &JUNC_MAGIC, sizeof(uint64_t));
        ptadd_status st = junction_state_get(ctx, (char*)buf + base + sizeof(uint64_t));
        if (st != PTADD_OK) return st;
    }
    *bytes = need;
    return PTADD_OK;
}

ptadd_status ptadd_set_state(ptadd_ctx* ctx, const void* buf, size_t bytes)
{
    CHECK_CTX(ctx);
    if (!ctx->have_net) {
        set_error("no network loaded");
        return PTADD_ERR_STATE;
    }
    if (!buf) return arg_error("buf is NULL");
    const int64_t n = ctx->net.n_nodes;
    const size_t base = 2 * sizeof(uint64_t) + 3 * n * sizeof(double);
    const size_t need = base + (ctx->junc ? sizeof(uint64_t) + junction_state_bytes(ctx) : 0);
    uint64_t hdr[2];
    if (bytes != need)
        return arg_error("state size does not match the loaded network (or junctions are on in one and off in the other)");
    memcpy(hdr, buf, sizeof(hdr));
    if (hdr[0] != STATE_MAGIC || hdr[1] != (uint64_t)n) return arg_error("state blob does not match the network");
    if (ctx->junc) {
        uint64_t jm;
        memcpy(&jm, (const char*)buf + base, sizeof(jm));
        if (jm != JUNC_MAGIC) return arg_error("state blob holds no junction state");
    }
    PTADD_CUDA(cudaMemcpyAsync(ctx->net.pos[ctx->net.cur], (const char*)buf + sizeof(hdr), 3 * n * sizeof(double),
                               cudaMemcpyHostToDevice, ctx->stream));
    PTADD_CUDA(cudaStreamSynchronize(ctx->stream));
    if (ctx->junc) return junction_state_set(ctx, (const char*)buf + base + sizeof(uint64_t));
    return PTADD_OK;
}

ptadd_status ptadd_fma_peak(int device, int fp64, double seconds, double* flops)
{
    if (!flops) return arg_error("flops is NULL");
    if (fp64 < 0 || fp64 > 2) return arg_error("mode must be 0 (FP32), 1 (FP64) or 2 (packed FP32 pairs)");
    int ndev = 0;
    PTADD_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return arg_error("device index out of range");
    PTADD_CUDA(cudaSetDevice(device));
    int sms = 0;
    PTADD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    double* sink = nullptr;
    if (dalloc(&sink, 1) != PTADD_OK) return PTADD_ERR_NOMEM;
    cudaStream_t s;
    PTADD_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int threads = 256, blocks = sms * 8;
    const int chains = 8;
    long iters = fp64 == 1 ? 2000 : 20000;
    double best = 0.0;
    ptadd_status st = PTADD_OK;
    for (int pass = 0; pass < 16 && st == PTADD_OK; ++pass) {
        cudaEventRecord(e0, s);
        cudaError_t e = launch_fma_chains(fp64, blocks, threads, iters, sink, s);
        cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            set_error("fma peak kernel failed: %s", cudaGetErrorString(e));
            st = PTADD_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double f = 2.0 * chains * (fp64 == 2 ? 2.0 : 1.0) * (double)iters * blocks * threads / (ms * 1e-3);
        if (pass >= 2 && f > best) best = f;
        if (pass >= 3 && ms * 1e-3 >= seconds / 2) break;
        // grow the run towards the requested duration
        if (ms * 1e-3 < seconds / 2 && iters < (1L << 30)) iters *= 2;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    cudaFree(sink);
    *flops = best;
    return st;
}

}  // extern "C"
