// closure.cu -- the closure sweep of a coupled load path (the PTA closure of
// Sec. 3 asked for at many material points): surrogate answers inside its
// trust region, batched DD ensembles outside it; and the realisation
// generator those ensembles are drawn from.
//
// A DD closure at (sigma, rho_mobile[12], rho_sessile[12]) is the mean of
// sym(R^Lp) (Eq. 2.5, Voigt order) over `ens` realisations of circular glide
// loops of 32 nodes whose mobile and sessile line densities per FCC slip
// system follow the 24 densities:
//   - class counts (24 classes: 12 systems x mobile/sessile) are the floor of
//     n_loops x share plus one loop more for the classes picked by systematic
//     sampling of the fractional parts, so each class is within one loop of
//     its share;
//   - radii are stratified over (r_min, r_max) within each class, line senses
//     balanced (+1/-1) within each class, centres uniform in the cube, phases
//     uniform;
//   - the cube volume is set from the drawn loops' total length, so the total
//     density is exact; sessile loops are pinned.
// Random numbers: xoshiro256** (Blackman and Vigna), its state seeded by
// SplitMix64 (Vigna) from seed ^ (q * 0x9E3779B97F4A7C15) for realisation q,
// so every realisation has its own stream whatever the batching.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ptadd_internal.cuh"

namespace ptadd {
namespace {

constexpr int NPL = 32;                // nodes per loop
constexpr double R_MIN = 0.05e-6, R_MAX = 0.2e-6;
constexpr uint64_t STREAM_STEP = 0x9E3779B97F4A7C15ull;

struct Rng {
    uint64_t s[4];
    explicit Rng(uint64_t seed)
    {
        uint64_t x = seed;
        for (uint64_t& v : s) v = splitmix(x);
    }
    static uint64_t splitmix(uint64_t& x)
    {
        uint64_t z = (x += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
    uint64_t next()
    {
        const uint64_t r = rotl(s[1] * 5, 7) * 9;
        const uint64_t t = s[1] << 17;
        s[2] ^= s[0];
        s[3] ^= s[1];
        s[1] ^= s[2];
        s[0] ^= s[3];
        s[2] ^= t;
        s[3] = rotl(s[3], 45);
        return r;
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }  // [0, 1)
    int below(int k) { return (int)(uniform() * k); }                                  // 0 .. k-1
};

// The 12 FCC {111}<110> systems in the order of the density inputs: planes
// (111), (-111), (1-11), (11-1); in each, the <110> directions in the order
// [01-1], [10-1], [1-10], [011], [101], [110] that lie in the plane.
void fcc_systems(double bh[12][3], double nh[12][3])
{
    const double nrm[4][3] = {{1, 1, 1}, {-1, 1, 1}, {1, -1, 1}, {1, 1, -1}};
    const double cand[6][3] = {{0, 1, -1}, {1, 0, -1}, {1, -1, 0}, {0, 1, 1}, {1, 0, 1}, {1, 1, 0}};
    int k = 0;
    for (int p = 0; p < 4; ++p)
        for (int c = 0; c < 6; ++c)
            if (cand[c][0] * nrm[p][0] + cand[c][1] * nrm[p][1] + cand[c][2] * nrm[p][2] == 0.0) {
                for (int e = 0; e < 3; ++e) {
                    bh[k][e] = cand[c][e] / sqrt(2.0);
                    nh[k][e] = nrm[p][e] / sqrt(3.0);
                }
                ++k;
            }
}

// One realisation appended to the output arrays (node, loop and pin arrays
// grow by n_loops*32, n_loops, n_loops*32).  Returns the volume.
double draw_realisation(uint64_t stream_seed, const double* rho24, int n_loops, double bmag,
                        std::vector<double>& xyz, std::vector<double>& burgers, std::vector<double>& normal,
                        std::vector<uint8_t>& pinned)
{
    Rng rng(stream_seed);
    double bh[12][3], nh[12][3];
    fcc_systems(bh, nh);
    double tot = 0.0;
    for (int c = 0; c < 24; ++c) tot += rho24[c];
    double e[24];
    int counts[24];
    int assigned = 0;
    for (int c = 0; c < 24; ++c) {
        e[c] = n_loops * (tot > 0 ? rho24[c] / tot : 1.0 / 24);
        counts[c] = (int)floor(e[c]);
        assigned += counts[c];
    }
    const int extra = n_loops - assigned;
    if (extra > 0) {  // systematic sampling: positions u, u+1, ... over the cumulative remainders
        const double u = rng.uniform();
        double cum = 0.0;
        int j = 0;
        for (int c = 0; c < 24 && j < extra; ++c) {
            cum += e[c] - counts[c];
            while (j < extra && u + j < cum) {
                ++counts[c];
                ++j;
            }
        }
        counts[23] += extra - j;  // rounding of the cumulative sum
    }
    // per loop: class, radius, sense
    std::vector<int> cls;
    std::vector<double> radius, sense;
    for (int c = 0; c < 24; ++c) {
        const int k = counts[c];
        if (k == 0) continue;
        std::vector<int> perm(k);
        for (int i = 0; i < k; ++i) perm[i] = i;
        for (int i = k - 1; i > 0; --i) std::swap(perm[i], perm[rng.below(i + 1)]);
        std::vector<double> sg(k);
        for (int i = 0; i < k; ++i) sg[i] = i < k / 2 ? 1.0 : -1.0;
        if (k % 2) sg[k - 1] = rng.uniform() < 0.5 ? -1.0 : 1.0;
        for (int i = k - 1; i > 0; --i) std::swap(sg[i], sg[rng.below(i + 1)]);
        for (int i = 0; i < k; ++i) {
            cls.push_back(c);
            radius.push_back(R_MIN + (R_MAX - R_MIN) * (perm[i] + rng.uniform()) / k);
            sense.push_back(sg[i]);
        }
    }
    const double chord = 2.0 * sin(M_PI / NPL) * NPL;
    double rsum = 0.0;
    for (double r : radius) rsum += r;
    const double volume = tot > 0 ? chord * rsum / tot : 1e-18;
    const double edge = cbrt(volume);
    for (size_t l = 0; l < cls.size(); ++l) {
        const int s = cls[l] % 12;
        const double* e1 = bh[s];
        const double* n = nh[s];
        const double e2[3] = {n[1] * e1[2] - n[2] * e1[1], n[2] * e1[0] - n[0] * e1[2], n[0] * e1[1] - n[1] * e1[0]};
        double cen[3];
        for (int d = 0; d < 3; ++d) cen[d] = rng.uniform() * edge;
        const double phi0 = rng.uniform() * 2.0 * M_PI;
        for (int k = 0; k < NPL; ++k) {
            const double phi = phi0 + sense[l] * (2.0 * M_PI / NPL) * k;
            const double cp = cos(phi), sp = sin(phi);
            for (int d = 0; d < 3; ++d) xyz.push_back(cen[d] + radius[l] * (cp * e1[d] + sp * e2[d]));
            pinned.push_back(cls[l] >= 12 ? 1 : 0);
        }
        for (int d = 0; d < 3; ++d) {
            burgers.push_back(bmag * e1[d]);
            normal.push_back(n[d]);
        }
    }
    return volume;
}

ptadd_status carg(const char* m)
{
    set_error("%s", m);
    return PTADD_ERR_ARG;
}

}  // namespace
}  // namespace ptadd

using namespace ptadd;

extern "C" {

ptadd_status ptadd_closure_realisation(const ptadd_material* mat, uint64_t seed, const double* rho24,
                                       int32_t n_loops, double* xyz, double* burgers, double* normal,
                                       uint8_t* pinned, double* volume)
{
    if (!mat || !rho24 || !xyz || !burgers || !normal || !pinned || !volume)
        return carg("ptadd_closure_realisation: null argument");
    if (n_loops < 1) return carg("ptadd_closure_realisation: need n_loops >= 1");
    for (int c = 0; c < 24; ++c)
        if (!(rho24[c] >= 0.0) || !isfinite(rho24[c])) return carg("ptadd_closure_realisation: densities must be finite and >= 0");
    if (!(mat->b > 0.0)) return carg("ptadd_closure_realisation: need b > 0");
    std::vector<double> x, b, n;
    std::vector<uint8_t> p;
    const double v = draw_realisation(seed, rho24, n_loops, mat->b, x, b, n, p);
    memcpy(xyz, x.data(), x.size() * sizeof(double));
    memcpy(burgers, b.data(), b.size() * sizeof(double));
    memcpy(normal, n.data(), n.size() * sizeof(double));
    memcpy(pinned, p.data(), p.size());
    *volume = v;
    return PTADD_OK;
}

ptadd_status ptadd_closure_sweep(ptadd_ctx* ctx, int64_t n_pts, const double* sig6, const double* rho24,
                                 int32_t ens, int64_t segments, int64_t steps, double dt, uint64_t seed,
                                 double* Lp_sym6, uint8_t* used_fallback)
{
    if (!ctx || !sig6 || !rho24 || !Lp_sym6) return carg("ptadd_closure_sweep: null argument");
    if (n_pts < 1 || ens < 1 || steps < 1 || !(dt > 0.0) || !isfinite(dt))
        return carg("ptadd_closure_sweep: need n_pts >= 1, ens >= 1, steps >= 1, dt > 0");
    if (segments < 2 * NPL || segments % NPL)
        return carg("ptadd_closure_sweep: segments must be a multiple of 32, at least 64");
    const int n_loops = (int)(segments / NPL);
    // 1. surrogate answers and trust region for every point
    std::vector<double> feat((size_t)n_pts * 30);
    for (int64_t i = 0; i < n_pts; ++i) {
        memcpy(&feat[i * 30], sig6 + i * 6, 6 * sizeof(double));
        memcpy(&feat[i * 30 + 6], rho24 + i * 24, 24 * sizeof(double));
    }
    std::vector<uint8_t> inr((size_t)n_pts);
    ptadd_status st = ptadd_surrogate_predict(ctx, n_pts, feat.data(), Lp_sym6, inr.data());
    if (st != PTADD_OK) return st;
    std::vector<int64_t> miss;
    for (int64_t i = 0; i < n_pts; ++i) {
        if (used_fallback) used_fallback[i] = inr[i] ? 0 : 1;
        if (!inr[i]) miss.push_back(i);
    }
    if (miss.empty()) return PTADD_OK;
    // 2. the misses: ens realisations each, batched (about 4M segments per batch)
    const int64_t total = (int64_t)miss.size() * ens;
    const int64_t per_batch = std::max<int64_t>(1, (int64_t(1) << 22) / segments);
    std::vector<double> acc(miss.size() * 6, 0.0);
    for (int64_t q0 = 0; q0 < total; q0 += per_batch) {
        const int32_t R = (int32_t)std::min(per_batch, total - q0);
        std::vector<double> xyz, burgers, normal, vol(R), s6((size_t)R * 6);
        std::vector<uint8_t> pinned;
        std::vector<int64_t> node_off(R + 1, 0), loop_off;
        for (int32_t r = 0; r < R; ++r) {
            const int64_t q = q0 + r, pt = miss[q / ens];
            vol[r] = draw_realisation(seed ^ ((uint64_t)q * STREAM_STEP), rho24 + pt * 24, n_loops, ctx->mat.b, xyz,
                                      burgers, normal, pinned);
            memcpy(&s6[(size_t)r * 6], sig6 + pt * 6, 6 * sizeof(double));
            node_off[r + 1] = (int64_t)(xyz.size() / 3);
        }
        const int64_t nl = (int64_t)(burgers.size() / 3);
        loop_off.resize(nl + 1);
        for (int64_t l = 0; l <= nl; ++l) loop_off[l] = l * NPL;
        st = ptadd_batch_set(ctx, R, node_off.data(), nl, loop_off.data(), xyz.data(), burgers.data(), normal.data(),
                             pinned.data(), s6.data(), vol.data());
        if (st != PTADD_OK) return st;
        std::vector<double> Lp((size_t)R * 9);
        st = ptadd_batch_advance(ctx, steps, dt, Lp.data(), nullptr);
        if (st != PTADD_OK) return st;
        for (int32_t r = 0; r < R; ++r) {
            const double* L = &Lp[(size_t)r * 9];
            double* a = &acc[(size_t)((q0 + r) / ens) * 6];
            a[0] += L[0];
            a[1] += L[4];
            a[2] += L[8];
            a[3] += 0.5 * (L[5] + L[7]);
            a[4] += 0.5 * (L[2] + L[6]);
            a[5] += 0.5 * (L[1] + L[3]);
        }
    }
    for (size_t m = 0; m < miss.size(); ++m)
        for (int c = 0; c < 6; ++c) Lp_sym6[miss[m] * 6 + c] = acc[m * 6 + c] / ens;
    return PTADD_OK;
}

ptadd_status ptadd_system_densities(int64_t n_nodes, const double* xyz, int64_t n_loops, const int64_t* loop_off,
                                    const double* burgers, const double* normal, const uint8_t* pinned, double volume,
                                    double* rho24)
{
    if (n_nodes < 0 || n_loops < 1 || !xyz || !loop_off || !burgers || !normal || !rho24 ||
        !(volume > 0.0) || !isfinite(volume))
        return carg("ptadd_system_densities: bad sizes, NULL array or non-positive volume");
    if (loop_off[0] != 0 || loop_off[n_loops] != n_nodes)
        return carg("ptadd_system_densities: loop_off must start at 0 and end at n_nodes");
    double bh[12][3], nh[12][3];
    fcc_systems(bh, nh);
    double acc[24] = {0};
    for (int64_t k = 0; k < n_loops; ++k) {
        const int64_t s = loop_off[k], e = loop_off[k + 1];
        if (e - s < 2) return carg("ptadd_system_densities: every loop needs >= 2 nodes");
        const double* b = burgers + 3 * k;
        const double* nv = normal + 3 * k;
        const double bn = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
        const double nn = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
        int sys = -1;
        for (int i = 0; i < 12 && bn > 0.0 && nn > 0.0; ++i) {
            const double cb = fabs(b[0] * bh[i][0] + b[1] * bh[i][1] + b[2] * bh[i][2]) / bn;
            const double cn = fabs(nv[0] * nh[i][0] + nv[1] * nh[i][1] + nv[2] * nh[i][2]) / nn;
            if (cb > 1.0 - 1e-9 && cn > 1.0 - 1e-9) sys = i;
        }
        if (sys < 0) {
            set_error("ptadd_system_densities: loop %lld is not on an FCC {111}<110> system", (long long)k);
            return PTADD_ERR_ARG;
        }
        for (int64_t a = s; a < e; ++a) {
            const int64_t c = (a + 1 < e) ? a + 1 : s;
            const double dx = xyz[3 * c] - xyz[3 * a], dy = xyz[3 * c + 1] - xyz[3 * a + 1],
                         dz = xyz[3 * c + 2] - xyz[3 * a + 2];
            const double L = sqrt(dx * dx + dy * dy + dz * dz);
            if (!isfinite(L)) return carg("ptadd_system_densities: non-finite node position");
            const bool sessile = pinned && pinned[a] && pinned[c];
            acc[(sessile ? 12 : 0) + sys] += L;
        }
    }
    for (int m = 0; m < 24; ++m) rho24[m] = acc[m] / volume;
    return PTADD_OK;
}

}  // extern "C"
