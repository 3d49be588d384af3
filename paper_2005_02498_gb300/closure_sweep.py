"""Closure sweep along a mesoscale load path: surrogate inside its trust
region, batched DD ensembles outside it.

    python -m paper_2005_02498_gb300.closure_sweep --state surrogate.bin

Material points: a grid^3 lattice in the unit cube.  Load: sigma(x, k) =
(k / K) S(x), k = 1..K, where every component of S is a seeded sum of four
random low-wavenumber Fourier modes scaled to a maximum of 200 MPa (a
prescribed smooth field; no finite-element feedback).  Densities: total
mobile and sessile line densities per point from smooth fields,
log-uniformly distributed between 2e12 and 2e13 1/m^2 over the grid, split
over the 12 slip systems by Dirichlet-type shares (normalised exponential
scores of smooth fields), the marginals of the surrogate's training inputs.
Each point needs one closure per load step.  Points inside the surrogate's
trust region take the surrogate's answer (averaged over the 48 symmetric
images of the point, `surrogate.closure_symmetries`, unless --no-symmetrise); the others fall back to the mean
of `--members` DD realisations of `--loops` loops (4096 segments by default;
batched, one launch sequence per load step).
A random sample of (point, step) pairs is re-evaluated with
`--check-members`-realisation DD ensembles to measure the sweep's error.
`--eval-steps` runs an evenly spaced subset of the load steps and
extrapolates the time to all of them.  Prints one JSON line.
"""

from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import ptadd
from . import workloads as W
from .surrogate import closure_symmetries, generate, symmetrised_answers, symmetrised_inputs


def smooth_field(rng, pts, n_modes=4, kmax=2):
    """Sum of n_modes cos(2 pi k.x + phi) with integer wave vectors |k_i| <= kmax."""
    val = np.zeros(pts.shape[0])
    for _ in range(n_modes):
        k = rng.integers(-kmax, kmax + 1, size=3)
        while not k.any():
            k = rng.integers(-kmax, kmax + 1, size=3)
        val += rng.normal() * np.cos(2 * np.pi * pts @ k + rng.uniform(0, 2 * np.pi))
    return val


def _uniform_scores(f):
    """Smooth field -> values whose distribution over the grid is uniform on (0, 1) (ranks)."""
    r = np.argsort(np.argsort(f))
    return (r + 0.5) / f.size


def material_points(seed, grid, stress_max=200e6, rho_min=2e12, rho_max=2e13):
    """Smooth random fields with the marginals of the training inputs: total
    densities log-uniform in [rho_min, rho_max], per-system shares of
    Dirichlet(1) type (normalised exponential scores of smooth fields)."""
    rng = np.random.default_rng(seed)
    g = (np.arange(grid) + 0.5) / grid
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    S = np.stack([smooth_field(rng, pts) for _ in range(6)], 1)
    S *= stress_max / np.max(np.abs(S), axis=0, keepdims=True)
    rho = np.zeros((pts.shape[0], 24))
    for col in (0, 12):
        u = _uniform_scores(smooth_field(rng, pts))
        tot = 10 ** (np.log10(rho_min) + u * (np.log10(rho_max) - np.log10(rho_min)))
        e = np.stack([-np.log1p(-_uniform_scores(smooth_field(rng, pts))) for _ in range(12)], 1)
        rho[:, col:col + 12] = e / e.sum(1, keepdims=True) * tot[:, None]
    return pts, S, rho


def sweep(ctx, S, rho, K, ks_run, members, steps, dt, loops, seed, symmetrise=True, device=0,
          max_fallback_s=600.0):
    """Answer every material point at the load steps ks_run (of K): the
    surrogate (on the device, averaged over the 48 symmetric images with
    `symmetrise`) inside its trust region, the mean of `members` batched DD
    realisations outside it.  Returns dict(answers [K, n, 6], used_dd [K, n],
    surrogate_s, fallback_s, fallback_closures, wall_s)."""
    import torch

    n = S.shape[0]
    answers = np.zeros((K, n, 6))
    used_dd = np.zeros((K, n), bool)
    t_sur = t_dd = 0.0
    dd_closures = 0
    st = torch.cuda.Stream(device=device)
    ctx.set_stream(st.cuda_stream)
    G = len(closure_symmetries()) if symmetrise else 1
    feat_d = torch.empty((G * n, 30), dtype=torch.float64, device="cuda:%d" % device)
    lp_d = torch.empty((G * n, 6), dtype=torch.float64, device=feat_d.device)
    reg_d = torch.empty(G * n, dtype=torch.uint8, device=feat_d.device)
    t_all = time.perf_counter()
    for k in ks_run:
        feats = np.hstack([S * (k / K), rho])
        t0 = time.perf_counter()
        xs = symmetrised_inputs(feats) if G > 1 else feats
        feat_d.copy_(torch.from_numpy(xs))
        ctx.surrogate_predict_dev(G * n, feat_d.data_ptr(), lp_d.data_ptr(), reg_d.data_ptr())
        st.synchronize()
        ys = lp_d.cpu().numpy()
        if G > 1:
            lp, g0 = symmetrised_answers(ys, n)
            inr = reg_d[g0 * n:(g0 + 1) * n].cpu().numpy().astype(bool)
        else:
            lp = ys
            inr = reg_d.cpu().numpy().astype(bool)
        t_sur += time.perf_counter() - t0
        miss = np.flatnonzero(~inr)
        if miss.size and dd_closures and t_dd / dd_closures * (dd_closures + miss.size) > max_fallback_s:
            raise SystemExit("fallback work would exceed max_fallback_s; %d misses at load step %d" % (miss.size, k))
        if miss.size:
            t0 = time.perf_counter()
            ctx.set_stream(None)
            y, _, _ = generate(ctx, feats[miss], members, seed + 100 + k, steps, dt, loops)
            ctx.set_stream(st.cuda_stream)
            lp[miss] = y
            t_dd += time.perf_counter() - t0
            dd_closures += miss.size
        answers[k - 1] = lp
        used_dd[k - 1] = ~inr
    wall = time.perf_counter() - t_all
    ctx.set_stream(None)
    return {"answers": answers, "used_dd": used_dd, "surrogate_s": t_sur, "fallback_s": t_dd,
            "fallback_closures": dd_closures, "wall_s": wall}


def load_steps_run(K, eval_steps):
    """The load steps a run evaluates: all K, or eval_steps evenly spaced ones."""
    if eval_steps and eval_steps < K:
        return sorted(set(int(round(x)) for x in np.linspace(1, K, eval_steps)))
    return list(range(1, K + 1))


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--state", required=True, help="fitted surrogate state (surrogate.py --save)")
    p.add_argument("--grid", type=int, default=16)
    p.add_argument("--load-steps", type=int, default=100)
    p.add_argument("--members", type=int, default=64)
    p.add_argument("--check", type=int, default=256)
    p.add_argument("--check-members", type=int, default=16)
    p.add_argument("--loops", type=int, default=128)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--dt", type=float, default=5e-13)
    p.add_argument("--seed", type=int, default=1005)
    p.add_argument("--eval-steps", type=int, default=0,
                   help="run only this many evenly spaced load steps and extrapolate (0 = all)")
    p.add_argument("--max-fallback-s", type=float, default=600.0,
                   help="stop before the fallback DD work of a run is estimated to exceed this")
    p.add_argument("--no-symmetrise", dest="symmetrise", action="store_false",
                   help="answer with the plain surrogate instead of its average over the 48 symmetric images")
    p.add_argument("--device", type=int, default=0)
    a = p.parse_args(argv)

    pts, S, rho = material_points(a.seed, a.grid)
    n = pts.shape[0]
    K = a.load_steps
    rng = np.random.default_rng(a.seed + 1)
    mat = W.Material().as_tuple()
    ks_run = load_steps_run(K, a.eval_steps)
    with ptadd.Context(mat, ptadd.PTADD_MIXED, a.device) as ctx:
        ctx.surrogate_set_state(open(a.state, "rb").read())
        r = sweep(ctx, S, rho, K, ks_run, a.members, a.steps, a.dt, a.loops, a.seed, a.symmetrise, a.device,
                  a.max_fallback_s)
        answers, used_dd, t_sur, t_dd, dd_closures = (r["answers"], r["used_dd"], r["surrogate_s"],
                                                      r["fallback_s"], r["fallback_closures"])
        total = r["wall_s"] * K / len(ks_run)
        # all-DD reference on a random sample of (step, point) pairs of the run steps
        kr = np.asarray(ks_run) - 1
        pick = rng.choice(len(kr) * n, size=min(a.check, len(kr) * n), replace=False)
        ks, ps = kr[pick // n], pick % n
        feats = np.hstack([S[ps] * ((ks + 1) / K)[:, None], rho[ps]])
        t0 = time.perf_counter()
        ref, _, _ = generate(ctx, feats, a.check_members, a.seed + 7, a.steps, a.dt, a.loops)
        t_ref = time.perf_counter() - t0
    got = answers[ks, ps]
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    sur = ~used_dd[ks, ps]
    run = np.asarray(ks_run) - 1
    out = {
        "points": n, "load_steps": K, "closures": n * K, "load_steps_run": len(ks_run),
        "total_s_extrapolated": total, "closures_per_s": n * K / total,
        "surrogate_s": t_sur, "fallback_dd_s": t_dd,
        "fallback_fraction": float(used_dd[run].mean()), "fallback_closures": int(dd_closures),
        "fallback_members": a.members, "burst_steps": a.steps, "dt": a.dt, "symmetrised": bool(a.symmetrise),
        "check": {"pairs": int(pick.size), "members": a.check_members,
                  "rel_err_vs_all_dd": err,
                  "rel_err_surrogate_answers": float(np.linalg.norm(got[sur] - ref[sur]) / np.linalg.norm(ref[sur]))
                  if sur.any() else None,
                  "dd_realisations_per_s": pick.size * a.check_members / t_ref},
    }
    # an all-DD sweep answers every (point, step) with the fallback's ensemble
    out["all_dd_closures_per_s"] = out["check"]["dd_realisations_per_s"] / a.members
    out["all_dd_estimate_s"] = n * K / out["all_dd_closures_per_s"]
    out["speedup_vs_all_dd"] = out["all_dd_estimate_s"] / total
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
