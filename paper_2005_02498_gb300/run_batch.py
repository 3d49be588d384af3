"""Run a batched ensemble of independent realisations through the C ABI.

    python -m paper_2005_02498_gb300.run_batch --R 256 --steps 20 --precision mixed --autotune

Workload (seeded): R realisations, N_r ~ U{n_min..n_max} segments in loops of
32, every stress component ~ U(-200, 200) MPa, sessile (pinned) loop
fraction ~ U(0.1, 0.9), loop density 16 per um^3, dt = 1e-11 s.  One PTA
closure is one realisation's burst of --burst-steps (2000) steps; the
closures/s figure extrapolates the measured time per step to that burst.
Optionally times plain FP64 on the first --fp64-R realisations and reports
its closures/s extrapolated per segment pair to the whole batch.  With
--junction-radius the burst runs with junctions (ptadd_batch_set_junctions:
maximum break time --junction-a, stuck displacement --junction-stuck, every
realisation on its own clock) and reports their counts and the clocks.
Prints one JSON line.
"""

from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import ptadd
from . import workloads as W


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--R", type=int, default=256)
    p.add_argument("--n-min", type=int, default=1024)
    p.add_argument("--n-max", type=int, default=16384)
    p.add_argument("--seed", type=int, default=1003)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--burst-steps", type=int, default=2000)
    p.add_argument("--dt", type=float, default=1e-11)
    p.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    p.add_argument("--autotune", action="store_true")
    p.add_argument("--fp64-R", type=int, default=0)
    p.add_argument("--fp64-steps", type=int, default=2)
    p.add_argument("--device", type=int, default=0)
    p.add_argument("--junction-radius", type=float, default=0.0, help="m; 0: junctions off")
    p.add_argument("--junction-a", type=float, default=1e-3)
    p.add_argument("--junction-stuck", type=float, default=2.556e-12)
    a = p.parse_args(argv)

    t0 = time.perf_counter()
    batch = W.batch_ensemble(a.seed, R=a.R, n_min=a.n_min, n_max=a.n_max)
    t_gen = time.perf_counter() - t0
    prec = ptadd.PTADD_FP64 if a.precision == "fp64" else ptadd.PTADD_MIXED
    out = {"R": a.R, "segments": int(batch.xyz.shape[0]), "precision": a.precision, "seed": a.seed,
           "generate_s": t_gen}
    with ptadd.Context(W.Material().as_tuple(), prec, a.device) as ctx:
        t0 = time.perf_counter()
        ctx.batch_set(batch)
        out["set_s"] = time.perf_counter() - t0
        if a.autotune:
            t0 = time.perf_counter()
            ctx.batch_autotune()
            out["autotune_s"] = time.perf_counter() - t0
        info = ctx.batch_info()
        out.update({k: info[k] for k in ("pairs_per_step", "work_items", "tile_targets", "chunk_sources", "tuned")})
        if a.junction_radius > 0:
            ctx.batch_set_junctions(a.junction_radius, a.junction_a, a.junction_stuck, a.seed)
        ctx.batch_advance(2, a.dt)  # warm-up (captures the step graph)
        ctx.batch_set_nodes(batch.xyz)
        if a.junction_radius > 0:  # clear the warm-up's junctions and clocks
            ctx.batch_set_junctions(a.junction_radius, a.junction_a, a.junction_stuck, a.seed)
            ctx.batch_advance(2, a.dt)  # (the graph is captured again)
            ctx.batch_set_nodes(batch.xyz)
            ctx.batch_set_junctions(a.junction_radius, a.junction_a, a.junction_stuck, a.seed)
        t0 = time.perf_counter()
        Lp, rho = ctx.batch_advance(a.steps, a.dt)
        el = time.perf_counter() - t0
        ms_step = 1e3 * el / a.steps
        if a.junction_radius > 0:
            per, _ = ctx.batch_junctions()
            out["junctions"] = {"radius_m": a.junction_radius, "a_s": a.junction_a, "stuck_m": a.junction_stuck,
                                "formed": int(sum(q["formed"] for q in per)),
                                "held": int(sum(q["held"] for q in per)),
                                "broken": int(sum(q["broken"] for q in per)),
                                "jumps": int(sum(q["jumps"] for q in per)),
                                "realisations_with_junctions": int(sum(q["formed"] > 0 for q in per)),
                                "clock_median_s": float(np.median([q["clock"] for q in per]))}
        out.update({"steps": a.steps, "ms_per_step": ms_step,
                    "pair_evals_per_s": info["pairs_per_step"] * a.steps / el,
                    "closures_per_s": a.R / (ms_step * 1e-3 * a.burst_steps),
                    "burst_steps": a.burst_steps,
                    "Lp_norm_median": float(np.median(np.linalg.norm(Lp.reshape(a.R, -1), axis=1))),
                    "finite": bool(np.all(np.isfinite(Lp)))})
    if a.fp64_R > 0:
        sub = W.batch_from_networks([batch.realisation(r) for r in range(a.fp64_R)])
        with ptadd.Context(W.Material().as_tuple(), ptadd.PTADD_FP64, a.device) as ctx:
            ctx.batch_set(sub)
            pairs_sub = ctx.batch_info()["pairs_per_step"]
            ctx.batch_advance(1, a.dt)
            ctx.batch_set_nodes(sub.xyz)
            t0 = time.perf_counter()
            ctx.batch_advance(a.fp64_steps, a.dt)
            el = time.perf_counter() - t0
        rate = pairs_sub * a.fp64_steps / el
        out["fp64_subsample"] = {"R": a.fp64_R, "steps": a.fp64_steps, "pair_evals_per_s": rate,
                                 "closures_per_s_extrapolated":
                                     a.R / (out["pairs_per_step"] / rate * a.burst_steps)}
        out["speedup_vs_fp64"] = out["pair_evals_per_s"] / rate
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
