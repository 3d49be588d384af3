"""Junctions and thermally activated breaking (Sec. 2.2) over a long run:
the time-averaged plastic distortion rate with and without them, and what
the junction kernels cost per DD step.

    python -m paper_2005_02498_gb300.run_junctions --loops 40 --chunks 60

The microstructure follows the paper's recipe (Sec. 3.2.1): mobile density
shared by Schmid factor, a much larger sessile density of pinned loops.  A
plain run (no junctions) and a run with junctions start from the same
network; the latter runs `chunks` bursts of `steps` DD steps, its
junction state carried from burst to burst.  Without junctions the loops
keep moving and |R^Lp| stays near the free-flight value; with them, the
network ends up held at junctions, the DD clock jumps to the next break, and
the average over DD time falls by orders of magnitude (the paper quotes
about 1e-2 1/s for its MoDELib boxes).
"""

from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import ptadd
from . import workloads as W


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--loops", type=int, default=40)
    ap.add_argument("--sigma", type=float, default=100e6, help="uniaxial [001] stress, Pa")
    ap.add_argument("--rho-m", type=float, default=1e13)
    ap.add_argument("--rho-s", type=float, default=2e14)
    ap.add_argument("--steps", type=int, default=2000, help="DD steps per burst")
    ap.add_argument("--chunks", type=int, default=60, help="bursts with junctions")
    ap.add_argument("--plain-chunks", type=int, default=10, help="bursts without junctions")
    ap.add_argument("--dt", type=float, default=5e-13)
    ap.add_argument("--capture", type=float, default=10e-9, help="capture radius, m")
    ap.add_argument("--a", type=float, default=1e-3, help="maximum break time, s")
    ap.add_argument("--stuck-b", type=float, default=1e-2, help="stuck displacement per step, in b")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--seed", type=int, default=21)
    ap.add_argument("--device", type=int, default=0)
    ap.add_argument("--progress", action="store_true", help="also print one JSON line per burst")
    a = ap.parse_args(argv)
    mat = W.Material()
    net = W.junction_microstructure(a.seed, W.uniaxial_stress(a.sigma), a.rho_m, a.rho_s, n_loops=a.loops)
    mobile = int((net.pinned.reshape(a.loops, -1)[:, 0] == 0).sum())
    prec = ptadd.PTADD_FP64 if a.precision == "fp64" else ptadd.PTADD_MIXED
    out = {"workload": "%d loops of 32 nodes (%d mobile), rho_m %.1e, rho_s %.1e 1/m^2, %.0f MPa [001], dt %.1e s"
                       % (a.loops, mobile, a.rho_m, a.rho_s, a.sigma / 1e6, a.dt),
           "precision": a.precision, "capture_m": a.capture, "a_s": a.a, "stuck_b": a.stuck_b}
    with ptadd.Context(mat.as_tuple(), prec, a.device) as ctx:
        ctx.set_network(net)
        ctx.advance(10, a.dt)  # warm-up
        ctx.set_network(net)
        s_lp, s_t, t0 = np.zeros((3, 3)), 0.0, time.perf_counter()
        for _ in range(a.plain_chunks):
            lp, _ = ctx.advance(a.steps, a.dt)
            s_lp += lp * a.steps * a.dt
            s_t += a.steps * a.dt
        plain_wall = time.perf_counter() - t0
        out["plain"] = {"steps": a.plain_chunks * a.steps, "dd_time_s": s_t,
                        "Lp_norm": float(np.linalg.norm(s_lp / s_t)),
                        "us_per_step": 1e6 * plain_wall / (a.plain_chunks * a.steps)}
        if a.progress:
            print(json.dumps({"plain": out["plain"]}), flush=True)
        ctx.set_network(net)
        ctx.set_junctions(a.capture, a.a, a.stuck_b * mat.b, a.seed)
        s_lp, s_t, recs, t0 = np.zeros((3, 3)), 0.0, [], time.perf_counter()
        prev_clock = 0.0
        for _ in range(a.chunks):
            lp, _ = ctx.advance(a.steps, a.dt)
            j = ctx.junctions()
            dur = j["clock"] - prev_clock  # the burst's steps plus its jumps
            prev_clock = j["clock"]
            s_lp += lp * dur
            s_t += dur
            recs.append({"Lp_norm": float(np.linalg.norm(lp)), "dd_time_s": dur, "held": j["held"],
                         "formed": j["formed"], "broken": j["broken"], "jumps": j["jumps"],
                         "wall_s": time.perf_counter() - t0})
            if a.progress:
                print(json.dumps({"burst": len(recs), **recs[-1]}), flush=True)
        wall = time.perf_counter() - t0
        j = ctx.junctions()
        out["junctions"] = {"steps": a.chunks * a.steps, "dd_time_s": s_t, "jumped_s": j["jumped"],
                            "Lp_norm": float(np.linalg.norm(s_lp / s_t)), "formed": j["formed"],
                            "broken": j["broken"], "jumps": j["jumps"], "held": j["held"],
                            "us_per_step": 1e6 * wall / (a.chunks * a.steps), "bursts": recs}
    out["junction_overhead_per_step"] = out["junctions"]["us_per_step"] / out["plain"]["us_per_step"] - 1.0
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
