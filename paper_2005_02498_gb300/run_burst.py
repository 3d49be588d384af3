"""Run one DD burst on a named synthetic workload through the C ABI.

    python -m paper_2005_02498_gb300.run_burst --workload large --steps 2 --precision fp64
    python -m paper_2005_02498_gb300.run_burst --workload junctions --steps 500 --with-junctions

Workloads: the small, medium and large loop networks, and the junction
microstructure of the paper's recipe (Sec. 3.2.1: 40 loops of 32 nodes,
mobile density 1e13 1/m^2 shared by Schmid factor, sessile 2e14 1/m^2 of
pinned loops, 100 MPa [001], dt 5e-13 s).  --with-junctions turns on
junctions and their thermally activated breaking (Sec. 2.2: capture radius
10 nm, maximum break time 1e-3 s, stuck below 1e-2 b per step).  A warm-up
burst of --warmup steps runs first (from the same start).  Prints the
averaged Lp (1/s), rho (1/m^2), the wall time and the time per DD step as
one JSON line.
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
    p.add_argument("--workload", default="large", choices=["small", "medium", "large", "junctions"])
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--dt", type=float, default=None)
    p.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    p.add_argument("--device", type=int, default=0)
    p.add_argument("--with-junctions", action="store_true")
    p.add_argument("--warmup", type=int, default=0)
    a = p.parse_args(argv)
    mat = W.Material()
    if a.workload == "junctions":
        net = W.junction_microstructure(21, W.uniaxial_stress(100e6), 1e13, 2e14, n_loops=40)
        dt = a.dt if a.dt else 5e-13
    else:
        net = {"small": W.small_loop_network, "medium": W.medium_loop_network,
               "large": W.large_loop_network}[a.workload]()
        dt = a.dt if a.dt else {"small": W.SMALL_LOOPS, "medium": W.MEDIUM_LOOPS,
                                "large": W.LARGE_LOOPS}[a.workload]["dt"]
    prec = ptadd.PTADD_FP64 if a.precision == "fp64" else ptadd.PTADD_MIXED
    out = {"workload": a.workload, "precision": a.precision, "steps": a.steps, "dt": dt,
           "junctions": bool(a.with_junctions)}
    with ptadd.Context(mat.as_tuple(), prec, a.device) as ctx:
        for k in range(2 if a.warmup > 0 else 1):
            ctx.set_network(net)
            if a.with_junctions:
                ctx.set_junctions(10e-9, 1e-3, 1e-2 * mat.b, 21)
            steps = a.warmup if (k == 0 and a.warmup > 0) else a.steps
            t0 = time.perf_counter()
            Lp, rho = ctx.advance(steps, dt)
            t1 = time.perf_counter()
        info = ctx.info()
        if a.with_junctions:
            j = ctx.junctions()
            out["junction_state"] = {kk: j[kk] for kk in ("held", "formed", "broken", "jumps", "clock")}
    out.update({"segments": info["n_nodes"], "seconds": t1 - t0, "us_per_step": 1e6 * (t1 - t0) / max(1, a.steps),
                "pair_evals_per_s": info["pairs_per_step"] * a.steps / (t1 - t0),
                "Lp_avg": np.asarray(Lp).tolist(), "rho_avg": rho})
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
