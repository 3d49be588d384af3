"""Run one DD burst on a named synthetic workload through the C ABI.

    python -m paper_2005_02498_gb300.run_burst --workload large --steps 2 --precision fp64

Prints the averaged Lp (1/s), rho (1/m^2) and the wall time as one JSON line.
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
    p.add_argument("--workload", default="large", choices=["small", "medium", "large"])
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--dt", type=float, default=None)
    p.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    p.add_argument("--device", type=int, default=0)
    a = p.parse_args(argv)
    net = {"small": W.small_loop_network, "medium": W.medium_loop_network,
           "large": W.large_loop_network}[a.workload]()
    dt = a.dt if a.dt else {"small": W.SMALL_LOOPS, "medium": W.MEDIUM_LOOPS, "large": W.LARGE_LOOPS}[a.workload]["dt"]
    prec = ptadd.PTADD_FP64 if a.precision == "fp64" else ptadd.PTADD_MIXED
    with ptadd.Context(W.Material().as_tuple(), prec, a.device) as ctx:
        ctx.set_network(net)
        t0 = time.perf_counter()
        Lp, rho = ctx.advance(a.steps, dt)
        t1 = time.perf_counter()
        info = ctx.info()
    print(json.dumps({"workload": a.workload, "precision": a.precision, "steps": a.steps, "dt": dt,
                      "segments": info["n_nodes"], "seconds": t1 - t0,
                      "pair_evals_per_s": info["pairs_per_step"] * a.steps / (t1 - t0),
                      "Lp_avg": np.asarray(Lp).tolist(), "rho_avg": rho}))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
