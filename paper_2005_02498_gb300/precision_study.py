"""Error against throughput of the two GPU precisions on the large network.

    python -m paper_2005_02498_gb300.precision_study --steps 50

For each time step in --dts (default: the workload's 1e-11 s and the stable
5e-13 s) three bursts start from the same 32 768-segment network: plain
FP64, mixed (FP32 far field, FP64 near field and integration), and FP64 from
positions moved by one ulp.  The last one measures how far the trajectory
itself amplifies rounding: at 1e-11 s explicit Euler is unstable for the
smaller loops, so two FP64 runs differing by one ulp already disagree, and
the mixed path can only be measured against that floor.  Reported per dt:
the relative (Frobenius) difference of the averaged Lp and the relative
max-norm difference of the final displacements, mixed vs FP64 and perturbed
FP64 vs FP64, and the pair evaluations per second of each precision
(CUDA events inside the library).  The oracle comparison of the forces lives
in the GPU tests.  Prints one JSON line.
"""

from __future__ import annotations

import argparse
import json

import numpy as np

from . import ptadd
from . import workloads as W


def _burst(mat, net, prec, steps, dt, device):
    with ptadd.Context(mat, prec, device) as c:
        c.set_network(net)
        c.profile_reset(True)
        Lp, rho = c.advance(steps, dt)
        prof = c.profile_read()
        x = c.get_nodes()
    return Lp, rho, x, prof["pair_evals"] / (prof["pair_ms"] * 1e-3)


def _relfro(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _reldisp(x, y, x0):
    return float(np.max(np.abs(x - y)) / np.max(np.abs(y - x0)))


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--dts", type=float, nargs="+", default=[W.LARGE_LOOPS["dt"], 5e-13])
    p.add_argument("--device", type=int, default=0)
    a = p.parse_args(argv)

    mat = W.Material().as_tuple()
    net = W.large_loop_network()
    pert = net.copy()
    pert.xyz = np.nextafter(net.xyz, np.inf)
    out = {"workload": "large loop network, 32768 segments", "steps": a.steps, "runs": []}
    for dt in a.dts:
        L64, r64, x64, v64 = _burst(mat, net, ptadd.PTADD_FP64, a.steps, dt, a.device)
        Lmx, rmx, xmx, vmx = _burst(mat, net, ptadd.PTADD_MIXED, a.steps, dt, a.device)
        Lpt, _, xpt, _ = _burst(mat, pert, ptadd.PTADD_FP64, a.steps, dt, a.device)
        out["runs"].append({
            "dt": dt,
            "mixed_vs_fp64": {"Lp_rel": _relfro(Lmx, L64), "rho_rel": abs(rmx / r64 - 1),
                              "disp_rel": _reldisp(xmx, x64, net.xyz)},
            "one_ulp_fp64_vs_fp64": {"Lp_rel": _relfro(Lpt, L64), "disp_rel": _reldisp(xpt, x64, net.xyz)},
            "pair_evals_per_s": {"fp64": v64, "mixed": vmx, "ratio": vmx / v64},
        })
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
