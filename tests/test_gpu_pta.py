"""GPU parity of the Practical Time Averaging driver (pta.py, Sec. 3.1) with
the oracle's independent implementation of the same loop, FP64 bursts on the
512-segment network.

The later slow steps start from states reached after one to two hundred DD
steps, past the close approach of two loops on this network, where the
trajectory amplifies rounding differences strongly: the oracle started from
positions moved by one ulp differs from itself by ~1e-3 in the second slow
step.  So each record is held to max(1e-8, 10 x that one-ulp floor),
computed here, and the decisions (chunks per average, extensions, jumps)
must agree while the preceding records' floor is below 1e-6.  A first slow
step without jumps starts from the initial network (floor ~1e-10) and is
held to 1e-8; with jumps it starts after them, past the close approach.
"""

import dataclasses

import numpy as np
import pytest

from oracle import pta as OP
from paper_2005_02498_gb300 import ptadd
from paper_2005_02498_gb300 import pta
from paper_2005_02498_gb300 import workloads as W

pytestmark = pytest.mark.gpu
MAT = W.Material().as_tuple()


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("lpdot_max,steps", [(1e30, 3), (0.0, 1)])
def test_pta_driver_matches_oracle(lpdot_max, steps):
    p = pta.PTAParams(chunk=10, max_chunks=4, extend_chunks=3, lpdot_max=lpdot_max, max_jumps=2)
    q = dataclasses.replace(p)  # the oracle reads the same attributes
    net = W.small_loop_network()
    pert = net.copy()
    pert.xyz = np.nextafter(net.xyz, np.inf)
    with ptadd.Context(MAT, ptadd.PTADD_FP64, 0) as c:
        got = pta.run(c, net, p, steps)
    ref = OP.run(MAT, net, q, steps)
    ref_p = OP.run(MAT, pert, q, steps)
    assert len(got) == len(ref) == steps
    worst = 0.0  # largest one-ulp floor of the records so far
    for k, (g, r, rp) in enumerate(zip(got, ref, ref_p)):
        if worst < 1e-6:
            assert (g["jumps"], g["chunks"], g["extended"]) == (r["jumps"], r["chunks"], r["extended"]), k
        floor = max(_rel(rp[key], r[key]) for key in ("Lp", "Lp_prev"))
        tol = max(1e-8, 10 * floor)
        if k == 0 and r["jumps"] == 0:  # starts from the initial network: well conditioned
            assert floor < 1e-9
        for key in ("Lp", "Lp_prev"):
            assert _rel(g[key], r[key]) <= tol, (k, key, _rel(g[key], r[key]), floor)
        assert abs(g["t"] - r["t"]) <= tol * max(r["t"], 1e-12)
        worst = max(worst, floor)
