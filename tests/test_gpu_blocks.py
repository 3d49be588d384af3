"""GPU parity of the block-level coupling driver (blocks.py, Sec. 4.2.1)
with the oracle's increment: three blocks, the 512-segment network in each,
FP64 bursts in one batch, two increments (the first with one block above the
0.5 MPa gap and two inflated, the second all inflated, with the limit rule
holding at one block).

The rates are differences of two running averages a fraction of a percent
apart.  The oracle started from positions moved by one ulp gives the effect
of ONE rounding-sized perturbation at the start (the floor); the GPU and the
oracle round differently at every DD step, and each of those perturbations
grows no more than the one at the start, so each record is held to
max(1e-8, floor x the DD steps run so far), computed here."""

import dataclasses

import numpy as np
import pytest

from oracle import blocks as OB
from paper_2005_02498_gb300 import blocks as B
from paper_2005_02498_gb300 import ptadd
from paper_2005_02498_gb300 import workloads as W

pytestmark = pytest.mark.gpu
MAT = W.Material().as_tuple()


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _oracle(net, xyz0, p, incs):
    xyz = [xyz0.copy() for _ in range(3)]
    state = {"Lp": np.zeros((3, 3, 3)), "Lpdot": np.zeros((3, 3, 3))}
    n = net.copy()
    return [OB.increment(MAT, n, xyz, state, Tk, Tkm1, dtp, p) for Tk, Tkm1, dtp in incs]


def test_block_driver_matches_oracle():
    p = B.BlockParams(chunk=10, max_chunks=3, strain_step=1000.0)  # the limit at block 2 only
    q = dataclasses.replace(p)
    net = W.small_loop_network()
    T0 = np.zeros((3, 6))
    T0[:, 2] = [40e6, 50e6, 60e6]
    T1 = T0 + np.array([[0, 0, 1e6, 0, 0, 0], [0, 0, 2e6, 0, 0, 1e5], [0, 0, 9e6, 0, 0, 0]])
    T2 = T1 + np.array([[0, 0, 2e6, 0, 0, 0], [0, 0, 1e6, 0, 0, 0], [0, 0, 0.5e6, 0, 0, 0]])
    incs = [(T1, T0, 1.0), (T2, T1, 1.0)]
    with ptadd.Context(MAT, ptadd.PTADD_FP64, 0) as c:
        box = B.BlockPTA(c, net, 3, p)
        got = [box.increment(*inc) for inc in incs]
    ref = _oracle(net, net.xyz, q, incs)
    ref_p = _oracle(net, np.nextafter(net.xyz, np.inf), q, incs)
    assert ref[0]["mag"][2] == 1.0 and ref[0]["mag"][0] > 1 and np.all(ref[1]["mag"] > 1)
    assert list(ref[1]["limit"]) == [False, False, True]
    steps = 0
    for k, (g, r, rp) in enumerate(zip(got, ref, ref_p)):
        assert g["chunks"] == r["chunks"], k
        steps += sum(r["chunks"]) * p.chunk
        assert np.array_equal(g["limit"], r["limit"])
        assert np.allclose(g["mag"], r["mag"], rtol=1e-13)
        for key in ("R_prev", "R_t", "Lpdot", "Lp"):
            for blk in range(3):
                floor = _rel(rp[key][blk], r[key][blk]) if np.linalg.norm(r[key][blk]) > 0 else 0.0
                tol = max(1e-8, steps * floor)
                if np.linalg.norm(r[key][blk]) == 0:
                    assert np.linalg.norm(g[key][blk]) == 0, (k, key, blk)
                else:
                    assert _rel(g[key][blk], r[key][blk]) <= tol, (k, key, blk, _rel(g[key][blk], r[key][blk]),
                                                                   floor)
        assert np.linalg.norm(g["Lpdot"]) > 0
