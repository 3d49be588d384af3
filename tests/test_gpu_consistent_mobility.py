"""GPU parity of the consistent (Galerkin) mobility of Eq. 2.1
(ptadd_set_mobility) with the oracle's dense per-loop solve.

Networks: the 512-segment loop workload (free rings: the cyclic solve), the
same with every seventh node pinned (chains between pinned nodes), and the
paper's junction microstructure (fully pinned sessile loops beside free
mobile ones), alone and as one batch of three.  Bursts of 40 steps at dt =
5e-13 s, where the trajectories are well conditioned; FP64 to the FP64
bars, mixed to the mixed ones.
"""

import numpy as np
import pytest

import oracle as O
from paper_2005_02498_gb300 import ptadd
from paper_2005_02498_gb300 import workloads as W

pytestmark = pytest.mark.gpu
MAT = W.Material().as_tuple()
STEPS, DT = 40, 5e-13


def relmax(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(b)))


def relfro(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def _networks():
    small = W.small_loop_network()
    pinned = small.copy()
    pinned.pinned = (np.arange(pinned.n_nodes) % 7 == 3).astype(np.uint8)
    junc = W.junction_microstructure(12, W.uniaxial_stress(200e6), 1e13, 3e13, n_loops=20)
    return {"free": small, "pinned": pinned, "sessile": junc}


@pytest.mark.parametrize("name", ["free", "pinned", "sessile"])
@pytest.mark.parametrize("precision", [ptadd.PTADD_FP64, ptadd.PTADD_MIXED])
def test_consistent_mobility_burst_matches_oracle(name, precision):
    net = _networks()[name]
    ref = O.burst(MAT, net, STEPS, DT, consistent_mass=True)
    lumped = O.burst(MAT, net, STEPS, DT)
    with ptadd.Context(MAT, precision, 0) as c:
        c.set_network(net)
        c.set_applied_stress(net.sig_app)
        c.set_mobility(True)
        Lp, rho = c.advance(STEPS, DT)
        x = c.get_nodes()
    # the two mobilities differ by far more than the bars below
    assert relmax(lumped["xyz"] - net.xyz, ref["xyz"] - net.xyz) > 1e-3
    if precision == ptadd.PTADD_FP64:
        assert relmax(x, ref["xyz"]) <= 1e-9
        assert relmax(x - net.xyz, ref["xyz"] - net.xyz) <= 1e-7
        assert relmax(Lp, ref["Lp_avg"]) <= 1e-8
        assert abs(rho / ref["rho_avg"] - 1) <= 1e-12
    else:
        assert relmax(x - net.xyz, ref["xyz"] - net.xyz) <= 1e-4
        assert relfro(Lp, ref["Lp_avg"]) <= 1e-2
        assert abs(rho / ref["rho_avg"] - 1) <= 1e-6
    pin = net.pinned.astype(bool)
    assert np.all(x[pin] == net.xyz[pin])


def test_set_mobility_arguments_and_junctions():
    net = _networks()["sessile"]
    with ptadd.Context(MAT, ptadd.PTADD_FP64, 0) as c:
        c.set_network(net)
        c.set_applied_stress(net.sig_app)
        with pytest.raises(ptadd.PtaddError) as e:
            ptadd._check(c._lib.ptadd_set_mobility(c._h, 2))
        assert e.value.status == 1
        c.set_junctions(2e-8, 2.5e-11, 0.0, 5)
        with pytest.raises(ptadd.PtaddError) as e:
            c.set_mobility(True)
        assert e.value.status == 5
        c.set_junctions(None)
        c.set_mobility(True)
        with pytest.raises(ptadd.PtaddError) as e:
            c.set_junctions(2e-8, 2.5e-11, 0.0, 5)
        assert e.value.status == 5
        # back to the lumped form: the plain burst of the oracle
        c.set_mobility(False)
        Lp, rho = c.advance(5, DT)
        ref = O.burst(MAT, net, 5, DT)
        assert relmax(Lp, ref["Lp_avg"]) <= 1e-8


@pytest.mark.parametrize("precision", [ptadd.PTADD_FP64, ptadd.PTADD_MIXED])
def test_consistent_mobility_in_the_batch_matches_oracle(precision):
    nets = list(_networks().values())
    refs = [O.burst(MAT, nt, STEPS, DT, consistent_mass=True) for nt in nets]
    batch = W.batch_from_networks(nets)
    with ptadd.Context(MAT, precision, 0) as c:
        c.set_mobility(True)
        c.batch_set(batch)
        Lp, rho = c.batch_advance(STEPS, DT)
        x = c.batch_get_nodes()
        with pytest.raises(ptadd.PtaddError) as e:
            c.batch_set_junctions(2e-8, 2.5e-11, 0.0, 5)
        assert e.value.status == 5
    for r, (nt, ref) in enumerate(zip(nets, refs)):
        a, b = batch.node_off[r], batch.node_off[r + 1]
        if precision == ptadd.PTADD_FP64:
            assert relmax(x[a:b], ref["xyz"]) <= 1e-9, r
            assert relmax(x[a:b] - nt.xyz, ref["xyz"] - nt.xyz) <= 1e-7, r
            assert relmax(Lp[r], ref["Lp_avg"]) <= 1e-8, r
            assert abs(rho[r] / ref["rho_avg"] - 1) <= 1e-12, r
        else:
            assert relmax(x[a:b] - nt.xyz, ref["xyz"] - nt.xyz) <= 1e-4, r
            assert relfro(Lp[r], ref["Lp_avg"]) <= 1e-2, r
