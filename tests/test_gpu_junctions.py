"""GPU parity of the burst with junctions and thermally activated breaking
(ptadd_set_junctions, Sec. 2.2) with the oracle's junction burst, on the
paper's microstructure recipe (Sec. 3.2.1): 20 loops of 32 nodes (4 mobile,
16 sessile), 200 MPa [001], capture radius 20 nm, maximum break time 50 DD
steps, FP64 pair kernel, with the sessile loops of both of the paper's cases
(their Burgers vectors in their planes, or out of them as in Lomer-Cottrell
locks).  Two stuck rules: never (junctions form and break on the clock) and
always while a junction is held (the clock jumps to every break).  The case is checked to be well conditioned first: the oracle's
junction decisions do not change when the start positions move by 1e-10
relative, far more than the GPU and the oracle differ by."""

import numpy as np
import pytest

import oracle as O
from paper_2005_02498_gb300 import ptadd
from paper_2005_02498_gb300 import workloads as W

pytestmark = pytest.mark.gpu
MAT = W.Material().as_tuple()
STEPS, DT, RC, AMAX, SEED = 100, 5e-13, 2e-8, 2.5e-11, 5


def _net(case=2):
    return W.junction_microstructure(12, W.uniaxial_stress(200e6), 1e13, 3e13, n_loops=20, sessile_case=case)


def _relmax(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(b)))


@pytest.mark.parametrize("case", [2, 1])
@pytest.mark.parametrize("stuck", [0.0, 1.0])
def test_junction_burst_matches_oracle(stuck, case):
    net = _net(case)
    ref = O.burst_junctions(MAT, net, STEPS, DT, RC, AMAX, stuck, SEED)
    pert = net.copy()
    pert.xyz = net.xyz * (1 + 1e-10 * np.random.default_rng(0).uniform(-1, 1, net.xyz.shape))
    refp = O.burst_junctions(MAT, pert, STEPS, DT, RC, AMAX, stuck, SEED)
    for k in ("seg", "last", "count", "counts"):
        assert np.array_equal(ref["state"][k], refp["state"][k]), "ill-conditioned case: " + k
    formed, broken, jumps = ref["state"]["counts"]
    assert formed >= 10 and broken >= 10 and (jumps >= 10 if stuck else jumps == 0)
    with ptadd.Context(MAT, ptadd.PTADD_FP64, 0) as c:
        c.set_network(net)
        c.set_applied_stress(net.sig_app)
        c.set_junctions(RC, AMAX, stuck, SEED)
        Lp, rho = c.advance(STEPS, DT)
        x = c.get_nodes()
        j = c.junctions()
    st = ref["state"]
    assert np.array_equal(j["seg"], st["seg"]) and np.array_equal(j["last"], st["last"])
    assert np.array_equal(j["count"], st["count"])
    assert (j["formed"], j["broken"], j["jumps"]) == (formed, broken, jumps)
    assert j["held"] == int((st["seg"] >= 0).sum())
    assert np.allclose(j["break_time"], st["brk"], rtol=1e-12, atol=0)
    assert np.isclose(j["clock"], st["clock"][0], rtol=1e-12) and np.isclose(j["jumped"], st["clock"][1], rtol=1e-12)
    assert _relmax(x, ref["xyz"]) <= 1e-9
    assert _relmax(x - net.xyz, ref["xyz"] - net.xyz) <= 1e-6
    assert _relmax(Lp, ref["Lp_avg"]) <= 1e-8
    assert abs(rho / ref["rho_avg"] - 1) <= 1e-12


def test_no_capture_leaves_the_burst_unchanged_and_state_round_trips():
    net = _net()
    with ptadd.Context(MAT, ptadd.PTADD_FP64, 0) as c:
        c.set_network(net)
        c.set_applied_stress(net.sig_app)
        Lp0, rho0 = c.advance(20, DT)
        x0 = c.get_nodes()
        c.set_network(net)
        c.set_applied_stress(net.sig_app)
        c.set_junctions(0.0, AMAX, 0.0, SEED)  # nothing can be captured
        Lp1, rho1 = c.advance(20, DT)
        assert np.array_equal(c.get_nodes(), x0) and np.array_equal(Lp1, Lp0) and rho1 == rho0
        # save, run, restore, run again: the same junctions and positions
        c.set_junctions(RC, AMAX, 1.0, SEED)
        c.advance(30, DT)
        blob = c.get_state()
        LpA, _ = c.advance(30, DT)
        xA, jA = c.get_nodes(), c.junctions()
        c.set_state(blob)
        LpB, _ = c.advance(30, DT)
        xB, jB = c.get_nodes(), c.junctions()
        assert np.array_equal(xA, xB) and np.array_equal(LpA, LpB)
        for k in ("seg", "last", "count", "break_time", "clock", "jumped", "formed", "broken", "jumps"):
            assert np.array_equal(jA[k], jB[k]), k
        c.set_junctions(None)
        with pytest.raises(ptadd.PtaddError):
            c.junctions()
        with pytest.raises(ptadd.PtaddError):
            c.set_state(blob)  # a blob with junction state, junctions off
