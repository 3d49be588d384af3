"""GPU parity of junctions in the batched ensemble (ptadd_batch_set_junctions;
Sec. 2.2 inside the independent bursts of Sec. 4.1) with the oracle's
junction burst run on every realisation alone.

Three realisations of the paper's microstructure recipe (Sec. 3.2.1) of
different sizes and applied stresses (16, 20 and 24 loops of 32 nodes, each
with mobile and sessile loops; the 16-loop one with Lomer-Cottrell-type
sessiles, Case 1 of Sec. 3.2, the others with Case 2), capture radius 20 nm,
maximum break time 50 DD steps, FP64 pair kernel, 100 steps (the batch runs
them as 50 replays of its two-step graph).  Realisation r draws its break
fractions from the stream of seed ^ (r * 0x9E3779B97F4A7C15), so the oracle
runs it with that seed.  Two stuck rules: never, and always while a junction is held (every
realisation then jumps its own clock to each of its breaks).  Each case is
checked to be well conditioned first: the oracle's decisions do not change
when the start positions move by 1e-10 relative.
"""

import numpy as np
import pytest

import oracle as O
from paper_2005_02498_gb300 import ptadd
from paper_2005_02498_gb300 import workloads as W

pytestmark = pytest.mark.gpu
MAT = W.Material().as_tuple()
STEPS, DT, RC, AMAX, SEED = 100, 5e-13, 2e-8, 2.5e-11, 5
CASES = [(12, 20, 200e6, 2), (13, 16, 180e6, 1), (14, 24, 220e6, 2)]  # (seed, loops, uniaxial stress, sessile case)
MASK = (1 << 64) - 1


def _seed(r):
    return (SEED ^ (r * 0x9E3779B97F4A7C15)) & MASK


def _nets():
    return [W.junction_microstructure(s, W.uniaxial_stress(sg), 1e13, 3e13, n_loops=nl, sessile_case=c)
            for s, nl, sg, c in CASES]


def _relmax(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(b)))


@pytest.mark.parametrize("stuck", [0.0, 1.0])
def test_batched_junctions_match_the_oracle_per_realisation(stuck):
    nets = _nets()
    refs = []
    for r, nt in enumerate(nets):
        ref = O.burst_junctions(MAT, nt, STEPS, DT, RC, AMAX, stuck, _seed(r))
        pert = nt.copy()
        pert.xyz = nt.xyz * (1 + 1e-10 * np.random.default_rng(r).uniform(-1, 1, nt.xyz.shape))
        refp = O.burst_junctions(MAT, pert, STEPS, DT, RC, AMAX, stuck, _seed(r))
        for k in ("seg", "last", "count", "counts"):
            assert np.array_equal(ref["state"][k], refp["state"][k]), "ill-conditioned case: %d %s" % (r, k)
        formed, broken, jumps = ref["state"]["counts"]
        assert formed >= 5 and broken >= 5 and (jumps >= 5 if stuck else jumps == 0)
        refs.append(ref)
    batch = W.batch_from_networks(nets)
    with ptadd.Context(MAT, ptadd.PTADD_FP64, 0) as c:
        c.batch_set(batch)
        c.batch_set_junctions(RC, AMAX, stuck, SEED)
        Lp, rho = c.batch_advance(STEPS, DT)
        x = c.batch_get_nodes()
        per, arr = c.batch_junctions()
    for r, (nt, ref) in enumerate(zip(nets, refs)):
        a, b = batch.node_off[r], batch.node_off[r + 1]
        st = ref["state"]
        formed, broken, jumps = st["counts"]
        assert np.array_equal(arr["seg"][a:b], st["seg"]), r
        assert np.array_equal(arr["last"][a:b], st["last"]), r
        assert np.array_equal(arr["count"][a:b], st["count"]), r
        assert (per[r]["formed"], per[r]["broken"], per[r]["jumps"]) == (formed, broken, jumps), r
        assert per[r]["held"] == int((st["seg"] >= 0).sum())
        assert np.allclose(arr["break_time"][a:b], st["brk"], rtol=1e-12, atol=0)
        assert np.isclose(per[r]["clock"], st["clock"][0], rtol=1e-12)
        assert np.isclose(per[r]["jumped"], st["clock"][1], rtol=1e-12, atol=0)
        assert _relmax(x[a:b], ref["xyz"]) <= 1e-9
        assert _relmax(x[a:b] - nt.xyz, ref["xyz"] - nt.xyz) <= 1e-6
        assert _relmax(Lp[r], ref["Lp_avg"]) <= 1e-8
        assert abs(rho[r] / ref["rho_avg"] - 1) <= 1e-12
    if stuck:  # the clocks ran apart: each realisation jumped to its own breaks
        assert len({round(p["clock"] / 1e-15) for p in per}) == len(per)


def test_batched_junctions_off_and_out_of_reach_leave_the_burst_unchanged():
    nets = _nets()
    batch = W.batch_from_networks(nets)
    with ptadd.Context(MAT, ptadd.PTADD_FP64, 0) as c:
        c.batch_set(batch)
        Lp0, rho0 = c.batch_advance(20, DT)
        x0 = c.batch_get_nodes()
        with pytest.raises(ptadd.PtaddError) as e:
            c.batch_junctions()
        assert e.value.status == 5  # off
        c.batch_set(batch)
        c.batch_set_junctions(0.0, AMAX, 0.0, SEED)  # nothing can be captured
        Lp1, rho1 = c.batch_advance(20, DT)
        assert np.array_equal(c.batch_get_nodes(), x0) and np.array_equal(Lp1, Lp0) and np.array_equal(rho1, rho0)
        per, arr = c.batch_junctions()
        assert all(p["formed"] == 0 and p["held"] == 0 for p in per) and np.all(arr["seg"] == -1)
        assert all(np.isclose(p["clock"], 20 * DT, rtol=1e-12) for p in per)
        # switched off again: the plain burst from the same start
        c.batch_set(batch)
        c.batch_set_junctions(RC, AMAX, 1.0, SEED)
        c.batch_set_junctions(None)
        Lp2, rho2 = c.batch_advance(20, DT)
        assert np.array_equal(c.batch_get_nodes(), x0) and np.array_equal(Lp2, Lp0)
        with pytest.raises(ptadd.PtaddError) as e:
            c.batch_set_junctions(-1.0, AMAX, 0.0, SEED)
        assert e.value.status == 1


def test_batched_junctions_in_mixed_precision_form_and_break():
    """The mixed pair kernel moves the nodes ~1e-7 relative away from the FP64
    path, which can change a capture decision, so here the bar is behaviour:
    junctions form, hold and break in every realisation and the burst stays
    finite."""
    nets = _nets()
    with ptadd.Context(MAT, ptadd.PTADD_MIXED, 0) as c:
        c.batch_set(W.batch_from_networks(nets))
        c.batch_set_junctions(RC, AMAX, 1.0, SEED)
        Lp, rho = c.batch_advance(STEPS, DT)
        per, _ = c.batch_junctions()
    assert np.all(np.isfinite(Lp)) and np.all(rho > 0)
    assert all(p["formed"] >= 3 and p["broken"] >= 1 and p["jumps"] >= 1 for p in per)
