"""The oracle's Practical Time Averaging loop (Sec. 3.1) against the rules of
the paper's single-box algorithm, on the 512-segment network (CPU).  The
bursts themselves are pinned in test_oracle_pins.py; here the control flow:
the difference quotient, the jump rule, the extension rule, the step control
and the load ramp."""

import dataclasses

import numpy as np

import oracle as O
from oracle import pta as OP
from paper_2005_02498_gb300 import workloads as W

MAT = W.Material().as_tuple()


@dataclasses.dataclass
class P:
    rate: float = 1e9
    pattern: tuple = (0.0, 0.0, 1.0, 0.0, 0.0, 0.0)
    delta: float = 5e-3
    h0: float = 1e-2
    h_max: float = 1e-1
    dt: float = 5e-13
    chunk: int = 10
    tol_lp: float = 2e-2
    tol_rho: float = 1e-3
    max_chunks: int = 4
    extend_chunks: int = 3
    lpdot_max: float = 1e30
    max_jumps: int = 2
    strain_step: float = 0.002


def test_pta_records_follow_the_rules():
    p = P()
    recs = OP.run(MAT, W.small_loop_network(), p, 3)
    assert recs[0]["t"] == 0.0 and recs[0]["load"] == p.rate * p.delta  # l(-Delta) = 0
    for k, r in enumerate(recs):
        assert r["jumps"] == 0  # threshold out of reach
        assert np.allclose(r["Lpdot"], (r["Lp"] - r["Lp_prev"]) / p.delta, rtol=1e-12, atol=0)
        # the t - Delta average was extended until it no longer exceeded the t one, or the cap was hit
        assert np.linalg.norm(r["Lp_prev"]) <= np.linalg.norm(r["Lp"]) or r["extended"] == p.extend_chunks
        assert 1 <= r["chunks"][0] <= p.max_chunks and 1 <= r["chunks"][1] <= p.max_chunks
        assert r["load"] == p.rate * (r["t"] + p.delta)
        if k + 1 < len(recs):
            h = min(p.h_max, p.strain_step / np.linalg.norm(r["Lp"]))
            assert abs(recs[k + 1]["t"] - (r["t"] + h)) <= 1e-15 * max(1.0, r["t"] + h)


def test_pta_network_that_cannot_move_converges_in_two_chunks():
    """Every node pinned: each chunk's averages are Lp = 0 and the constant
    rho = length / volume, so each running average converges as soon as it
    can be compared (two chunks), nothing jumps or is extended, and the slow
    step is the largest allowed."""
    p = P()
    net = W.small_loop_network()
    net.pinned = np.ones(net.n_nodes, dtype=np.uint8)
    length = sum(np.linalg.norm(np.roll(net.xyz[a:b], -1, 0) - net.xyz[a:b], axis=1).sum()
                 for a, b in zip(net.loop_off[:-1], net.loop_off[1:]))
    rho = length / net.volume
    recs = OP.run(MAT, net, p, 2)
    for r in recs:
        assert r["chunks"] == [2, 2] and r["jumps"] == 0 and r["extended"] == 0
        assert np.all(r["Lp"] == 0.0) and np.all(r["Lpdot"] == 0.0) and r["rhodot"] == 0.0
        assert abs(r["rho"] / rho - 1) < 1e-12
    assert recs[1]["t"] == p.h_max


def test_pta_jump_rule_restarts_until_the_cap():
    p = P(lpdot_max=0.0, max_jumps=2, max_chunks=2)
    recs = OP.run(MAT, W.small_loop_network(), p, 1)
    assert recs[0]["jumps"] == 2


def test_pta_first_step_is_two_plain_bursts_when_one_chunk_is_allowed():
    """With one chunk per average and no extension, the first slow step is one
    burst at l(-Delta) = 0 and one burst at l(0) from where that one ended."""
    p = P(max_chunks=1, extend_chunks=0)
    net = W.small_loop_network()
    rec = OP.run(MAT, net, p, 1)[0]
    n1 = net.copy()
    n1.sig_app = np.zeros(6)
    r1 = O.burst(MAT, n1, p.chunk, p.dt)
    n2 = net.copy()
    n2.xyz = r1["xyz"]
    n2.sig_app = np.array(p.pattern) * p.rate * p.delta
    r2 = O.burst(MAT, n2, p.chunk, p.dt)
    assert np.array_equal(rec["Lp_prev"], r1["Lp_avg"]) and np.array_equal(rec["Lp"], r2["Lp_avg"])


def _chain(net, p, loads):
    """Plain oracle bursts of p.chunk steps, one per load value (times the
    pattern), each from the end state of the one before."""
    out, xyz = [], net.xyz.copy()
    for load in loads:
        m = net.copy()
        m.xyz, m.sig_app = xyz, np.array(p.pattern) * load
        out.append(O.burst(MAT, m, p.chunk, p.dt))
        xyz = out[-1]["xyz"]
    return out


def test_pta_second_step_starts_where_the_first_ended():
    """The microstructure is carried: the second slow step's bursts at
    l(t1 - Delta) and l(t1) continue from the end of the first step's l(0)
    burst."""
    p = P(max_chunks=1, extend_chunks=0)
    net = W.small_loop_network()
    recs = OP.run(MAT, net, p, 2)
    t1 = recs[1]["t"]
    # l(t) = rate (t + Delta), at t = t1 - Delta and at t = t1 (rounded as written)
    r = _chain(net, p, [0.0, p.rate * p.delta, p.rate * ((t1 - p.delta) + p.delta), p.rate * (t1 + p.delta)])
    assert np.array_equal(recs[0]["Lp"], r[1]["Lp_avg"])
    assert np.array_equal(recs[1]["Lp_prev"], r[2]["Lp_avg"]) and np.array_equal(recs[1]["Lp"], r[3]["Lp_avg"])


def test_pta_jump_restarts_the_pair_from_the_end_of_the_pair():
    """A jump restarts both averages from the state the l(t) burst ended in:
    with the threshold at 0 and one jump allowed, the step is the pair of
    bursts that follows the first pair."""
    p = P(max_chunks=1, extend_chunks=0, lpdot_max=0.0, max_jumps=1)
    net = W.small_loop_network()
    rec = OP.run(MAT, net, p, 1)[0]
    r = _chain(net, p, [0.0, p.rate * p.delta, 0.0, p.rate * p.delta])
    assert rec["jumps"] == 1
    assert np.array_equal(rec["Lp_prev"], r[2]["Lp_avg"]) and np.array_equal(rec["Lp"], r[3]["Lp_avg"])


class _StandInContext:
    """The single-realisation calls pta.run makes, answered by the oracle's
    burst on the host, so that the product's PTA driver is checked on the CPU
    against the oracle's independent loop."""

    def set_network(self, net):
        self.net, self.xyz, self.sig = net, net.xyz.copy(), net.sig_app.copy()

    def set_applied_stress(self, sig6):
        self.sig = np.asarray(sig6, float).copy()

    def get_state(self):
        return self.xyz.copy()

    def set_state(self, blob):
        self.xyz = blob.copy()

    def advance(self, n, dt):
        m = self.net.copy()
        m.xyz, m.sig_app = self.xyz, self.sig
        r = O.burst(MAT, m, n, dt)
        self.xyz = r["xyz"]
        return r["Lp_avg"], r["rho_avg"]


def test_product_pta_driver_follows_the_oracle_loop():
    from paper_2005_02498_gb300 import pta
    for lpdot_max, steps in ((1e30, 3), (0.0, 1)):
        p = P(lpdot_max=lpdot_max, max_chunks=3, extend_chunks=2)
        net = W.small_loop_network()
        got = pta.run(_StandInContext(), net, p, steps)
        want = OP.run(MAT, net, p, steps)
        for g, r in zip(got, want):
            assert (g["jumps"], g["chunks"], g["extended"]) == (r["jumps"], r["chunks"], r["extended"])
            assert g["t"] == r["t"]
            for key in ("Lp", "Lp_prev", "Lpdot"):
                assert np.allclose(g[key], r[key], rtol=1e-12, atol=0), key
            assert np.isclose(g["rhodot"], r["rhodot"], rtol=1e-9)
