"""The block-level front end of the coupling (Sec. 4.2, 4.2.1) on the CPU:
the oracle's block average and stress pair against closed forms, the C-ABI
host functions against the oracle, and the oracle's increment (lock step,
rescale, Lp update, limit rule) with stand-in bursts whose answers are known."""

import dataclasses

import numpy as np
import pytest

import oracle as O
from oracle import blocks as OB
from paper_2005_02498_gb300 import blocks as B
from paper_2005_02498_gb300 import ptadd
from paper_2005_02498_gb300 import workloads as W

EDGE = 1e-6
MAT = W.Material().as_tuple()


def _mesh(side=3, elems=4):
    return B.synthetic_mesh(side, elems, EDGE, EDGE)


def test_mesh_weights_add_up_to_the_block_volume():
    pts, w, blk = _mesh()
    for r in range(9):
        assert np.isclose(w[blk == r].sum(), EDGE ** 3, rtol=1e-13)
        sel = pts[blk == r]
        bx, by = r % 3, r // 3
        assert sel[:, 0].min() > bx * EDGE and sel[:, 0].max() < (bx + 1) * EDGE
        assert sel[:, 1].min() > by * EDGE and sel[:, 1].max() < (by + 1) * EDGE


def test_oracle_block_average_closed_forms():
    pts, w, blk = _mesh()
    centre = np.array([[(r % 3 + 0.5) * EDGE, (r // 3 + 0.5) * EDGE] for r in range(9)])
    # piecewise constant: the constants
    c = np.arange(54, dtype=float).reshape(9, 6) - 20.0
    got = OB.block_average(c[blk], w, blk, 9)
    assert np.allclose(got, c, rtol=1e-14, atol=0)
    # linear in position: the value at the block centre
    T = np.zeros((len(w), 6))
    T[:, 0] = 3.0 + 2e6 * pts[:, 0] - 5e6 * pts[:, 1]
    T[:, 5] = -1.0 + 7e6 * pts[:, 1]
    got = OB.block_average(T, w, blk, 9)
    assert np.allclose(got[:, 0], 3.0 + 2e6 * centre[:, 0] - 5e6 * centre[:, 1], rtol=1e-13)
    assert np.allclose(got[:, 5], -1.0 + 7e6 * centre[:, 1], rtol=1e-13)
    # (x - x_c)^2 averages to edge^2 / 12 over a square (the 2 x 2 Gauss rule is exact for it)
    T = np.zeros((len(w), 6))
    T[:, 2] = ((pts[:, 0] - centre[blk, 0]) / EDGE) ** 2
    assert np.allclose(OB.block_average(T, w, blk, 9)[:, 2], 1.0 / 12.0, rtol=1e-13)


def test_oracle_stress_pair_closed_forms():
    rng = np.random.default_rng(5)
    A, Bm = rng.normal(size=(4, 6)) * 50e6, rng.normal(size=(4, 6)) * 20e6
    t, dt, ds = 3.0, 0.7, 0.1
    # a stress rising linearly in time: the extrapolation lands on T(t + Delta*)
    Tp, Tt, mag = OB.stress_pair(A + Bm * t, A + Bm * (t - dt), ds, dt, 0.5e6)
    assert np.all(mag == 1.0)
    assert np.allclose(Tp, A + Bm * t, rtol=1e-14) and np.allclose(Tt, A + Bm * (t + ds), rtol=1e-12, atol=1e-3)
    # a small gap is raised to gap_min along its own direction
    Tp, Tt, mag = OB.stress_pair(A + Bm * 1e-3 * t, A + Bm * 1e-3 * (t - dt), ds, dt, 0.5e6)
    gap0 = Bm * 1e-3 * ds
    for r in range(4):
        g = Tt[r] - Tp[r]
        full = np.array([[g[0], g[5], g[4]], [g[5], g[1], g[3]], [g[4], g[3], g[2]]])
        assert np.isclose(np.linalg.norm(full), 0.5e6, rtol=1e-12)
        assert np.allclose(g, mag[r] * gap0[r], rtol=1e-10, atol=1e-6)
        assert mag[r] > 1
    # the norm is that of the full tensor: a shear gap s counts as sqrt(2) s
    Tp, Tt, mag = OB.stress_pair(np.array([[0, 0, 0, 0, 0, 1e5]]), np.zeros((1, 6)), 1.0, 1.0, 0.5e6)
    assert np.isclose(mag[0], 0.5e6 / (np.sqrt(2) * 1e5), rtol=1e-14)
    # no gap: nothing to inflate, rates scaled to 0
    Tp, Tt, mag = OB.stress_pair(A, A, ds, dt, 0.5e6)
    assert np.all(np.isinf(mag)) and np.array_equal(Tp, Tt)
    Tp, Tt, mag = OB.stress_pair(A, None, ds, 0.0, 0.5e6)
    assert np.all(np.isinf(mag)) and np.array_equal(Tp, A)


def test_c_abi_block_functions_match_the_oracle():
    rng = np.random.default_rng(6)
    pts, w, blk = _mesh()
    T = rng.normal(size=(len(w), 6)) * 80e6
    got = ptadd.block_average(T, w, blk, 9)
    assert np.allclose(got, OB.block_average(T, w, blk, 9), rtol=1e-13, atol=1e-6)
    Tk = rng.normal(size=(20, 6)) * 50e6
    step = rng.normal(size=(20, 6)) * 10 ** rng.uniform(4, 7, size=(20, 1))
    step[3] = 0.0
    for Tkm1, dtp in ((Tk - step, 0.8), (None, 0.0), (Tk - step, 0.0)):
        got = ptadd.block_stress_pair(Tk, Tkm1, 0.1, dtp, 0.5e6)
        want = OB.stress_pair(Tk, Tkm1, 0.1, dtp, 0.5e6)
        assert np.array_equal(got[0], want[0])
        assert np.allclose(got[1], want[1], rtol=1e-14, atol=1e-7)
        assert np.array_equal(np.isinf(got[2]), np.isinf(want[2]))
        fin = np.isfinite(want[2])
        assert np.allclose(got[2][fin], want[2][fin], rtol=1e-13)


def test_c_abi_block_functions_reject_bad_input():
    T, w, blk = np.zeros((4, 6)), np.ones(4), np.array([0, 0, 1, 1], np.int32)
    ptadd.block_average(T, w, blk, 2)
    for args in ((T, w, np.array([0, 0, 1, 2], np.int32), 2),  # index out of range
                 (T, np.array([1, 0, 1, 1.0]), blk, 2),        # zero weight
                 (T, w, blk, 3),                               # empty block
                 (np.full((4, 6), np.nan), w, blk, 2)):
        with pytest.raises(ptadd.PtaddError):
            ptadd.block_average(*args)
    with pytest.raises(ptadd.PtaddError):
        ptadd.block_stress_pair(np.zeros((1, 6)), None, 0.0, 1.0, 0.5e6)
    with pytest.raises(ptadd.PtaddError):
        ptadd.block_stress_pair(np.full((1, 6), np.inf), None, 0.1, 1.0, 0.5e6)


@dataclasses.dataclass
class P:
    delta_star: float = 0.1
    gap_min: float = 0.5e6
    stress_jump: float = 3e6
    strain_step: float = 0.002
    dt: float = 5e-13
    chunk: int = 10
    tol_lp: float = 2e-2
    tol_rho: float = 1e-3
    max_chunks: int = 8


C = np.arange(9.0).reshape(3, 3) * 1e-9 + np.eye(3) * 1e-8  # Lp per Pa of sigma_zz


def _linear_burst(mat, net, n, dt):
    """Stand-in burst: the average answer is linear in the stress and the
    microstructure does not change."""
    return {"xyz": net.xyz, "Lp_avg": C * net.sig_app[2], "rho_avg": 1e12 + 1e3 * net.sig_app[2]}


def test_rescaled_rate_is_the_rate_of_the_original_stress_pair():
    """With an answer linear in the stress, dividing by mag gives exactly the
    rate of the un-inflated pair: the reason the coupling rescales."""
    net = W.small_loop_network()
    Tk = np.zeros((3, 6))
    Tk[:, 2] = [40e6, 50e6, 60e6]
    Tkm1 = Tk.copy()
    Tkm1[:, 2] -= [1e6, 2e6, 9e6]
    state = {"Lp": np.zeros((3, 3, 3)), "Lpdot": np.zeros((3, 3, 3))}
    rec = OB.increment(None, net, [net.xyz.copy() for _ in range(3)], state, Tk, Tkm1, 1.0, P(), _linear_burst)
    assert rec["chunks"] == [2, 2]
    assert rec["mag"][0] > 1 and rec["mag"][1] > 1 and rec["mag"][2] == 1.0
    for r in range(3):
        want = C * (0.1 * (Tk[r, 2] - Tkm1[r, 2])) / 0.1
        assert np.allclose(rec["Lpdot"][r], want, rtol=1e-9, atol=0)
        assert np.isclose(rec["rhodot"][r], 1e3 * (Tk[r, 2] - Tkm1[r, 2]), rtol=1e-9)
    assert np.array_equal(rec["Lp"], np.zeros((3, 3, 3)))  # the previous rate was 0
    # next increment: Lp moves by the previous rate times dt^{k-1}
    prev = state["Lpdot"].copy()
    rec2 = OB.increment(None, net, [net.xyz.copy() for _ in range(3)], state, Tk, Tkm1, 2.5, P(), _linear_burst)
    assert np.allclose(rec2["Lp"], prev * 2.5, rtol=1e-15, atol=0)


def test_limit_rule_freezes_the_block_and_stops_the_load():
    net = W.small_loop_network()
    Tk = np.zeros((2, 6))
    Tk[:, 2] = [40e6, 50e6]
    state = {"Lp": np.zeros((2, 3, 3)), "Lpdot": np.zeros((2, 3, 3))}
    state["Lpdot"][1] = np.eye(3) * 0.03 / np.sqrt(3)  # |Lpdot| = 0.03 /s
    rec = OB.increment(None, net, [net.xyz.copy() for _ in range(2)], state, Tk, Tk - 1e6, 1.0, P(), _linear_burst)
    assert list(rec["limit"]) == [False, True] and not rec["load_on"]  # 0.03 * 0.1 >= 0.002
    assert np.array_equal(rec["Lpdot"][1], np.zeros((3, 3))) and np.linalg.norm(rec["Lpdot"][0]) > 0


def _drifting_burst(mat, net, n, dt):
    """Stand-in burst whose answer settles geometrically; the call count is
    carried in the positions and the decay rate in sigma_xx."""
    k = net.xyz[0, 0] + 1.0
    xyz = net.xyz.copy()
    xyz[0, 0] = k
    q = net.sig_app[0]
    return {"xyz": xyz, "Lp_avg": np.eye(3) * (1.0 + q ** k), "rho_avg": 1.0}


def test_phases_run_in_lock_step_until_every_block_has_converged():
    net = W.small_loop_network()
    net.xyz[0, 0] = 0.0
    p = P(tol_lp=1e-3, max_chunks=100)
    alone = []
    for q in (0.3, 0.6, 0.8):
        T = np.array([[q, 0, 0, 0, 0, 0]])
        st = {"Lp": np.zeros((1, 3, 3)), "Lpdot": np.zeros((1, 3, 3))}
        alone.append(OB.increment(None, net, [net.xyz.copy()], st, T, None, 0.0, p, _drifting_burst)["chunks"][0])
    assert alone[0] < alone[1] < alone[2] < p.max_chunks
    T = np.array([[q, 0, 0, 0, 0, 0] for q in (0.3, 0.6, 0.8)])
    st = {"Lp": np.zeros((3, 3, 3)), "Lpdot": np.zeros((3, 3, 3))}
    rec = OB.increment(None, net, [net.xyz.copy() for _ in range(3)], st, T, None, 0.0, p, _drifting_burst)
    assert rec["chunks"][0] == max(alone)


def test_stress_step_control_halves_down_to_delta_star():
    p = P()
    Tk = np.zeros((2, 6))
    calls = []

    def solve(dt):
        calls.append(dt)
        out = Tk.copy()
        out[1, 0] = 10e6 * dt  # 10 MPa per second
        return out

    dt, T = B.stress_step_control(solve, Tk, 1.0, p)
    assert calls == [1.0, 0.5, 0.25] and dt == 0.25 and T[1, 0] == 2.5e6
    calls.clear()
    dt, _ = B.stress_step_control(lambda h: Tk + 1e9 * h, Tk, 1.0, p)
    assert dt == p.delta_star


class _StandInBatch:
    """The batch calls of a context, answered by the oracle's burst on the
    host (or another burst function of the same signature), so that the
    product's block driver can be checked on the CPU."""

    def __init__(self, net, burst_fn=O.burst):
        self.net, self.burst_fn = net, burst_fn

    def batch_set(self, batch):
        self.xyz = [batch.xyz[batch.node_off[r]:batch.node_off[r + 1]].copy() for r in range(batch.R)]

    def batch_set_stress(self, sig6):
        self.sig = np.asarray(sig6, float).reshape(-1, 6).copy()

    def batch_advance(self, n, dt):
        lp, rho = np.zeros((len(self.xyz), 3, 3)), np.zeros(len(self.xyz))
        for r in range(len(self.xyz)):
            m = self.net.copy()
            m.xyz, m.sig_app = self.xyz[r], self.sig[r]
            b = self.burst_fn(MAT, m, n, dt)
            self.xyz[r], lp[r], rho[r] = b["xyz"], b["Lp_avg"], b["rho_avg"]
        return lp, rho


def test_block_driver_follows_the_oracle_increment():
    """The product's driver and the oracle's increment, on the same bursts
    (the oracle's), take the same decisions and give the same rates."""
    net = W.small_loop_network()
    p = P(chunk=5, max_chunks=3)
    Tk = np.zeros((2, 6))
    Tk[:, 2] = [45e6, 55e6]
    steps = [(Tk - np.array([[0, 0, 1e6, 0, 0, 0], [0, 0, 8e6, 0, 0, 2e5]]), 1.0),
             (Tk + np.array([[0, 0, 2e6, 0, 0, 0], [0, 0, 1e6, 0, 0, 0]]), 0.5)]
    box = B.BlockPTA(_StandInBatch(net), net, 2, p)
    xyz = [net.xyz.copy(), net.xyz.copy()]
    state = {"Lp": np.zeros((2, 3, 3)), "Lpdot": np.zeros((2, 3, 3))}
    prev = None
    for T_other, dtp in steps:
        T_km1, T_k = (T_other, Tk) if prev is None else (prev, T_other)
        got = box.increment(T_k, T_km1, dtp)
        want = OB.increment(MAT, net, xyz, state, T_k, T_km1, dtp, p)
        assert got["chunks"] == want["chunks"]
        assert np.array_equal(got["limit"], want["limit"])
        for key in ("T_prev", "T_t", "mag", "R_prev", "R_t", "Lpdot", "rhodot", "Lp"):
            assert np.allclose(got[key], want[key], rtol=1e-12, atol=0), key
        prev = T_k


def test_block_driver_runs_in_lock_step_like_the_oracle():
    """Blocks whose answers settle at different rates: the product's driver,
    like the oracle's increment, keeps every block running until the slowest
    one has converged."""
    net = W.small_loop_network()
    net.xyz[0, 0] = 0.0
    p = P(tol_lp=1e-3, max_chunks=100)
    T = np.array([[q, 0, 0, 0, 0, 0] for q in (0.3, 0.6, 0.8)])
    st = {"Lp": np.zeros((3, 3, 3)), "Lpdot": np.zeros((3, 3, 3))}
    want = OB.increment(None, net, [net.xyz.copy() for _ in range(3)], st, T, None, 0.0, p, _drifting_burst)
    got = B.BlockPTA(_StandInBatch(net, _drifting_burst), net, 3, p).increment(T, None, 0.0)
    assert got["chunks"] == want["chunks"] and want["chunks"][0] > 2
    assert np.allclose(got["R_prev"], want["R_prev"], rtol=1e-15, atol=0)


def test_synthetic_coupling_run_on_stand_in_bursts():
    """The prescribed-field driver: the stress-based step halves a step that
    would change a block stress by more than 3 MPa, the first increment has
    no previous stress (rates 0), and once a block meets the limit condition
    the load stops and the step drops to Delta*."""
    net = W.small_loop_network()
    p = B.BlockParams(chunk=2, max_chunks=2)
    recs = B.run_synthetic(_StandInBatch(net), net, p, side=2, increments=3, rate=5e6)
    assert recs[0]["dt"] == 0.5  # 5 MPa/s x 1 s x (1 + 0.5/4) > 3 MPa; half of it is not
    assert recs[0]["mag"] == [None] * 4 and recs[0]["Lpdot_norm"] == [0.0] * 4
    # gaps of 0.1 s / 0.5 s x 2.5 MPa x (1 -/+ 0.5/4): the lower row raised to 0.5 MPa, the upper row not
    assert recs[1]["mag"][2:] == [1.0, 1.0] and min(recs[1]["mag"][:2]) > 1 and min(recs[1]["Lpdot_norm"]) > 0
    assert recs[2]["limit"] == [True] * 4 and recs[2]["dt"] == p.delta_star
    assert recs[2]["load"] == recs[1]["load"] + 5e6 * recs[1]["dt"]
