"""The oracle's junctions and thermally activated breaking (Sec. 2.2) and the
paper's microstructure recipe (Sec. 3.2.1), against what fixes them from
outside: the published SplitMix64 test vector (the mixing function and the
stream of break fractions), closed-form capture times of
a loop that expands at a known speed, the clock of a stuck network, the
plain burst when no junction can form, and the Schmid factors of [001]
tension."""

import math

import numpy as np

import oracle as O
from paper_2005_02498_gb300 import workloads as W

MAT = W.Material().as_tuple()
MU, NU, BV, A, BDRAG = MAT
GOLDEN = 0x9E3779B97F4A7C15


def test_splitmix64_published_vector():
    # SplitMix64 seeded with 1234567: its first five outputs (Vigna's reference generator)
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
            16408922859458223821]
    got = [O.splitmix64_mix((1234567 + k * GOLDEN) & (2 ** 64 - 1)) for k in range(1, 6)]
    assert got == want
    # node 0's break fractions are that stream's outputs, top 53 bits on [0, 1):
    # the k-th draw (k = 0, 1, ...) is the generator's (k+1)-th output
    assert [O.junction_fraction(1234567, 0, k) for k in range(5)] == [(w >> 11) * 2.0 ** -53 for w in want]


def test_break_fractions_are_uniform_on_the_unit_interval():
    f = np.array([O.junction_fraction(99, p, k) for p in range(200) for k in range(10)])
    assert f.min() >= 0.0 and f.max() < 1.0
    assert len(np.unique(f)) == f.size
    assert abs(f.mean() - 0.5) < 0.02 and abs(f.var() - 1 / 12) < 0.01


def test_point_segment_distance_closed_forms():
    x1, x2 = np.array([0.0, 0.0, 0.0]), np.array([2.0, 0.0, 0.0])
    assert O.point_segment_dist2([1.0, 3.0, 4.0], x1, x2) == 25.0   # beside: perpendicular distance
    assert O.point_segment_dist2([-3.0, 4.0, 0.0], x1, x2) == 25.0  # before x1: distance to x1
    assert O.point_segment_dist2([5.0, 0.0, 4.0], x1, x2) == 25.0   # past x2: distance to x2
    assert O.point_segment_dist2([1.0, 0.0, 0.0], x1, x1) == 1.0    # zero-length segment


def _loop_and_line(R0, D, h=50e-9, tau=-100e6, N=32):
    """A circular glide loop (radius R0, plane z = 0, b along x, nodes
    counter-clockwise from angle 0) and a pinned straight line along z
    through (D, 0, 0): a two-node sessile loop."""
    phi = 2 * math.pi * np.arange(N) / N
    loop = np.stack([R0 * np.cos(phi), R0 * np.sin(phi), np.zeros(N)], 1)
    line = np.array([[D, 0.0, -h], [D, 0.0, h]])
    xyz = np.vstack([loop, line])
    off = np.array([0, N, N + 2], np.int64)
    burgers = np.array([[BV, 0, 0], [0, BV, 0]], float)
    normal = np.array([[0, 0, 1.0], [1.0, 0, 0]])
    pinned = np.r_[np.zeros(N, np.uint8), np.ones(2, np.uint8)]
    sig = np.array([0, 0, 0, 0, tau, 0.0])  # sigma_xz: the loop's resolved shear
    return W.Network(xyz, off, burgers, normal, pinned, (1e-6) ** 3, sig)


def test_capture_time_of_an_expanding_loop():
    """Without interactions a regular polygon loop under resolved shear tau
    expands radially at |tau| b cos(pi/N) / B, so node 0 reaches the line at
    distance D - r_c at a known step; it stops there and nodes more hops
    away than steps since the capture keep the free expansion."""
    N, R0, D, rc, dt, n = 32, 50e-9, 60e-9, 2e-9, 1e-12, 40
    net = _loop_and_line(R0, D)
    vr = 100e6 * BV * math.cos(math.pi / N) / BDRAG
    steps_to_reach = (D - rc - R0) / (vr * dt)
    assert 0.2 < steps_to_reach % 1 < 0.8  # well away from a step boundary
    i_cap = math.floor(steps_to_reach) + 1
    a, seed = 1e-3, 7
    r = O.burst_junctions(MAT, net, n, dt, rc, a, 0.0, seed, interactions=False)
    st = r["state"]
    assert st["seg"][0] == N and st["count"][0] == 1 and list(st["counts"]) == [1, 0, 0]
    assert np.all(st["seg"][1:N] == -1)
    assert math.isclose(st["brk"][0], i_cap * dt + a * O.junction_fraction(seed, 0, 0), rel_tol=1e-12)
    radius = np.linalg.norm(r["xyz"][:N, :2], axis=1)
    assert math.isclose(radius[0], R0 + vr * i_cap * dt, rel_tol=1e-12)
    assert n - i_cap < N // 2
    assert math.isclose(radius[N // 2], R0 + vr * n * dt, rel_tol=1e-12)
    assert math.isclose(r["S_t"], n * dt, rel_tol=1e-12) and r["state"]["clock"][1] == 0.0
    # the held node keeps still in a second burst
    r2 = O.burst_junctions(MAT, W.Network(r["xyz"], net.loop_off, net.burgers, net.normal, net.pinned,
                                          net.volume, net.sig_app), 5, dt, rc, a, 0.0, seed, state=st,
                           interactions=False)
    assert np.array_equal(r2["xyz"][0], r["xyz"][0])


def test_stuck_network_jumps_to_the_break_and_the_node_stays_free():
    """No stress and no interactions: nothing moves.  Node 0 starts within
    r_c of the line, is held at step 0, the clock jumps to its break time
    a f, the junction breaks at step 1, and the node does not form a
    junction with the same line again."""
    N, dt, n, rc, a = 32, 1e-12, 5, 2e-9, 1e-9
    net = _loop_and_line(50e-9, 50.5e-9, tau=0.0)
    seed = next(s for s in range(100) if O.junction_fraction(s, 0, 0) > 0.05)
    f0 = O.junction_fraction(seed, 0, 0)
    r = O.burst_junctions(MAT, net, n, dt, rc, a, 1e-15, seed, interactions=False)
    st = r["state"]
    assert list(st["counts"]) == [1, 1, 1]
    assert st["seg"][0] == -1 and st["last"][0] == 1 and st["count"][0] == 1
    assert math.isclose(st["clock"][1], a * f0 - dt, rel_tol=1e-12)
    assert math.isclose(st["clock"][0], a * f0 + (n - 1) * dt, rel_tol=1e-12)
    assert math.isclose(r["S_t"], a * f0 + (n - 1) * dt, rel_tol=1e-12)
    assert np.array_equal(r["xyz"], net.xyz) and np.all(r["Lp_avg"] == 0.0)
    seg = np.roll(net.xyz[:N], -1, 0) - net.xyz[:N]
    length = np.linalg.norm(seg, axis=1).sum() + 2 * 2 * 50e-9
    assert math.isclose(r["rho_avg"], length / net.volume, rel_tol=1e-13)  # rho kept through the jump
    # the jump puts the start of step 1 exactly at the break time, and a
    # junction is released by the step that starts at (or after) its break
    r2 = O.burst_junctions(MAT, net, 2, dt, rc, a, 1e-15, seed, interactions=False)
    assert list(r2["state"]["counts"]) == [1, 1, 1] and r2["state"]["seg"][0] == -1


def test_no_junction_reduces_to_the_plain_burst():
    net = W.junction_microstructure(5, W.uniaxial_stress(100e6), 1e13, 4e13, n_loops=10)
    assert 0 < net.pinned.sum() < net.n_nodes
    plain = O.burst(MAT, net, 6, 5e-13)
    r = O.burst_junctions(MAT, net, 6, 5e-13, 0.0, 1e-3, 0.0, 1)
    assert np.array_equal(r["xyz"], plain["xyz"]) and np.array_equal(r["Lp_avg"], plain["Lp_avg"])
    assert r["rho_avg"] == plain["rho_avg"] and list(r["state"]["counts"]) == [0, 0, 0]


def test_schmid_factors_of_001_tension_and_the_mobile_share():
    f = W.schmid_factors(W.uniaxial_stress(100e6))
    assert np.allclose(np.sort(np.abs(f)), [0] * 4 + [1 / math.sqrt(6)] * 8, atol=1e-15)
    net = W.junction_microstructure(3, W.uniaxial_stress(100e6), 2e12, 2e13, n_loops=48)
    sys_idx = W.slip_system_index(net.burgers, net.normal)
    mobile = net.pinned.reshape(net.n_loops, -1)[:, 0] == 0
    assert np.all(np.abs(f[sys_idx[mobile]]) > 0.4)  # no mobile loop on a system without resolved shear
    counts = np.bincount(sys_idx[~mobile], minlength=12)
    assert counts.max() - counts.min() <= 1  # sessile spread evenly
    assert mobile.sum() in (4, 5)  # 48 loops x 2e12 / 2.2e13
