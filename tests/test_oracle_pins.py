"""Pins of the FP64 CPU oracle against closed forms, invariants and brute force.

Each test fixes the oracle against something other than itself: textbook
fields (Hirth-Lothe), the regularised screw field of the nonsingular theory,
exact identities of the discretisation, finite differences, long-double
quadrature of the integrand written out index by index, and magnitudes the
paper prints.  CPU only.
"""

import json
import math
import os
import zlib

import numpy as np
import pytest

import oracle as O
from paper_2005_02498_gb300 import workloads as W

MU, NU, BB, A = 48e9, 0.34, 2.556e-10, 2.556e-10
MAT = (MU, NU, BB, A, 1e-4)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def voigt(s):
    return np.array([s[0, 0], s[1, 1], s[2, 2], s[1, 2], s[0, 2], s[0, 1]])


def full(v):
    return np.array([[v[0], v[5], v[4]], [v[5], v[1], v[3]], [v[4], v[3], v[2]]])


def rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300)


def random_rotation(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


# ----------------------------------------------------------------- P15
def test_gauss4_integrates_degree7_exactly():
    xi, w = O.gauss4()
    for k in range(8):
        assert abs(np.sum(w * xi ** k) - 1.0 / (k + 1)) < 1e-15
    assert abs(np.sum(w * xi ** 8) - 1.0 / 9) > 1e-7  # degree 8 is not exact


# ------------------------------------------------ derivatives of R_a
def test_ra_third_derivatives_match_finite_differences():
    rng = np.random.default_rng(3)
    ld = np.longdouble
    for _ in range(4):
        R = rng.normal(size=3) * 2.0
        a = 0.7
        d3, dl = O.ra_derivs(R, a)
        h = ld(1e-3)

        def f(x):
            x = np.asarray(x, dtype=ld)
            return np.sqrt(np.sum(x * x) + ld(a) ** 2)

        fd = np.zeros((3, 3, 3))
        E = np.eye(3, dtype=ld)
        for i in range(3):
            for j in range(3):
                for k in range(3):
                    acc = ld(0)
                    for si in (1, -1):
                        for sj in (1, -1):
                            for sk in (1, -1):
                                acc += si * sj * sk * f(R + h * (si * E[i] + sj * E[j] + sk * E[k]))
                    fd[i, j, k] = float(acc / (8 * h ** 3))
        assert rel(d3, fd) < 1e-5
        # gradient of the Laplacian is the contraction of the third derivatives
        assert rel(dl, np.einsum("ipp->i", d3)) < 1e-14


# ----------------------------------------------------------------- P1
@pytest.mark.parametrize("r_over_a", [0.0, 0.3, 1.0, 3.0, 100.0])
def test_regularised_infinite_screw(r_over_a):
    """sigma_theta_z = mu b r (r^2 + 2a^2) / (2 pi (r^2 + a^2)^2) for b = t = z."""
    half = 0.5e10 * A  # end corrections ~ (r/half)^2 < 1e-15
    x1, x2, bv = np.array([0, 0, -half]), np.array([0, 0, half]), np.array([0, 0, BB])
    r = r_over_a * A
    for ang in (0.0, 0.7, 2.5):
        p = np.array([r * math.cos(ang), r * math.sin(ang), 0.0])
        s = full(O.seg_stress(MAT, x1, x2, bv, p))
        stz = MU * BB * r * (r * r + 2 * A * A) / (2 * math.pi * (r * r + A * A) ** 2)
        # sigma_xz = -stz sin, sigma_yz = stz cos; every other component zero
        exp = np.zeros((3, 3))
        exp[0, 2] = exp[2, 0] = -stz * math.sin(ang)
        exp[1, 2] = exp[2, 1] = stz * math.cos(ang)
        scale = max(stz, MU * BB / (2 * math.pi * A) * 1e-3)
        assert np.max(np.abs(s - exp)) / scale < 1e-12


def test_short_screw_expression_is_far_field_limit():
    """mu b r/(2 pi (r^2+a^2)) differs from the full form by a^2/(r^2+a^2)."""
    half = 0.5e10 * A
    x1, x2, bv = np.array([0, 0, -half]), np.array([0, 0, half]), np.array([0, 0, BB])
    for r_over_a in (32.0, 100.0, 1000.0):
        r = r_over_a * A
        s = O.seg_stress(MAT, x1, x2, bv, [r, 0, 0])[3]
        short = MU * BB * r / (2 * math.pi * (r * r + A * A))
        assert abs(s / short - 1.0) <= A * A / (r * r + A * A) * 1.0000001
        assert abs(s / short - 1.0) < 1e-3


# ----------------------------------------------------------------- P2
@pytest.mark.parametrize("nu", [0.0, 0.25, 0.34])
def test_hirth_lothe_edge_limit(nu):
    mat = (MU, nu, BB, 1e-7 * A, 1e-4)
    half = 0.5e10 * A
    x1, x2 = np.array([0, 0, -half]), np.array([0, 0, half])
    D = MU * BB / (2 * math.pi * (1 - nu))
    for (x, y) in [(3 * A, 2 * A), (-5 * A, 7 * A), (10 * A, -1 * A), (0.0, 4 * A)]:
        s = full(O.seg_stress(mat, x1, x2, [BB, 0, 0], [x, y, 0]))
        r2 = x * x + y * y
        e = np.zeros((3, 3))
        e[0, 0] = -D * y * (3 * x * x + y * y) / r2 ** 2
        e[1, 1] = D * y * (x * x - y * y) / r2 ** 2
        e[0, 1] = e[1, 0] = D * x * (x * x - y * y) / r2 ** 2
        e[2, 2] = nu * (e[0, 0] + e[1, 1])
        assert np.max(np.abs(s - e)) / np.max(np.abs(e)) < 1e-12


def test_hirth_lothe_screw_limit_and_far_field():
    half = 0.5e10 * A
    x1, x2, bv = np.array([0, 0, -half]), np.array([0, 0, half]), np.array([0, 0, BB])
    mat0 = (MU, NU, BB, 1e-7 * A, 1e-4)
    for (x, y) in [(3 * A, 2 * A), (-5 * A, 7 * A)]:
        s = full(O.seg_stress(mat0, x1, x2, bv, [x, y, 0]))
        r2 = x * x + y * y
        assert abs(s[0, 2] - (-MU * BB * y / (2 * math.pi * r2))) / (MU * BB / (2 * math.pi * math.sqrt(r2))) < 1e-12
        assert abs(s[1, 2] - (MU * BB * x / (2 * math.pi * r2))) / (MU * BB / (2 * math.pi * math.sqrt(r2))) < 1e-12
    # far field with the physical core: deviation is O(a^2/r^2)
    D = MU * BB / (2 * math.pi * (1 - NU))
    for r_over_a in (30.0, 300.0):
        x, y = 0.6 * r_over_a * A, 0.8 * r_over_a * A
        s = full(O.seg_stress(MAT, x1, x2, [BB, 0, 0], [x, y, 0]))
        r2 = x * x + y * y
        exx = -D * y * (3 * x * x + y * y) / r2 ** 2
        assert abs(s[0, 0] / exx - 1) < 3 * A * A / r2


# --------------------------------------------------------- P3, P8
def _random_case(rng, kind):
    x1 = rng.normal(size=3) * 20 * A
    t = rng.normal(size=3)
    t /= np.linalg.norm(t)
    L = rng.uniform(5, 80) * A
    x2 = x1 + L * t
    bv = rng.normal(size=3)
    bv *= BB / np.linalg.norm(bv)
    perp = np.cross(t, rng.normal(size=3))
    perp /= np.linalg.norm(perp)
    if kind == "generic":
        x = rng.normal(size=3) * 30 * A
    elif kind == "on_extension":  # beyond the end, near the line: d ~ a
        x = x2 + rng.uniform(2, 40) * A * t + rng.uniform(0, 0.5) * A * perp
    elif kind == "behind_start":
        x = x1 - rng.uniform(2, 40) * A * t + rng.uniform(0, 0.5) * A * perp
    elif kind == "on_segment":  # field point on the line inside the segment
        x = x1 + rng.uniform(0.1, 0.9) * L * t
    elif kind == "near_side":
        x = x1 + rng.uniform(0.0, 1.0) * L * t + rng.uniform(0.2, 2.0) * A * perp
    else:  # far
        x = x1 + rng.normal(size=3) * 3000 * A
    return x1, x2, bv, x


@pytest.mark.parametrize("kind", ["generic", "on_extension", "behind_start", "on_segment", "near_side", "far"])
def test_analytic_matches_brute_force_quadrature(kind):
    rng = np.random.default_rng(zlib.crc32(kind.encode()))
    for _ in range(4):
        x1, x2, bv, x = _random_case(rng, kind)
        L = np.linalg.norm(x2 - x1)
        panels = int(min(2048, max(32, 8 * L / A)))
        q = O.seg_stress_quad(MAT, x1, x2, bv, x, panels=panels, order=16)
        # P3; the scale is the core-size stress mu|b|/a, which bounds the integrand
        core = MU * BB / A
        assert np.max(np.abs(q - q.T)) <= 1e-17 * core
        s = O.seg_stress(MAT, x1, x2, bv, x)
        err = np.max(np.abs(s - voigt(q)))
        # on the line itself terms of size mu|b|/a cancel: a few ulps of that scale
        assert err < 1e-13 * np.max(np.abs(q)) or err < 1e-15 * core, kind


# --------------------------------------------------------- P4, P5
def test_linear_in_burgers_vector():
    rng = np.random.default_rng(5)
    x1, x2, _, x = _random_case(rng, "generic")
    b1, b2 = rng.normal(size=3) * BB, rng.normal(size=3) * BB
    s1 = O.seg_stress(MAT, x1, x2, b1, x)
    s2 = O.seg_stress(MAT, x1, x2, b2, x)
    s12 = O.seg_stress(MAT, x1, x2, 2.5 * b1 - 0.75 * b2, x)
    assert rel(s12, 2.5 * s1 - 0.75 * s2) < 1e-14


def test_translation_invariance_and_rotation_covariance():
    rng = np.random.default_rng(6)
    for _ in range(5):
        x1, x2, bv, x = _random_case(rng, "generic")
        s = full(O.seg_stress(MAT, x1, x2, bv, x))
        sh = rng.normal(size=3) * 1000 * A
        st = full(O.seg_stress(MAT, x1 + sh, x2 + sh, bv, x + sh))
        assert rel(st, s) < 1e-12
        Q = random_rotation(rng)
        sr = full(O.seg_stress(MAT, Q @ x1, Q @ x2, Q @ bv, Q @ x))
        assert rel(sr, Q @ s @ Q.T) < 1e-12


# ----------------------------------------------------------------- P6
def test_split_segment_is_additive():
    rng = np.random.default_rng(7)
    for kind in ("generic", "near_side", "on_extension", "far"):
        x1, x2, bv, x = _random_case(rng, kind)
        for f in (0.5, 0.13):
            xm = x1 + f * (x2 - x1)
            s = O.seg_stress(MAT, x1, x2, bv, x)
            s2 = O.seg_stress(MAT, x1, xm, bv, x) + O.seg_stress(MAT, xm, x2, bv, x)
            assert rel(s2, s) < 1e-13


# ----------------------------------------------------------------- P7
def _polygon(n, radius, centre, e1, e2, bvec, sense=1.0):
    phi = sense * 2 * math.pi * np.arange(n) / n
    xyz = centre + radius * (np.cos(phi)[:, None] * e1 + np.sin(phi)[:, None] * e2)
    return W.Network(xyz, np.array([0, n], np.int64), np.asarray(bvec, float)[None, :],
                     np.cross(e1, e2)[None, :], np.zeros(n, np.uint8), 1e-18, np.zeros(6))


def test_closed_loop_far_field_decays_as_r_cubed():
    rng = np.random.default_rng(8)
    Rl = 200 * A
    net = _polygon(32, Rl, np.zeros(3), np.array([1.0, 0, 0]), np.array([0, 1.0, 0]), [BB, 0, 0])
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    rs = np.array([10, 30, 100, 300, 1000]) * Rl
    mags = []
    for r in rs:
        s = O.stress_at(MAT, net, (r * d)[None, :])[0]
        mags.append(np.linalg.norm(s))
        # cancellation: from far away the loop sum is far below one segment's field
        one = O.seg_stress(MAT, net.xyz[0], net.xyz[1], net.burgers[0], r * d)
        if r >= 300 * Rl:
            assert np.linalg.norm(s) < 0.2 * np.linalg.norm(one)
    slope = np.polyfit(np.log(rs), np.log(mags), 1)[0]
    assert abs(slope + 3.0) < 0.01


def test_closed_loop_field_is_in_equilibrium():
    """div sigma = 0 for a closed loop (the spread-core field is an eigenstrain field)."""
    rng = np.random.default_rng(9)
    e1 = np.array([1.0, 0, 0])
    e2 = np.array([0, 0.6, 0.8])
    net = _polygon(12, 30 * A, np.zeros(3), e1, e2, [0.3 * BB, 0.5 * BB, -0.2 * BB])
    for _ in range(4):
        p = rng.normal(size=3) * 25 * A
        h = 1e-3 * A
        div = np.zeros(3)
        for j in range(3):
            dp = np.zeros(3)
            dp[j] = h
            sp = full(O.stress_at(MAT, net, (p + dp)[None, :])[0])
            sm = full(O.stress_at(MAT, net, (p - dp)[None, :])[0])
            div += (sp[:, j] - sm[:, j]) / (2 * h)
        s0 = full(O.stress_at(MAT, net, p[None, :])[0])
        # compare with the size of a single partial derivative of sigma
        scale = np.max(np.abs(s0)) / np.linalg.norm(p)
        assert np.max(np.abs(div)) < 1e-6 * scale
    # an open segment alone is not in equilibrium, so the check has teeth
    p = np.array([3.0, 7.0, -2.0]) * A
    h = 1e-3 * A
    div = np.zeros(3)
    for j in range(3):
        dp = np.zeros(3)
        dp[j] = h
        sp = full(O.seg_stress(MAT, net.xyz[0], net.xyz[1], net.burgers[0], p + dp))
        sm = full(O.seg_stress(MAT, net.xyz[0], net.xyz[1], net.burgers[0], p - dp))
        div += (sp[:, j] - sm[:, j]) / (2 * h)
    s0 = full(O.seg_stress(MAT, net.xyz[0], net.xyz[1], net.burgers[0], p))
    assert np.max(np.abs(div)) > 1e-3 * np.max(np.abs(s0)) / np.linalg.norm(p)


# ----------------------------------------------------------------- P9
def test_parallel_like_screws_repel():
    half = 0.5e9 * A
    dsep = 50 * A
    mat0 = (MU, NU, BB, 1e-6 * A, 1e-4)
    x1, x2 = np.array([0, 0, -half]), np.array([0, 0, half])
    bv = np.array([0, 0, BB])
    s = full(O.seg_stress(mat0, x1, x2, bv, [dsep, 0, 0]))
    f = np.cross(s @ bv, np.array([0, 0, 1.0]))  # (sigma b) x t on the second screw
    assert f[0] > 0 and abs(f[1]) < 1e-12 * f[0] and abs(f[2]) < 1e-12 * f[0]
    assert abs(f[0] / (MU * BB * BB / (2 * math.pi * dsep)) - 1) < 1e-12
    # opposite sign attracts
    s = full(O.seg_stress(mat0, x2, x1, bv, [dsep, 0, 0]))
    f = np.cross(s @ bv, np.array([0, 0, 1.0]))
    assert f[0] < 0


# ---------------------------------------------------------- P10-P14
def _shear_tensor(bhat, n, tau):
    return tau * (np.outer(bhat, n) + np.outer(n, bhat))


def test_power_identity_uniform_stress():
    rng = np.random.default_rng(10)
    net = W.loop_ensemble(11, 6, 0.5e-6, np.zeros(6))
    sig = rng.uniform(-100e6, 100e6, size=6)
    net.sig_app = sig
    F = O.nodal_forces(MAT, net, interactions=False)
    v = O.velocities(MAT, net, F)
    Lp, _ = O.lp_rho(net, v)
    lhs = net.volume * np.sum(full(sig) * Lp)
    rhs = np.sum(F * v)
    assert abs(lhs - rhs) <= 1e-13 * abs(rhs)
    assert rhs > 0  # drag dissipates


@pytest.mark.parametrize("N", [8, 32, 256])
def test_polygon_loop_lp_closed_form(N):
    """Regular N-gon, uniform resolved shear tau, no self stress:
    Lp = cos^2(pi/N) * (1/V) sum_i tau |b|^2 l_i / B  m (x) n   (Eq. 2.9 at N -> inf)."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_magnitudes.json")))
    tau = gold["free_segment_Lp"]["applied_shear_pa"]
    Bd = gold["material_table"]["drag_B_pa_s"]
    mat = (MU, NU, BB, A, Bd)
    bh, nh = W.fcc_slip_systems()
    k = 4
    m, n = bh[k], nh[k]
    for sense in (1.0, -1.0):
        net = _polygon(N, 500 * A, np.array([1.0, 2.0, 3.0]) * 1e-7, m, np.cross(n, m), BB * m, sense)
        net.volume = 1e-18
        S = _shear_tensor(m, n, tau)
        net.sig_app = voigt(S)
        F = O.nodal_forces(mat, net, interactions=False)
        v = O.velocities(mat, net, F)
        Lp, rho = O.lp_rho(net, v)
        seg = np.roll(net.xyz, -1, axis=0) - net.xyz
        ltot = np.sum(np.linalg.norm(seg, axis=1))
        eq29 = tau * BB ** 2 * ltot / (Bd * net.volume) * np.outer(m, n)
        assert rel(Lp, math.cos(math.pi / N) ** 2 * eq29) < 1e-12
        # node speed tau|b|/B cos(pi/N); per-length Lp magnitude -> tau/B (Sec. 2.2)
        assert rel(np.linalg.norm(v, axis=1), np.full(N, tau * BB / Bd * math.cos(math.pi / N))) < 1e-12
    per_length = np.linalg.norm(Lp) * net.volume / (ltot * BB ** 2)
    assert abs(per_length / (tau / Bd) - math.cos(math.pi / N) ** 2) < 1e-12
    assert 0.5 * gold["free_segment_Lp"]["order_of_magnitude_per_s"] < tau / Bd < 5 * gold["free_segment_Lp"]["order_of_magnitude_per_s"]


def test_lp_equals_swept_area_rate():
    """(V/|b|) Lp:(b_hat (x) n) = -dA/dt for a planar loop with any in-plane velocities."""
    rng = np.random.default_rng(12)
    bh, nh = W.fcc_slip_systems()
    m, n = bh[7], nh[7]
    e2 = np.cross(n, m)
    for sense in (1.0, -1.0):
        net = _polygon(20, 300 * A, np.zeros(3), m, e2, BB * m, sense)
        net.xyz = net.xyz + rng.normal(size=net.xyz.shape) * 20 * A * (np.outer(np.ones(20), m) + 0.5 * np.outer(np.ones(20), e2))
        vin = rng.normal(size=(20, 2))
        v = vin[:, :1] * m + vin[:, 1:] * e2

        def area(x):
            c = np.cross(x, np.roll(x, -1, axis=0)) @ n
            return 0.5 * np.sum(c)

        eps = 1e-3 * A
        dA = (area(net.xyz + eps * v) - area(net.xyz - eps * v)) / (2 * eps)
        Lp, _ = O.lp_rho(net, v)
        lhs = net.volume / BB * (m @ Lp @ n)
        assert abs(lhs + dA) <= 1e-9 * abs(dA)


def test_glide_invariant_and_euler_step():
    net = W.small_loop_network()
    net = W.Network(net.xyz[:32 * 4].copy(), net.loop_off[:5].copy(), net.burgers[:4].copy(),
                    net.normal[:4].copy(), net.pinned[:128].copy(), net.volume, net.sig_app)
    dt = 1e-12
    out = O.burst(MAT, net, 3, dt, trace=True)
    disp = out["xyz"] - net.xyz
    nrm = np.repeat(net.normal, 32, axis=0)
    assert np.max(np.abs(np.sum(disp * nrm, axis=1))) < 1e-12 * np.max(np.abs(disp))
    assert np.max(np.abs(disp)) > 0
    # one Euler step: x1 = x0 + v0 dt
    F = O.nodal_forces(MAT, net)
    v = O.velocities(MAT, net, F)
    one = O.burst(MAT, net, 1, dt)
    assert rel(one["xyz"] - net.xyz, v * dt) < 1e-12
    # running average of Eq. 2.5 with fixed dt is the mean of the samples
    assert rel(out["Lp_avg"], out["Lp_trace"].mean(axis=0)) < 1e-14
    assert abs(out["rho_avg"] - out["rho_trace"].mean()) < 1e-14 * out["rho_avg"]


def test_mobility_projection_and_pins():
    net = W.loop_ensemble(13, 3, 0.5e-6, W.uniaxial_stress(80e6))
    net.pinned[5:9] = 1
    F = O.nodal_forces(MAT, net)
    v = O.velocities(MAT, net, F)
    nrm = np.repeat(net.normal, 32, axis=0)
    assert np.max(np.abs(np.sum(v * nrm, axis=1))) < 1e-14 * np.max(np.abs(v))
    assert np.all(v[5:9] == 0)
    # explicit form at one node: v = (I - n n) F / (B M)
    a = 40
    xp, xa, xn = net.xyz[39], net.xyz[40], net.xyz[41]
    M = 0.5 * (np.linalg.norm(xa - xp) + np.linalg.norm(xn - xa))
    n = net.normal[1]
    exp = (F[a] - n * (n @ F[a])) / (MAT[4] * M)
    assert rel(v[a], exp) < 1e-14


def test_rho_of_regular_polygons():
    net = W.loop_ensemble(14, 5, 1e-6, np.zeros(6), nodes_per_loop=24)
    _, rho = O.lp_rho(net, np.zeros_like(net.xyz))
    radii = np.array([np.linalg.norm(net.xyz[24 * k] - net.xyz[24 * k:24 * k + 24].mean(axis=0)) for k in range(5)])
    exp = np.sum(24 * 2 * radii * math.sin(math.pi / 24)) / net.volume
    assert abs(rho / exp - 1) < 1e-13


def test_nodal_force_shape_functions_against_fine_quadrature():
    """F_a = int N_a(s) f(s) ds with N_start = 1 - xi, N_end = xi.

    A small target loop with a tiny Burgers vector sits in the smooth field of
    a source loop 100a away, so its own field (order |b_t|^2) is negligible and
    the 4-point rule is near exact.  The field changes by ~10% along a target
    segment, so swapping the shape functions would be caught."""
    bh, nh = W.fcc_slip_systems()
    tgt = _polygon(16, 30 * A, np.zeros(3), bh[0], np.cross(nh[0], bh[0]), 1e-6 * BB * bh[0])
    src = _polygon(16, 50 * A, np.array([100.0, 20.0, -30.0]) * A, bh[5], np.cross(nh[5], bh[5]), BB * bh[5])
    net = W.Network(np.vstack([tgt.xyz, src.xyz]), np.array([0, 16, 32], np.int64),
                    np.vstack([tgt.burgers, src.burgers]), np.vstack([tgt.normal, src.normal]),
                    np.zeros(32, np.uint8), 1e-18, np.array([0, 0, 20e6, 0, 0, 0.0]))
    F = O.nodal_forces(MAT, net)
    bv = net.burgers[0]
    z, w = np.polynomial.legendre.leggauss(64)
    s = 0.5 * (1 + z)
    for a in (0, 5, 11):
        nxt, prv = (a + 1) % 16, (a - 1) % 16
        tot = np.zeros(3)
        for (i, j, start) in ((a, nxt, True), (prv, a, False)):
            xa, xb = net.xyz[i], net.xyz[j]
            L = np.linalg.norm(xb - xa)
            t = (xb - xa) / L
            pts = xa[None, :] + s[:, None] * (xb - xa)[None, :]
            sig = O.stress_at(MAT, net, pts)
            f = np.array([np.cross(full(sv) @ bv, t) for sv in sig])
            Nfun = (1 - s) if start else s
            tot += L * np.sum((0.5 * w * Nfun)[:, None] * f, axis=0)
        assert rel(F[a], tot) < 2e-5
    sub = O.nodal_forces_subset(MAT, net, [0, 5, 11, 31])
    assert rel(sub, F[[0, 5, 11, 31]]) < 1e-15


# ----------------------------------------------------------------- P16
def test_fcc_schmid_factors_under_001_tension():
    bh, nh = W.fcc_slip_systems()
    assert np.allclose(np.abs(np.sum(bh * nh, axis=1)), 0)
    assert np.allclose(np.linalg.norm(bh, axis=1), 1) and np.allclose(np.linalg.norm(nh, axis=1), 1)
    sig = np.zeros((3, 3))
    sig[2, 2] = 1.0
    fs = np.array([b @ (sig @ n) / np.linalg.norm(sig) for b, n in zip(bh, nh)])
    assert np.sum(np.isclose(np.abs(fs), 1 / math.sqrt(6))) == 8
    assert np.sum(np.isclose(fs, 0)) == 4


def test_c2g_matrices_orthogonal():
    gold = json.load(open(os.path.join(GOLDEN, "paper_magnitudes.json")))
    rows = gold["c2g_tension"]["rows"]
    A_ = np.array([[eval(e, {"sqrt": math.sqrt}) for e in r] for r in rows])
    assert np.allclose(A_ @ A_.T, np.eye(3), atol=1e-15)
    assert abs(np.linalg.det(A_) - 1) < 1e-15


# ------------------------------------------------------ polar velocity
def test_polar_velocity_of_a_rigid_translation():
    """Every node moving with one velocity u: vbar_s = u on every segment, so
    V = (A / |B|) sum_s l_s u = A rho u (Eq. 2.11)."""
    net = W.loop_ensemble(15, 4, 0.5e-6, np.zeros(6), nodes_per_loop=19)
    u = np.array([3.0, -1.0, 2.0])
    core = 2.0 * BB ** 2
    V = O.polar_velocity(net, np.tile(u, (net.n_nodes, 1)), core)
    seg = np.concatenate([np.roll(net.xyz[a:b], -1, axis=0) - net.xyz[a:b]
                          for a, b in zip(net.loop_off[:-1], net.loop_off[1:])])
    rho = np.sum(np.linalg.norm(seg, axis=1)) / net.volume
    assert rel(V, core * rho * u) < 1e-13


@pytest.mark.parametrize("sense", [1.0, -1.0])
def test_polar_velocity_of_a_half_pinned_polygon(sense):
    """Regular N-gon under uniform resolved shear tau, no self stress, the
    nodes on one side of a diameter pinned.  A free node moves at
    tau |b| cos(pi/N) / B along its radial unit vector r_a (outwards when the
    loop expands), a pinned one not, and every segment has length
    l = 2 R sin(pi/N), so
      V = (A / |B|) sum_s l vbar_s = (A l / |B|) sum_free v_a
        = s (A l / |B|) (tau |b| cos(pi/N) / B) sum_free r_a,
    with s = +1 when the loop grows: by the swept-area identity pinned above
    the signed area A_n (orientation from the node order about n) changes at
    -(|B| / |b|) Lp:(b_hat (x) n), and the loop grows when that rate has the
    sign of A_n."""
    N, R = 32, 400 * A
    tau, Bd = 20e6, 1e-4
    mat = (MU, NU, BB, A, Bd)
    bh, nh = W.fcc_slip_systems()
    m, n = bh[2], nh[2]
    e2 = np.cross(n, m)
    centre = np.array([2.0, -1.0, 0.5]) * 1e-7
    net = _polygon(N, R, centre, m, e2, BB * m, sense)
    net.sig_app = voigt(_shear_tensor(m, n, tau))
    rhat = (net.xyz - centre) / R
    free = rhat @ m > 0.01
    net.pinned = (~free).astype(np.uint8)
    F = O.nodal_forces(mat, net, interactions=False)
    v = O.velocities(mat, net, F)
    Lp, _ = O.lp_rho(net, v)
    signed_area = 0.5 * np.sum(np.cross(net.xyz - centre, np.roll(net.xyz, -1, axis=0) - centre) @ n)
    s = -np.sign(m @ Lp @ n) * np.sign(signed_area)
    core = BB ** 2
    V = O.polar_velocity(net, v, core)
    l = 2 * R * math.sin(math.pi / N)
    exp = s * core * l / net.volume * tau * BB * math.cos(math.pi / N) / Bd * rhat[free].sum(axis=0)
    assert rel(V, exp) < 1e-12
    assert abs(V @ n) <= 1e-12 * np.linalg.norm(V)  # glide: V lies in the slip plane
    # a 1-step burst averages the step-start state: its R^V is this V
    one = O.burst(mat, net, 1, 1e-12, interactions=False, core_area=core)
    assert rel(one["V_avg"], V) < 1e-14


# ------------------------------------------------- consistent mass mobility
def _irregular_loop(n, rng, pinned_every=0):
    """A planar loop of n nodes at uneven angles and radii, in the (111) glide plane."""
    bh, nh = W.fcc_slip_systems()
    m, nn = bh[0], nh[0]
    e2 = np.cross(nn, m)
    phi = np.sort(rng.uniform(0, 2 * math.pi, n))
    rad = 300 * A * (1 + 0.3 * rng.uniform(-1, 1, n))
    xyz = rad[:, None] * (np.cos(phi)[:, None] * m + np.sin(phi)[:, None] * e2)
    pin = np.zeros(n, np.uint8)
    if pinned_every:
        pin[::pinned_every] = 1
    return W.Network(xyz, np.array([0, n], np.int64), (BB * m)[None, :], nn[None, :], pin, 1e-18, np.zeros(6)), nn


def _galerkin_load(net, g, B):
    """F_a = B int N_a g dl for the piecewise-linear field g (nodal values),
    integrated segment by segment with the 2-point Gauss rule (exact here,
    the integrand being quadratic) -- independent of any mass matrix."""
    x = net.xyz
    n = x.shape[0]
    F = np.zeros_like(g)
    xi = np.array([0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0)])
    for i in range(n):
        j = (i + 1) % n
        L = np.linalg.norm(x[j] - x[i])
        for q in xi:
            gq = (1 - q) * g[i] + q * g[j]
            F[i] += B * L * 0.5 * (1 - q) * gq
            F[j] += B * L * 0.5 * q * gq
    return F


@pytest.mark.parametrize("pinned_every", [0, 5])
def test_consistent_mobility_returns_a_piecewise_linear_velocity(pinned_every):
    """Eq. 2.1's weak form with linear shape functions: when the nodal loads
    are the Galerkin loads of a piecewise-linear in-plane velocity field g
    (zero at pinned nodes), the consistent mobility returns g exactly and
    the lumped one does not."""
    rng = np.random.default_rng(41 + pinned_every)
    net, nn = _irregular_loop(27, rng, pinned_every)
    g = rng.normal(size=(27, 3))
    g -= np.outer(g @ nn, nn)
    g[net.pinned.astype(bool)] = 0.0
    F = _galerkin_load(net, g, MAT[4])
    v = O.velocities(MAT, net, F, consistent=True)
    assert rel(v, g) < 1e-12
    assert np.all(v[net.pinned.astype(bool)] == 0.0)
    assert rel(O.velocities(MAT, net, F), g) > 1e-3


def test_consistent_and_lumped_mobility_agree_under_a_uniform_load():
    """A uniform load per length on a free loop: the Galerkin loads are
    B g (L_prev + L_next)/2, and both mobilities return g at every node."""
    rng = np.random.default_rng(44)
    net, nn = _irregular_loop(31, rng)
    g = np.cross(nn, [0.3, -0.2, 0.9])
    g = np.tile(g, (31, 1))
    F = _galerkin_load(net, g, MAT[4])
    assert rel(O.velocities(MAT, net, F, consistent=True), g) < 1e-12
    assert rel(O.velocities(MAT, net, F), g) < 1e-12


def test_consistent_mobility_of_a_regular_polygon_in_uniform_shear():
    """Regular N-gon under uniform resolved shear tau, no self stress: the
    nodal forces are radial, tau |b| l cos(pi/N) r_a with l the side; the
    consistent mass matrix maps a radial field of one speed w to
    B w l (2 + cos(2 pi/N))/3 r_a, so every node moves radially at
    tau |b| cos(pi/N) / (B (2 + cos(2 pi/N))/3) (the lumped speed
    tau |b| cos(pi/N)/B over (2 + cos(2 pi/N))/3)."""
    N, R, tau, Bd = 24, 500 * A, 30e6, 1e-4
    mat = (MU, NU, BB, A, Bd)
    bh, nh = W.fcc_slip_systems()
    m, n = bh[5], nh[5]
    e2 = np.cross(n, m)
    net = _polygon(N, R, np.zeros(3), m, e2, BB * m)
    net.sig_app = voigt(_shear_tensor(m, n, tau))
    F = O.nodal_forces(mat, net, interactions=False)
    v = O.velocities(mat, net, F, consistent=True)
    rhat = net.xyz / R
    speed = np.sum(v * rhat, axis=1)
    w = tau * BB * math.cos(math.pi / N) / (Bd * (2 + math.cos(2 * math.pi / N)) / 3)
    assert np.allclose(np.abs(speed), w, rtol=1e-12)
    assert np.all(np.sign(speed) == np.sign(speed[0]))
    assert np.max(np.abs(v - speed[:, None] * rhat)) <= 1e-12 * w  # radial
    vl = O.velocities(mat, net, F)
    assert np.allclose(np.abs(np.sum(vl * rhat, axis=1)), tau * BB * math.cos(math.pi / N) / Bd, rtol=1e-12)


def test_consistent_mass_burst_steps_with_the_consistent_velocities():
    """A loop in uniform shear, self stress off: one Euler step of the
    burst with the consistent mobility moves every node by its Galerkin
    velocity, and three steps keep the nodes in their glide plane."""
    N, R, tau, Bd = 16, 400 * A, 20e6, 1e-4
    mat = (MU, NU, BB, A, Bd)
    bh, nh = W.fcc_slip_systems()
    m, n = bh[1], nh[1]
    net = _polygon(N, R, np.array([1.0, 2.0, -1.0]) * 1e-7, m, np.cross(n, m), BB * m)
    net.sig_app = voigt(_shear_tensor(m, n, tau))
    dt = 5e-13
    out = O.burst(mat, net, 1, dt, interactions=False, consistent_mass=True)
    F = O.nodal_forces(mat, net, interactions=False)
    v = O.velocities(mat, net, F, consistent=True)
    assert rel(out["xyz"], net.xyz + v * dt) < 1e-15
    out3 = O.burst(mat, net, 3, dt, interactions=False, consistent_mass=True)
    assert np.max(np.abs((out3["xyz"] - net.xyz) @ n)) <= 1e-12 * np.max(np.abs(out3["xyz"] - net.xyz))
