"""Host-side checks of the seeded input generators (no GPU, no oracle)."""

import math

import numpy as np
import pytest

from paper_2005_02498_gb300 import workloads as W


def _loop_lengths(net):
    x = net.xyz.reshape(-1, 32, 3)
    return np.linalg.norm(np.roll(x, -1, axis=1) - x, axis=2).sum(axis=1)


def test_stratified_realisation_matches_the_requested_densities():
    rng = np.random.default_rng(3)
    for trial in range(20):
        rm = rng.dirichlet(np.ones(12)) * 10 ** rng.uniform(12.3, 13.3)
        rs = rng.dirichlet(np.ones(12)) * 10 ** rng.uniform(12.3, 13.3)
        n_loops = int(rng.choice([32, 48, 128]))
        net = W.realisation_for_densities(np.random.default_rng(trial), np.zeros(6), rm, rs, n_loops=n_loops,
                                          stratified=True)
        assert net.n_loops == n_loops
        L = _loop_lengths(net)
        # the total density is exact
        assert abs(L.sum() / net.volume / (rm.sum() + rs.sum()) - 1) < 1e-12
        # class counts: floor or ceil of the expected count, mobile = unpinned
        dens = np.concatenate([rm, rs])
        expect = n_loops * dens / dens.sum()
        sys_idx = W.slip_system_index(net.burgers, net.normal)
        pinned = net.pinned.reshape(-1, 32)[:, 0].astype(bool)
        cls = sys_idx + 12 * pinned
        counts = np.bincount(cls, minlength=24)
        assert np.all(counts >= np.floor(expect)) and np.all(counts <= np.ceil(expect))
        # radii inside the range; line senses balanced within each class
        r = L / (2 * 32 * np.sin(np.pi / 32))
        assert np.all(r >= 0.05e-6 * (1 - 1e-12)) and np.all(r <= 0.2e-6 * (1 + 1e-12))
        x = net.xyz.reshape(-1, 32, 3)
        sense = np.sign(np.einsum("ij,ij->i", np.cross(x[:, 0] - x.mean(1), x[:, 1] - x.mean(1)), net.normal))
        for c in range(24):
            s = sense[cls == c]
            assert abs(s.sum()) <= 1


def test_unstratified_realisation_is_unchanged_by_the_option():
    rm = np.full(12, 5e11)
    rs = np.full(12, 2e11)
    a = W.realisation_for_densities(np.random.default_rng(9), np.zeros(6), rm, rs, n_loops=32)
    b = W.realisation_for_densities(np.random.default_rng(9), np.zeros(6), rm, rs, n_loops=32, stratified=False)
    assert np.array_equal(a.xyz, b.xyz) and a.volume == b.volume


def test_cubic_rotations_permute_the_slip_systems():
    from paper_2005_02498_gb300.surrogate import _voigt_rotate, cubic_rotations
    rots, perms = cubic_rotations()
    assert len(rots) == 24
    bh, nh = W.fcc_slip_systems()
    rng = np.random.default_rng(4)
    sig = rng.normal(size=(5, 6))
    for Q, perm in zip(rots, perms):
        assert sorted(perm) == list(range(12))
        assert np.allclose(np.abs(np.einsum("sj,tj->st", bh @ Q.T, bh)[np.arange(12), perm]), 1.0)
        # resolved shear stresses are permuted (up to sign): tau_perm[s](Q s Q^T) = +-tau_s(s)
        rs = _voigt_rotate(sig, Q)
        for v, w in zip(sig, rs):
            S = np.array([[v[0], v[5], v[4]], [v[5], v[1], v[3]], [v[4], v[3], v[2]]])
            T = np.array([[w[0], w[5], w[4]], [w[5], w[1], w[3]], [w[4], w[3], w[2]]])
            tau = np.einsum("si,ij,sj->s", bh, S, nh)
            tau_r = np.einsum("si,ij,sj->s", bh, T, nh)
            assert np.allclose(np.abs(tau_r[perm]), np.abs(tau))


def test_oracle_burst_is_equivariant_under_cube_rotations():
    """The premise of the surrogate's data augmentation: a rotated
    realisation under the rotated stress has the rotated averaged rate."""
    import oracle as O
    from paper_2005_02498_gb300.surrogate import cubic_rotations

    mat = W.Material().as_tuple()
    net = W.small_loop_network()
    net.sig_app = np.array([30e6, -20e6, 50e6, 10e6, -15e6, 25e6])
    ref = O.burst(mat, net, 3, 5e-13)
    rots, _ = cubic_rotations()
    for Q in rots[[1, 7, 13, 22]]:
        r = net.copy()
        r.xyz = net.xyz @ Q.T
        r.burgers = net.burgers @ Q.T
        r.normal = net.normal @ Q.T
        s = net.sig_app
        S = np.array([[s[0], s[5], s[4]], [s[5], s[1], s[3]], [s[4], s[3], s[2]]])
        T = Q @ S @ Q.T
        r.sig_app = np.array([T[0, 0], T[1, 1], T[2, 2], T[1, 2], T[0, 2], T[0, 1]])
        got = O.burst(mat, r, 3, 5e-13)
        want = Q @ ref["Lp_avg"] @ Q.T
        assert np.linalg.norm(got["Lp_avg"] - want) <= 1e-9 * np.linalg.norm(want)
        assert abs(got["rho_avg"] / ref["rho_avg"] - 1) < 1e-12


def test_oracle_burst_is_odd_under_stress_and_burgers_flip():
    """The premise of the sign symmetry: negating the applied stress and
    every Burgers vector leaves the motion unchanged and negates the averaged
    rate (the balanced line senses make a Burgers flip a symmetry of the
    realisations)."""
    import oracle as O

    mat = W.Material().as_tuple()
    net = W.small_loop_network()
    net.sig_app = np.array([30e6, -20e6, 50e6, 10e6, -15e6, 25e6])
    ref = O.burst(mat, net, 3, 5e-13)
    f = net.copy()
    f.burgers = -net.burgers
    f.sig_app = -net.sig_app
    got = O.burst(mat, f, 3, 5e-13)
    assert np.linalg.norm(got["Lp_avg"] + ref["Lp_avg"]) <= 1e-12 * np.linalg.norm(ref["Lp_avg"])
    assert np.array_equal(got["xyz"], ref["xyz"])


def test_symmetric_images_map_back_to_their_source():
    from paper_2005_02498_gb300.surrogate import (closure_symmetries, cubic_images, symmetrised_answers,
                                                  symmetrised_inputs)
    rng = np.random.default_rng(6)
    X = np.hstack([rng.uniform(-2e8, 2e8, size=(7, 6)), 10 ** rng.uniform(12, 13, size=(7, 24))])
    Y = rng.normal(size=(7, 6))
    xs, ys = cubic_images(X, Y)
    assert len(closure_symmetries()) == 48 and xs.shape == (48 * 7, 30)
    assert np.array_equal(xs, symmetrised_inputs(X))
    back, g0 = symmetrised_answers(ys, 7)
    assert np.allclose(back, Y, rtol=1e-13, atol=1e-13)
    assert np.array_equal(xs[g0 * 7:(g0 + 1) * 7], X)
    # a constant answer (even in the stress) averages to zero: the symmetrised
    # surrogate is odd in sigma
    assert np.allclose(symmetrised_answers(np.ones((48 * 7, 6)), 7)[0], 0.0, atol=1e-15)


def test_closure_input_generators_follow_their_recipes():
    from paper_2005_02498_gb300.closure_sweep import material_points
    from paper_2005_02498_gb300.surrogate import feature_points

    f = feature_points(np.random.default_rng(3), 2000)
    assert f.shape == (2000, 30)
    assert np.all(np.abs(f[:, :6]) <= 200e6)
    for off in (6, 18):
        tot = f[:, off:off + 12].sum(1)
        assert np.all(f[:, off:off + 12] >= 0)
        assert tot.min() >= 2e12 * (1 - 1e-12) and tot.max() <= 2e13 * (1 + 1e-12)
        # log-uniform totals: the median of log10 sits mid-range
        assert abs(np.median(np.log10(tot)) - np.log10(2e12 * np.sqrt(10))) < 0.05

    pts, S, rho = material_points(5, 8)
    assert pts.shape == (512, 3) and S.shape == (512, 6) and rho.shape == (512, 24)
    assert np.allclose(np.max(np.abs(S), axis=0), 200e6)  # every component scaled to 200 MPa
    for off in (0, 12):
        tot = rho[:, off:off + 12].sum(1)
        assert np.all(rho[:, off:off + 12] > 0)
        # rank-uniform log10 totals between the bounds (the training marginals)
        lg = np.sort(np.log10(tot))
        u = (np.arange(lg.size) + 0.5) / lg.size
        assert np.allclose(lg, np.log10(2e12) + u * (np.log10(2e13) - np.log10(2e12)))


def test_native_closure_realisation_follows_the_densities():
    """The library's realisation generator (host code, no GPU): same recipe
    and slip-system order as the Python one, exact total density, class
    counts within one loop, balanced senses, reproducible streams."""
    from paper_2005_02498_gb300 import ptadd
    mat = W.Material().as_tuple()
    rng = np.random.default_rng(12)
    for trial in range(10):
        rho = np.concatenate([rng.dirichlet(np.ones(12)) * 10 ** rng.uniform(12.3, 13.3),
                              rng.dirichlet(np.ones(12)) * 10 ** rng.uniform(12.3, 13.3)])
        n_loops = int(rng.choice([8, 48, 128]))
        xyz, b, nv, pin, vol = ptadd.closure_realisation(mat, 1000 + trial, rho, n_loops)
        net = W.Network(xyz, np.arange(n_loops + 1, dtype=np.int64) * 32, b, nv, pin, vol, np.zeros(6))
        L = _loop_lengths(net)
        assert abs(L.sum() / vol / rho.sum() - 1) < 1e-12
        assert np.allclose(np.linalg.norm(b, axis=1), mat[2]) and np.allclose(np.linalg.norm(nv, axis=1), 1.0)
        assert np.allclose(np.einsum("ij,ij->i", b, nv), 0.0, atol=1e-20)
        cls = W.slip_system_index(b, nv) + 12 * pin.reshape(-1, 32)[:, 0]
        expect = n_loops * rho / rho.sum()
        counts = np.bincount(cls, minlength=24)
        assert np.all(counts >= np.floor(expect)) and np.all(counts <= np.ceil(expect))
        r = L / (2 * 32 * np.sin(np.pi / 32))
        assert np.all(r >= 0.05e-6 * (1 - 1e-12)) and np.all(r <= 0.2e-6 * (1 + 1e-12))
        x = xyz.reshape(-1, 32, 3)
        sense = np.sign(np.einsum("ij,ij->i", np.cross(x[:, 0] - x.mean(1), x[:, 1] - x.mean(1)), nv))
        for c in range(24):
            assert abs(sense[cls == c].sum()) <= 1
    a = ptadd.closure_realisation(mat, 5, rho, 16)
    b2 = ptadd.closure_realisation(mat, 5, rho, 16)
    c = ptadd.closure_realisation(mat, 6, rho, 16)
    assert np.array_equal(a[0], b2[0]) and not np.array_equal(a[0], c[0])


def test_native_closure_realisation_rejects_bad_arguments():
    import pytest
    from paper_2005_02498_gb300 import ptadd
    mat = W.Material().as_tuple()
    good = np.full(24, 1e11)
    bad = good.copy()
    bad[3] = -1.0
    with pytest.raises(ptadd.PtaddError):
        ptadd.closure_realisation(mat, 1, bad, 8)
    bad[3] = np.nan
    with pytest.raises(ptadd.PtaddError):
        ptadd.closure_realisation(mat, 1, bad, 8)
    with pytest.raises(ptadd.PtaddError):
        ptadd.closure_realisation(mat, 1, good, 0)
    with pytest.raises(ptadd.PtaddError):
        ptadd.closure_realisation((48e9, 0.34, 0.0, 2.556e-10, 1e-4), 1, good, 8)  # b = 0


def _golden_matrix(key):
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_magnitudes.json")))
    return np.array([[eval(e, {"sqrt": math.sqrt}) for e in r] for r in gold[key]["rows"]])


def test_c2g_matrices_are_the_papers_and_rotate_the_load_into_the_crystal():
    for dirs, key in ((W.C2G_TENSION, "c2g_tension"), (W.C2G_SHEAR, "c2g_shear")):
        A = W.c2g_matrix(*dirs)
        assert np.allclose(A, _golden_matrix(key), rtol=0, atol=1e-15)
        assert np.allclose(A @ A.T, np.eye(3), atol=1e-15) and abs(np.linalg.det(A) - 1) < 1e-15
    # uniaxial tension along global X: in the crystal, sigma (c1 x c1) with c1 = [0 -1 1]/sqrt(2);
    # the symmetric double slip orientation loads 4 systems on two {111} planes at 1/sqrt(6)
    A = W.c2g_matrix(*W.C2G_TENSION)
    sc = W.global_to_crystal_stress([100e6, 0, 0, 0, 0, 0], A)
    c1 = np.array([0, -1, 1]) / math.sqrt(2)
    full = np.array([[sc[0], sc[5], sc[4]], [sc[5], sc[1], sc[3]], [sc[4], sc[3], sc[2]]])
    assert np.allclose(full, 100e6 * np.outer(c1, c1), rtol=0, atol=1e-7)
    f = W.schmid_factors(sc)
    on = np.isclose(np.abs(f), 1 / math.sqrt(6), rtol=1e-12)
    assert on.sum() == 4 and np.allclose(f[~on], 0, atol=1e-15)
    bh, nh = W.fcc_slip_systems()
    assert len({tuple(np.round(n * math.sqrt(3)).astype(int)) for n in nh[on]}) == 2
    # simple shear in the global XY plane: all of it on the one system with b along X and n along Y
    B = W.c2g_matrix(*W.C2G_SHEAR)
    f = W.schmid_factors(W.global_to_crystal_stress([0, 0, 0, 0, 0, 50e6], B))
    k = int(np.argmax(np.abs(f)))
    assert math.isclose(abs(f[k]), 1 / math.sqrt(2), rel_tol=1e-12)
    assert np.sum(np.abs(f) > 0.7) == 1
    assert abs(abs(bh[k] @ B[0]) - 1) < 1e-12 and abs(abs(nh[k] @ B[1]) - 1) < 1e-12


def test_native_system_densities_closed_form_and_features():
    """ptadd_system_densities: regular 32-gon loops have perimeter
    64 R sin(pi/32) exactly, so each system's density is known in closed
    form; on a closure realisation it equals the generator's features."""
    from paper_2005_02498_gb300 import ptadd
    rng = np.random.default_rng(4)
    systems = np.array([0, 0, 5, 11, 7])
    radius = np.array([50e-9, 80e-9, 60e-9, 100e-9, 70e-9])
    xyz, off, bv, nv = W._loops_with_systems(rng, systems, 1e-6, 32, radius=radius)
    pin = np.repeat(np.array([0, 0, 0, 1, 1], np.uint8), 32)
    net = W.Network(xyz, off, bv, nv, pin, 1e-18, np.zeros(6))
    rho = ptadd.system_densities(net)
    want = np.zeros(24)
    for s_, r_, p_ in zip(systems, radius, [0, 0, 0, 1, 1]):
        want[12 * p_ + s_] += 64 * r_ * math.sin(math.pi / 32) / 1e-18
    assert np.allclose(rho, want, rtol=1e-12, atol=0)
    batch, feats = W.closure_ensemble(9, 3)
    for r in range(3):
        n0, n1 = int(batch.node_off[r]), int(batch.node_off[r + 1])
        l0, l1 = int(batch.loop_base[r]), int(batch.loop_base[r + 1])
        one = W.Network(batch.xyz[n0:n1], batch.loop_off[l0:l1 + 1] - batch.loop_off[l0], batch.burgers[l0:l1],
                        batch.normal[l0:l1], batch.pinned[n0:n1], float(batch.volume[r]), batch.sig6[r])
        assert np.allclose(ptadd.system_densities(one), feats[r, 6:], rtol=1e-12, atol=0)
    bad = net.copy()
    bad.burgers = bad.burgers.copy()
    bad.burgers[0] = [1e-10, 2e-10, 0.0]
    try:
        ptadd.system_densities(bad)
        raise AssertionError("a loop off the FCC systems must be rejected")
    except ptadd.PtaddError:
        pass


def test_junction_microstructure_sessile_cases():
    """Sec. 3.2's two cases share the geometry of a seed: Case 2 sessile
    loops have b in their planes, Case 1 (Lomer-Cottrell-type locks) along a
    <110> direction out of it, b . n = +-(2/sqrt 6)|b|, with |b| and the
    mobile loops unchanged."""
    sig = W.uniaxial_stress(100e6)
    c2 = W.junction_microstructure(5, sig, 1e13, 2e14, n_loops=40, sessile_case=2)
    c1 = W.junction_microstructure(5, sig, 1e13, 2e14, n_loops=40, sessile_case=1)
    for k in ("xyz", "loop_off", "normal", "pinned"):
        assert np.array_equal(getattr(c1, k), getattr(c2, k))
    assert c1.volume == c2.volume
    ses = np.array([bool(np.all(c2.pinned[a:b])) for a, b in zip(c2.loop_off[:-1], c2.loop_off[1:])])
    assert 0 < ses.sum() < ses.size
    mag2 = np.linalg.norm(c2.burgers, axis=1)
    bh2 = c2.burgers / mag2[:, None]
    assert np.all(np.abs(np.sum(bh2 * c2.normal, axis=1)) < 1e-12)  # every loop: b in its plane
    assert np.array_equal(c1.burgers[~ses], c2.burgers[~ses])
    assert np.allclose(np.linalg.norm(c1.burgers, axis=1), mag2, rtol=1e-14)
    bh1 = c1.burgers[ses] / mag2[ses, None]
    assert np.allclose(np.abs(np.sum(bh1 * c1.normal[ses], axis=1)), 2.0 / np.sqrt(6.0), rtol=1e-12)
    # along a <110> direction: two components +-1/sqrt 2, one zero
    assert np.allclose(np.sort(np.abs(bh1), axis=1), [0.0, 1 / np.sqrt(2.0), 1 / np.sqrt(2.0)], atol=1e-12)
    with pytest.raises(ValueError):
        W.junction_microstructure(5, sig, 1e13, 2e14, n_loops=40, sessile_case=3)
