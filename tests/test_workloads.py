"""Host-side checks of the seeded input generators (no GPU, no oracle)."""

import numpy as np

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
