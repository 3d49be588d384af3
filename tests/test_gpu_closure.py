"""GPU test of the closure sweep (ptadd_closure_sweep): points inside the
surrogate's trust region get the surrogate's answer, the others the mean of
an ensemble of DD bursts on realisations from ptadd_closure_realisation.
The fallback answers are recomputed here from the same seeded realisations
through the batch API."""

import numpy as np
import pytest

from paper_2005_02498_gb300 import ptadd
from paper_2005_02498_gb300 import workloads as W

pytestmark = pytest.mark.gpu
MAT = W.Material().as_tuple()
STEP = 0x9E3779B97F4A7C15
MASK = (1 << 64) - 1


def sym_voigt(Lp):
    S = 0.5 * (Lp + np.transpose(Lp, (0, 2, 1)))
    return np.stack([S[:, 0, 0], S[:, 1, 1], S[:, 2, 2], S[:, 1, 2], S[:, 0, 2], S[:, 0, 1]], axis=1)


def test_closure_sweep_surrogate_inside_dd_outside():
    rng = np.random.default_rng(31)
    n = 2048
    sig = rng.uniform(-200e6, 200e6, size=(n, 6))
    rho = 10 ** rng.uniform(11.5, 12.5, size=(n, 24))
    lp = np.tanh(sig / 1e8) * (np.log10(rho[:, :6]) - 10.0) * 50.0
    pts_sig = np.vstack([sig[:12], np.array([[5e9, 0, 0, 0, 0, 0], [0, -4e9, 0, 0, 0, 1e9]])])
    pts_rho = np.vstack([rho[:12], rho[12:14]])
    ens, segments, steps, dt, seed = 3, 256, 8, 5e-13, 12345
    with ptadd.Context(MAT, ptadd.PTADD_FP64, 0) as c:
        c.surrogate_fit(np.hstack([sig, rho]), lp, epochs=10, batch=256, lr=2e-3, seed=3)
        sur, inr = c.surrogate_predict(np.hstack([pts_sig, pts_rho]))
        out, used = c.closure_sweep(pts_sig, pts_rho, ens, segments, steps, dt, seed)
        out2, _ = c.closure_sweep(pts_sig, pts_rho, ens, segments, steps, dt, seed)
        assert inr[:12].sum() >= 8 and not inr[12:].any()
        assert np.array_equal(used, ~inr)
        assert np.array_equal(out[inr], sur[inr])
        assert np.array_equal(out, out2)  # reproducible
        # fallback points: the same realisations through the batch API
        miss = np.flatnonzero(~inr)
        nets = []
        for m, pt in enumerate(miss):
            for k in range(ens):
                q = m * ens + k
                xyz, b, nv, pin, vol = ptadd.closure_realisation(MAT, (seed ^ (q * STEP)) & MASK, pts_rho[pt],
                                                                 segments // 32)
                nets.append(W.Network(xyz, np.arange(segments // 32 + 1, dtype=np.int64) * 32, b, nv, pin, vol,
                                      pts_sig[pt].copy()))
        c.batch_set(W.batch_from_networks(nets))
        Lp, _ = c.batch_advance(steps, dt)
    want = sym_voigt(Lp).reshape(len(miss), ens, 6).mean(1)
    assert np.all(np.isfinite(out))
    assert np.max(np.abs(out[miss] - want)) <= 1e-9 * np.max(np.abs(want))
    assert np.linalg.norm(want) > 0


def test_closure_sweep_needs_a_fitted_surrogate_and_valid_sizes():
    with ptadd.Context(MAT, ptadd.PTADD_MIXED, 0) as c:
        with pytest.raises(ptadd.PtaddError):
            c.closure_sweep(np.zeros((1, 6)), np.ones((1, 24)) * 1e12, 2, 256, 4, 5e-13, 1)
        with pytest.raises(ptadd.PtaddError):
            c.closure_sweep(np.zeros((1, 6)), np.ones((1, 24)) * 1e12, 2, 100, 4, 5e-13, 1)  # not a multiple of 32
