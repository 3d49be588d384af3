"""The learned closure against the method it stands in for (the PTA closure
of Sec. 3: the burst-averaged plastic distortion rate at a material point).

A surrogate is fitted on the GPU, with the library's own tensor-core
training kernels, on closures that the GPU's batched DD bursts produce
(12 000 training and 1200 validation closures of 128 stratified glide loops,
100 mixed-precision steps at dt 5e-13 s, one realisation per input).  It is
then scored on 192 hold-out inputs against the mean of 24 DD realisations
per input, and checked for what it gains over the method without it:

  * the raw relative error (Frobenius over the hold-out set) of its answers,
    averaged over the 48 symmetric images of each input, is at most 3 %;
    the noise floor of the 24-member reference means is reported beside it,
    not subtracted;
  * without the network, a least-squares linear map of the same features
    fitted on the same DD closures errs at least twice as much;
  * it answers at least 1e4 times as many closures per second as the DD
    bursts that labelled it.

The closure sweep (ptadd_closure_sweep) is then run with this surrogate on
hold-out inputs inside its trust region and two inputs far outside it: the
inside points must get the surrogate's answer bit for bit, the outside ones
the mean of DD bursts on the library's own seeded realisations, recomputed
here through the batch API.
"""

import time

import numpy as np
import pytest

from paper_2005_02498_gb300 import ptadd
from paper_2005_02498_gb300 import surrogate as SU
from paper_2005_02498_gb300 import workloads as W

pytestmark = pytest.mark.gpu
MAT = W.Material().as_tuple()
N_TRAIN, N_VAL, N_EVAL, MEMBERS = 12000, 1200, 192, 24
STEPS, DT, LOOPS = 100, 5e-13, 128
STEP = 0x9E3779B97F4A7C15
MASK = (1 << 64) - 1


def linear_baseline(Xtr, Ytr, Xev):
    """Least-squares affine map of (sigma / 200 MPa, log10(rho + 1e10)) to the rates."""
    def design(X):
        return np.hstack([X[:, :6] / 200e6, np.log10(X[:, 6:] + 1e10), np.ones((X.shape[0], 1))])
    coef, *_ = np.linalg.lstsq(design(Xtr), Ytr, rcond=None)
    return design(Xev) @ coef


def test_surrogate_fitted_on_dd_closures_meets_the_rate_bar_and_beats_dd():
    rng = np.random.default_rng(2204)
    X = SU.feature_points(rng, N_TRAIN + N_VAL + N_EVAL)
    Xtr, Xva, Xho = X[:N_TRAIN], X[N_TRAIN:N_TRAIN + N_VAL], X[N_TRAIN + N_VAL:]
    singles = np.zeros((N_EVAL, MEMBERS, 6))
    with ptadd.Context(MAT, ptadd.PTADD_MIXED, 0) as c:
        Y, t_lab, _ = SU.generate(c, X[:N_TRAIN + N_VAL], 1, 2205, STEPS, DT, LOOPS)
        dd_cps = (N_TRAIN + N_VAL) / t_lab
        Ytr, Yva = Y[:N_TRAIN], Y[N_TRAIN:]
        Yho, _, _ = SU.generate(c, Xho, MEMBERS, 2206, STEPS, DT, LOOPS, singles=singles)
        val_err, curve, _ = SU.fit_early_stopping(c, Xtr, Ytr, Xva, Yva, epochs=40, seed=2207)
        pred, inr = SU.predict_symmetrised(c, Xho)
        plain, _ = c.surrogate_predict(Xho)
        big = np.tile(Xho, (2731, 1))[:1 << 18]
        c.surrogate_predict(big[:1024])
        t0 = time.perf_counter()
        c.surrogate_predict(big)
        sur_cps = big.shape[0] / (time.perf_counter() - t0)

        # the sweep with this surrogate: hold-out inputs inside the trust
        # region and two far outside it (stresses of several GPa)
        inside = np.flatnonzero(inr)[:6]
        sig = np.vstack([Xho[inside, :6], [[5e9, 0, 0, 0, 0, 0], [0, -4e9, 0, 0, 0, 1e9]]])
        rho = np.vstack([Xho[inside, 6:], Xho[:2, 6:]])
        ens, segments, seed = 2, 32 * LOOPS, 4242
        sur_ans, sur_in = c.surrogate_predict(np.hstack([sig, rho]))
        out, used = c.closure_sweep(sig, rho, ens, segments, STEPS, DT, seed)
        miss = np.flatnonzero(~sur_in)
        nets = []
        for m, pt in enumerate(miss):
            for k in range(ens):
                q = m * ens + k
                xyz, b, nv, pin, vol = ptadd.closure_realisation(MAT, (seed ^ (q * STEP)) & MASK, rho[pt], LOOPS)
                nets.append(W.Network(xyz, np.arange(LOOPS + 1, dtype=np.int64) * 32, b, nv, pin, vol,
                                      sig[pt].copy()))
        c.batch_set(W.batch_from_networks(nets))
        Lp, _ = c.batch_advance(STEPS, DT)
    err = SU.relerr(pred, Yho)
    noise = float(np.linalg.norm(singles - Yho[:, None, :]) / np.sqrt(MEMBERS - 1) / np.linalg.norm(Yho)
                  / np.sqrt(MEMBERS))
    lin_err = SU.relerr(linear_baseline(Xtr, Ytr, Xho), Yho)
    per = np.linalg.norm(pred - Yho, axis=1)
    worst = np.argsort(per)[-3:]
    print("surrogate vs %d-member DD means: %.4f (plain %.4f, validation %.4f), reference noise floor %.4f, "
          "linear baseline %.4f, in region %.3f, surrogate %.3g closures/s vs DD %.3g closures/s; largest "
          "errors (share of the squared total, relative): %s"
          % (MEMBERS, err, SU.relerr(plain, Yho), val_err, noise, lin_err, inr.mean(), sur_cps, dd_cps,
             [(round(float(per[i] ** 2 / np.sum(per ** 2)), 3), round(float(per[i] / np.linalg.norm(Yho[i])), 3))
              for i in worst]))
    assert err <= 0.03
    assert err <= 0.5 * lin_err
    assert sur_cps >= 1e4 * dd_cps
    # sweep: surrogate inside, DD outside
    assert sur_in[:len(inside)].all() and not sur_in[len(inside):].any()
    assert np.array_equal(used, ~sur_in)
    assert np.array_equal(out[sur_in], sur_ans[sur_in])
    want = SU.sym_voigt(Lp).reshape(len(miss), ens, 6).mean(1)
    assert np.all(np.isfinite(out)) and np.linalg.norm(want) > 0
    assert np.max(np.abs(out[miss] - want)) <= 1e-9 * np.max(np.abs(want))
