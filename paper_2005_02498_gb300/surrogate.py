"""Surrogate closure: generate DD-labelled samples, train, evaluate, time.

    python -m paper_2005_02498_gb300.surrogate --samples 20000 --epochs 200

A closure input is (sigma, mobile and sessile line density per slip
system); a DD closure at that input is the burst-averaged plastic distortion
rate sym(R^Lp) (Voigt order) of a realisation of `--loops` glide loops drawn
to follow those densities (`workloads.realisation_for_densities`, stratified:
class counts, radii and line senses balanced, total density exact), computed
by batched mixed-precision DD bursts (`--dt`, `--steps`).  Realisations with
the same input differ, so a single closure is noisy: the network is trained
on one realisation per training point (it regresses to the conditional
mean) and scored on `--eval` hold-out points against the mean of
`--members` realisations.  The spread of single realisations around those
means gives the noise floor of that reference, and the model error with the
floor removed is reported beside the raw figure.  Training uses every
labelled sample in its 48 symmetric forms (`cubic_images`: the closure map
is equivariant under the 24 rotations of the cube, which permute the FCC
slip systems, and odd in the stress; see `closure_symmetries`), unless
`--no-augment`.  A subset is relabelled
with plain FP64 DD.  `--save-data` / `--load-data` keep the labelled set, so
training can be repeated without new DD work.
Inference is timed on `--infer` points resampled from the training
features, device-resident, and compared with the DD closures/s of the same
closure definition.  Prints one JSON line.
"""

from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import ptadd
from . import workloads as W


def sym_voigt(Lp):
    """[R,3,3] -> [R,6] sym(Lp) in the order xx, yy, zz, yz, xz, xy."""
    S = 0.5 * (Lp + np.transpose(Lp, (0, 2, 1)))
    return np.stack([S[:, 0, 0], S[:, 1, 1], S[:, 2, 2], S[:, 1, 2], S[:, 0, 2], S[:, 0, 1]], axis=1)


def label(ctx, batch, steps, dt):
    """DD closures of every realisation of a batch: sym(R^Lp) [R, 6]."""
    ctx.batch_set(batch)
    Lp, _ = ctx.batch_advance(steps, dt)
    return sym_voigt(Lp)


def feature_points(rng, n, rho_min=2e12, rho_max=2e13, stress_max=200e6):
    """Closure inputs: stress ~ U(-200, 200) MPa per component; total mobile and
    sessile densities log-uniform in [rho_min, rho_max]; per-system shares
    ~ Dirichlet(1, ..., 1) for each population.  [n, 30]."""
    f = np.zeros((n, 30))
    f[:, :6] = rng.uniform(-stress_max, stress_max, size=(n, 6))
    for col in (6, 18):
        tot = 10 ** rng.uniform(np.log10(rho_min), np.log10(rho_max), size=n)
        f[:, col:col + 12] = rng.dirichlet(np.ones(12), size=n) * tot[:, None]
    return f


def generate(ctx, feats, members, seed, steps, dt, n_loops=128, chunk=512, stratified=True, singles=None):
    """DD closures at the given feature points: the mean of sym(R^Lp) over
    `members` realisations drawn for each point (realisation_for_densities).
    If `singles` is an array [n, members, 6], every realisation's closure is
    also stored there."""
    rng = np.random.default_rng(seed)
    n = feats.shape[0]
    jobs = [(i, m) for i in range(n) for m in range(members)]
    acc = np.zeros((n, 6))
    t0 = time.perf_counter()
    pairs = 0
    for s0 in range(0, len(jobs), chunk):
        part = jobs[s0:s0 + chunk]
        nets = [W.realisation_for_densities(rng, feats[i, :6], feats[i, 6:18], feats[i, 18:], n_loops=n_loops,
                                            stratified=stratified)
                for i, _ in part]
        lab = label(ctx, W.batch_from_networks(nets), steps, dt)
        pairs += ctx.batch_info()["pairs_per_step"] * steps
        for (i, m), y in zip(part, lab):
            acc[i] += y
            if singles is not None:
                singles[i, m] = y
    return acc / members, time.perf_counter() - t0, pairs


def cubic_rotations():
    """The 24 proper rotations of the cube (signed permutation matrices,
    det +1) and, for each, the permutation of the 12 FCC slip systems it
    induces: Q b_s = +-b_perm[s], Q n_s = +-n_perm[s]."""
    import itertools
    bh, nh = W.fcc_slip_systems()
    rots, perms = [], []
    for p in itertools.permutations(range(3)):
        for signs in itertools.product((-1.0, 1.0), repeat=3):
            Q = np.zeros((3, 3))
            for i in range(3):
                Q[i, p[i]] = signs[i]
            if np.linalg.det(Q) < 0:
                continue
            qb, qn = bh @ Q.T, nh @ Q.T
            perm = np.argmax(np.abs(qb @ bh.T) * np.abs(qn @ nh.T), axis=1)
            rots.append(Q)
            perms.append(perm)
    return np.array(rots), np.array(perms)


def _voigt_rotate(v6, Q):
    """Voigt (xx, yy, zz, yz, xz, xy) symmetric tensors [n, 6] -> Q T Q^T."""
    T = np.zeros((v6.shape[0], 3, 3))
    T[:, 0, 0], T[:, 1, 1], T[:, 2, 2] = v6[:, 0], v6[:, 1], v6[:, 2]
    T[:, 1, 2] = T[:, 2, 1] = v6[:, 3]
    T[:, 0, 2] = T[:, 2, 0] = v6[:, 4]
    T[:, 0, 1] = T[:, 1, 0] = v6[:, 5]
    R = np.einsum("ij,njk,lk->nil", Q, T, Q)
    return np.stack([R[:, 0, 0], R[:, 1, 1], R[:, 2, 2], R[:, 1, 2], R[:, 0, 2], R[:, 0, 1]], axis=1)


def closure_symmetries():
    """The 48 exact symmetries of the closure map used here: the 24 cube
    rotations Q (with their slip-system permutations), each with a stress sign
    s = +-1.  Under (Q, s) the input maps to (s Q sigma Q^T, permuted
    densities) and the averaged rate to s Q Lp Q^T.

    Rotations: Q maps the FCC slip systems onto themselves, elasticity is
    isotropic, and the stratified realisations (loops in a cube, balanced
    line senses) and the input distribution are invariant.  Sign: negating
    sigma together with every Burgers vector leaves every force and velocity
    unchanged and negates Lp; negating a loop's Burgers vector is the same as
    reversing its line sense, which the balanced senses make a symmetry of
    the realisation distribution.  Returns a list of (Q, perm, s)."""
    rots, perms = cubic_rotations()
    return [(Q, perm, sg) for Q, perm in zip(rots, perms) for sg in (1.0, -1.0)]


def image_inputs(X, Q, perm, sg=1.0):
    """Closure inputs [n, 30] under the symmetry (Q, perm, sg)."""
    x = rotate_inputs(X, Q, perm)
    x[:, :6] *= sg
    return x


def cubic_images(X, Y):
    """All 48 symmetric copies (closure_symmetries) of closure samples.
    Returns ([48 n, 30], [48 n, 6])."""
    xs, ys = [], []
    for Q, perm, sg in closure_symmetries():
        xs.append(image_inputs(X, Q, perm, sg))
        ys.append(sg * _voigt_rotate(Y, Q))
    return np.concatenate(xs), np.concatenate(ys)


def rotate_inputs(X, Q, perm):
    """Closure inputs [n, 30] under the cube rotation Q (slip-system permutation perm)."""
    x = np.empty_like(X)
    x[:, :6] = _voigt_rotate(X[:, :6], Q)
    for off in (6, 18):
        x[:, off + perm] = X[:, off:off + 12]
    return x


def symmetrised_inputs(X):
    """[48 n, 30]: the images of X under closure_symmetries, image-major."""
    return np.concatenate([image_inputs(X, Q, perm, sg) for Q, perm, sg in closure_symmetries()])


def symmetrised_answers(ys, n):
    """Answers [48 n, 6] for symmetrised_inputs(X) -> their average mapped
    back to X (s Q^T y Q per image), and the index of the identity image."""
    syms = closure_symmetries()
    acc = np.zeros((n, 6))
    for g, (Q, _, sg) in enumerate(syms):
        acc += sg * _voigt_rotate(ys[g * n:(g + 1) * n], Q.T)
    g0 = next(g for g, (Q, _, sg) in enumerate(syms) if sg > 0 and np.array_equal(Q, np.eye(3)))
    return acc / len(syms), g0


def predict_symmetrised(ctx, X):
    """The surrogate averaged over the 48 symmetric images of each input (an
    exactly symmetric answer; in particular odd in sigma, so zero at zero
    stress).  Returns (lp6 [n, 6], in_region of the inputs themselves)."""
    n = X.shape[0]
    ys, inr = ctx.surrogate_predict(symmetrised_inputs(X))
    lp, g0 = symmetrised_answers(ys, n)
    return lp, inr[g0 * n:(g0 + 1) * n]


def relerr(pred, ref):
    return float(np.linalg.norm(pred - ref) / np.linalg.norm(ref))


def fit_early_stopping(ctx, Xfit, Yfit, Xval, Yval, augment=True, epochs=60, round_epochs=1, patience=3,
                       lr_drops=2, batch=512, lr=1e-3, seed=0):
    """Fit the context's surrogate on (Xfit, Yfit) with early stopping.

    The labels are single noisy realisations, so the network is trained in
    rounds of `round_epochs` and the round with the lowest relative error on
    the validation split (also single realisations, never augmented) is
    kept; on a plateau of `patience` rounds the best state is restored and
    the learning rate cut by 0.3, up to `lr_drops` times.  With `augment`
    every fit sample enters in its 48 symmetric forms (cubic_images).
    Returns (best validation error, [[epoch, lr, loss, val err], ...], fit samples)."""
    if augment:
        Xfit, Yfit = cubic_images(Xfit, Yfit)
        order = np.random.default_rng(seed + 11).permutation(Xfit.shape[0])
        Xfit, Yfit = Xfit[order], Yfit[order]
    best, best_err, curve, bad, drops, ep = None, np.inf, [], 0, 0, 0
    while ep < epochs:
        losses = ctx.surrogate_fit(Xfit, Yfit, epochs=round_epochs, batch=batch, lr=lr, seed=seed + ep)
        ep += round_epochs
        pv, _ = ctx.surrogate_predict(Xval)
        e = relerr(pv, Yval)
        curve.append([ep, lr, float(losses[-1]), e])
        if e < best_err - 1e-4:
            best, best_err, bad = ctx.surrogate_get_state(), e, 0
        else:
            bad += 1
            if bad >= patience:
                if drops >= lr_drops:
                    break
                ctx.surrogate_set_state(best)
                lr, drops, bad = lr * 0.3, drops + 1, 0
    ctx.surrogate_set_state(best)
    return best_err, curve, int(Xfit.shape[0])


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--samples", type=int, default=20000)
    p.add_argument("--holdout", type=float, default=0.1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--dt", type=float, default=5e-13)
    p.add_argument("--seed", type=int, default=1004)
    p.add_argument("--epochs", type=int, default=60, help="maximum epochs")
    p.add_argument("--round-epochs", type=int, default=1)
    p.add_argument("--patience", type=int, default=3)
    p.add_argument("--lr-drops", type=int, default=2, help="learning-rate cuts (x0.3) on a validation plateau")
    p.add_argument("--no-augment", dest="augment", action="store_false",
                   help="train on the labelled samples only, without their 48 symmetric images")
    p.add_argument("--val-frac", type=float, default=0.1)
    p.add_argument("--save-data", default=None, help="write the features and labels (npz)")
    p.add_argument("--batch", type=int, default=512)
    p.add_argument("--lr", type=float, default=1e-3)
    p.add_argument("--fp64-check", type=int, default=32, help="hold-out points relabelled with FP64 DD")
    p.add_argument("--members", type=int, default=16, help="realisations per hold-out ensemble mean")
    p.add_argument("--loops", type=int, default=128, help="loops per realisation")
    p.add_argument("--eval", type=int, default=400, help="hold-out points scored against ensemble means")
    p.add_argument("--load-data", default=None, help="reuse a labelled set written by --save-data")
    p.add_argument("--infer", type=int, default=1 << 20)
    p.add_argument("--device", type=int, default=0)
    p.add_argument("--save", default=None, help="write the fitted surrogate state to this file")
    a = p.parse_args(argv)

    mat = W.Material().as_tuple()
    out = {"samples": a.samples, "steps": a.steps, "dt": a.dt, "seed": a.seed, "loops_per_realisation": a.loops,
           "holdout_members": a.members}
    rng = np.random.default_rng(a.seed)
    ntr = int(round(a.samples * (1 - a.holdout)))
    X = feature_points(rng, a.samples)
    nev = min(a.eval, a.samples - ntr)
    with ptadd.Context(mat, ptadd.PTADD_MIXED, a.device) as ctx:
        if a.load_data:
            d = np.load(a.load_data)
            X, Ytr, Yho, Y1 = d["X"], d["Ytr"], d["Yho"], d["Y1"]
            assert X.shape[0] == a.samples and Yho.shape[0] == nev, "labelled set does not match the arguments"
            out["labels_from"] = a.load_data
            out["dd_closures_per_s"] = float(d["dd_closures_per_s"])
        else:
            # training labels: one realisation per point; the scored hold-out
            # points: ensemble means and one independent single realisation
            Ytr, t_gen, pairs = generate(ctx, X[:ntr], 1, a.seed + 1, a.steps, a.dt, a.loops)
            Yho, t_ho, _ = generate(ctx, X[ntr:ntr + nev], a.members, a.seed + 2, a.steps, a.dt, a.loops)
            out.update({"dd_label_s": t_gen, "dd_closures_per_s": ntr / t_gen, "dd_pair_evals_per_s": pairs / t_gen,
                        "holdout_label_s": t_ho})
            Y1, _, _ = generate(ctx, X[ntr:ntr + nev], 1, a.seed + 3, a.steps, a.dt, a.loops)
        nval = max(64, int(a.val_frac * ntr))
        nfit = ntr - nval
        t0 = time.perf_counter()
        best_err, curve, fit_samples = fit_early_stopping(ctx, X[:nfit], Ytr[:nfit], X[nfit:ntr], Ytr[nfit:ntr],
                                                          augment=a.augment, epochs=a.epochs,
                                                          round_epochs=a.round_epochs, patience=a.patience,
                                                          lr_drops=a.lr_drops, batch=a.batch, lr=a.lr, seed=a.seed)
        out["fit_samples"] = fit_samples
        out["train_s"] = time.perf_counter() - t0
        out["training_curve_epoch_lr_loss_valerr"] = curve
        out["best_val_rel_err"] = best_err
        pred, inr = ctx.surrogate_predict(X[ntr:ntr + nev])
        err = relerr(pred, Yho)
        single = relerr(Y1, Yho) * np.sqrt(a.members / (a.members + 1.0))  # one realisation vs the true mean
        floor = single / np.sqrt(a.members)
        out["holdout"] = {
            "n": int(nev),
            "rel_err_vs_ensemble_mean": err,
            "rel_err_in_region": relerr(pred[inr], Yho[inr]) if inr.any() else None,
            "in_region_frac": float(inr.mean()),
            "single_realisation_rel_spread": single,
            "ensemble_mean_noise_floor": floor,
            "rel_err_noise_corrected": float(np.sqrt(max(0.0, err * err - floor * floor))),
            "rel_err_symmetrised": relerr(predict_symmetrised(ctx, X[ntr:ntr + nev])[0], Yho),
            "mean_predictor_rel_err": relerr(np.broadcast_to(Ytr.mean(0), Yho.shape), Yho),
            "label_norm_median": float(np.median(np.linalg.norm(Yho, axis=1))),
        }
        train_pred, _ = ctx.surrogate_predict(X[:nfit])
        out["train_rel_err_vs_single_labels"] = relerr(train_pred, Ytr[:nfit])
        if a.save_data:
            np.savez_compressed(a.save_data, X=X, Ytr=Ytr, Yho=Yho, Y1=Y1, dd_closures_per_s=out["dd_closures_per_s"])
        if a.save:
            with open(a.save, "wb") as fh:
                fh.write(ctx.surrogate_get_state())

        # surrogate inference on device-resident points resampled from the training features
        try:
            import torch
            feats = X[rng.integers(0, ntr, size=a.infer)]
            fd = torch.from_numpy(feats).cuda(a.device)
            yd = torch.empty((a.infer, 6), dtype=torch.float64, device=fd.device)
            rd = torch.empty(a.infer, dtype=torch.uint8, device=fd.device)
            st = torch.cuda.Stream(device=fd.device)  # a real (non-default) stream shared with the library
            torch.cuda.synchronize()
            ctx.set_stream(st.cuda_stream)
            ctx.surrogate_predict_dev(a.infer, fd.data_ptr(), yd.data_ptr(), rd.data_ptr())  # warm-up
            st.synchronize()
            reps = 10
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(reps):
                ctx.surrogate_predict_dev(a.infer, fd.data_ptr(), yd.data_ptr(), rd.data_ptr())
            e1.record(st)
            st.synchronize()
            ms = e0.elapsed_time(e1) / reps
            ctx.set_stream(None)
            flops = 2.0 * (30 * 256 + 256 * 256 * 2 + 256 * 6) * a.infer
            out["inference"] = {"points": a.infer, "ms": ms, "closures_per_s": a.infer / (ms * 1e-3),
                                "tflops_algorithmic": flops / (ms * 1e-3) / 1e12,
                                "in_region_frac": float(rd.float().mean().item()),
                                "gain_vs_dd_closures": (a.infer / (ms * 1e-3)) / out["dd_closures_per_s"]}
        except ImportError:
            out["inference"] = None

    if a.fp64_check > 0:
        k = min(a.fp64_check, nev)
        with ptadd.Context(mat, ptadd.PTADD_FP64, a.device) as ctx64:
            y64, t64, _ = generate(ctx64, X[ntr:ntr + k], 1, a.seed + 3, a.steps, a.dt, a.loops)
        out["fp64_check"] = {"n": k, "mixed_vs_fp64_rel_err": relerr(Y1[:k], y64),
                             "fp64_dd_closures_per_s": k / t64}
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
