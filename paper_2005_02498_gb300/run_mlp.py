"""Time the surrogate MLP: training (tcgen05 GEMMs, Adam) and fused inference.

    python -m paper_2005_02498_gb300.run_mlp --points 1048576 --fit-samples 65536 --epochs 5

The network is fitted to a smooth synthetic closure (resolved-stress-like
response times log density) on `--fit-samples` points, so the timings need
no DD labels; then `--points` device-resident inputs drawn from the same
distribution are answered by the fused inference kernel.  Training time is
host-measured around `ptadd_surrogate_fit` (which synchronises); inference
is timed with CUDA events on the library's stream.  Prints one JSON line.
"""

from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import ptadd
from . import workloads as W

FLOP_FWD = 2.0 * (30 * 256 + 256 * 256 * 2 + 256 * 6)  # per point, unpadded


def synthetic(rng, n):
    sig = rng.uniform(-200e6, 200e6, size=(n, 6))
    rho = 10 ** rng.uniform(11, 13, size=(n, 24))
    lp = np.tanh(sig / 1e8) * (np.log10(rho[:, :6]) - 10.0) * 50.0
    return np.hstack([sig, rho]), lp


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--points", type=int, default=1 << 20)
    p.add_argument("--fit-samples", type=int, default=65536)
    p.add_argument("--epochs", type=int, default=5)
    p.add_argument("--batch", type=int, default=512)
    p.add_argument("--reps", type=int, default=20)
    p.add_argument("--device", type=int, default=0)
    a = p.parse_args(argv)

    import torch

    rng = np.random.default_rng(8)
    feat, lp = synthetic(rng, a.fit_samples)
    out = {"fit_samples": a.fit_samples, "epochs": a.epochs, "batch": a.batch, "points": a.points}
    with ptadd.Context(W.Material().as_tuple(), ptadd.PTADD_MIXED, a.device) as ctx:
        ctx.surrogate_fit(feat[:4096], lp[:4096], epochs=1, batch=a.batch, seed=1)  # warm-up
        t0 = time.perf_counter()
        losses = ctx.surrogate_fit(feat, lp, epochs=a.epochs, batch=a.batch, seed=2)
        t_fit = time.perf_counter() - t0
        samples = a.fit_samples * a.epochs
        out["train"] = {"s": t_fit, "samples_per_s": samples / t_fit,
                        "tflops_algorithmic": 3 * FLOP_FWD * samples / t_fit / 1e12,
                        "final_loss": float(losses[-1])}
        X, _ = synthetic(rng, a.points)
        fd = torch.from_numpy(X).cuda(a.device)
        yd = torch.empty((a.points, 6), dtype=torch.float64, device=fd.device)
        rd = torch.empty(a.points, dtype=torch.uint8, device=fd.device)
        st = torch.cuda.Stream(device=fd.device)
        torch.cuda.synchronize()
        ctx.set_stream(st.cuda_stream)
        for _ in range(3):
            ctx.surrogate_predict_dev(a.points, fd.data_ptr(), yd.data_ptr(), rd.data_ptr())
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(a.reps):
            ctx.surrogate_predict_dev(a.points, fd.data_ptr(), yd.data_ptr(), rd.data_ptr())
        e1.record(st)
        st.synchronize()
        ctx.set_stream(None)
        ms = e0.elapsed_time(e1) / a.reps
        out["inference"] = {"ms": ms, "closures_per_s": a.points / (ms * 1e-3),
                            "tflops_algorithmic": FLOP_FWD * a.points / (ms * 1e-3) / 1e12,
                            "in_region_frac": float(rd.float().mean().item()),
                            "finite": bool(torch.isfinite(yd).all().item())}
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
