#!/usr/bin/env python3
"""Benchmark of the DD burst: segment-pair evaluations per second.

Workload: 1024 circular FCC glide loops x 32 segments (32768 segments) in a
5 um cube, isotropic FCC (mu 48 GPa, nu 0.34, b 0.2556 nm, a = b), drag
B = 1e-4 Pa s, 50 MPa uniaxial [001], dt = 1e-11 s.  One benchmark step is
one pass of the whole burst hot path -- pair stress at 4 Gauss points of
every segment from every segment, Peach-Koehler nodal forces, glide
mobility, Lp/rho averaging, explicit Euler -- over `--dd-steps` DD steps.

  value   : device time (CUDA events on the library's stream) of the K
            timed steps, inputs resident in HBM, L2 flushed between steps;
  e2e     : the same metric through the C ABI with host buffers: per step
            positions copied in from pinned host memory (ptadd_set_nodes),
            the burst, positions and averages copied back;
  roofline: the pair-stress kernel, algorithmic FLOPs per launch over its
            CUDA-event time, against the FMA peak of its arithmetic type from
            the unit counts and the maximum SM clock (FP32: 128 FMA lanes per
            SM; FP64: 2 per SM), with the FMA-chain peaks measured in the
            same run beside it;
  cpu_baseline: the FP64 CPU oracle on a bounded sample of the same workload.

Multi-GPU (torchrun): every rank runs its own realisation (seed + rank);
no data-path collective; the timed region is bracketed by barriers and the
maximum time over ranks is reported ("scaling": "weak").
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2005_02498_gb300 import workloads as W  # noqa: E402

# Algorithmic FLOPs of one segment-pair evaluation (one source segment at the
# 4 Gauss points of one target segment), counted from the formulation in
# csrc/seg_field.cuh with an FMA as 2 FLOPs and each reciprocal or
# reciprocal square root as 1: 4 x 165 per field point + 19 per pair.
FLOPS_PER_PAIR = 4 * 165 + 19
L2_FLUSH_BYTES = 256 << 20


def _bf16_peak():
    """Dense BF16 tensor peak for a kernel timed alone (burst figure)."""
    try:
        return (float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]),
                "measured: MEASURED_PEAKS.json bf16_tflops (cuBLAS burst)")
    except (OSError, ValueError, KeyError):
        return 1900.0, "fallback: one earlier burst measurement of a GB300"


BF16_PEAK_TFLOPS, BF16_PEAK_SOURCE = _bf16_peak()
WORKLOAD = ("1024 circular FCC glide loops x 32 segments = 32768 segments, 5 um cube, "
            "mu 48 GPa, nu 0.34, b 0.2556 nm, a = b, B 1e-4 Pa s, 50 MPa [001], dt 1e-11 s")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    p.add_argument("--fp64-steps", type=int, default=2,
                   help="steps of plain FP64 DD timed beside the mixed path (0 = skip)")
    p.add_argument("--dd-steps", type=int, default=1, help="DD steps per benchmark step")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="target length of the CPU-baseline sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-closures", action="store_true", help="skip the PTA-closure legs (batched ensemble, sweep)")
    p.add_argument("--c3-steps", type=int, default=10, help="timed DD steps of the 256-realisation batch")
    p.add_argument("--c3-fp64-R", type=int, default=16, help="realisations of the plain FP64 batch subsample")
    p.add_argument("--sur-train", type=int, default=8000, help="DD-labelled closures the surrogate is fitted on")
    p.add_argument("--sweep-steps", type=int, default=3, help="load steps of the 100-step sweep that are run")
    # 48 members put the references' own noise floor near 2 % (16 gave 3.4 %, the size of the bar)
    p.add_argument("--ref-points", type=int, default=6, help="(point, step) pairs checked against FP64 DD")
    p.add_argument("--ref-members", type=int, default=48, help="FP64 DD realisations per reference mean")
    return p.parse_args()


def rank_seed(rank):
    """Seed of the realisation rank `rank` runs (independent realisations: weak scaling)."""
    return W.LARGE_LOOPS["seed"] + rank


def max_over_ranks(x, dist, device):
    """The maximum of a per-rank float over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Units processed by all ranks per second of the slowest rank."""
    return world * units_per_rank / seconds


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        with open(self.path) as f:
            summary = clock_summary(f)
        os.unlink(self.path)
        return summary


def clock_summary(lines):
    """Median and maximum SM clock and the throttle reasons seen, from the
    lines of `nvidia-smi --query-gpu=<ClockSampler.FIELDS>
    --format=csv,noheader,nounits`; None without a sample."""
    rows = []
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) >= 9:
            rows.append(parts)
    if not rows:
        return None

    def num(x):
        try:
            return float(x)
        except ValueError:
            return float("nan")

    sm = [num(r[1]) for r in rows]
    mx = [num(r[2]) for r in rows]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
    return {"sm_mhz": float(np.nanmedian(sm)), "sm_max_mhz": float(np.nanmax(mx)), "reasons": reasons,
            "samples": len(rows)}


# ---------------------------------------------------------------- helpers
def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("seg_field.cuh", "pair_tile.cuh", "dd_kernels.cu"):
        h.update(open(os.path.join(ROOT, "paper_2005_02498_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_capture(precision):
    """The committed ncu figures of the pair kernel (DRAM bytes per launch,
    executed FLOPs per evaluation), if the kernel source is unchanged since
    they were taken; else an empty dict."""
    path = os.path.join(ROOT, "profiles", "pair_kernel_traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return {}
    e = rec.get(precision)
    if not e or e.get("kernel_src_sha") != kernel_source_sha():
        return {}
    return e


def recorded_traffic(precision):
    """DRAM bytes per pair launch from a committed ncu capture, or None."""
    return recorded_capture(precision).get("dram_bytes_per_launch")


def cpu_sample(net, seconds, mat):
    """Oracle forces on a random node sample sized to take about `seconds`."""
    import oracle  # test infrastructure: only this baseline leg uses it
    rng = np.random.default_rng(7)
    k = 8
    t0 = time.perf_counter()
    oracle.nodal_forces_subset(mat, net, rng.choice(net.n_nodes, k, replace=False))
    dt = time.perf_counter() - t0
    k = int(max(8, min(net.n_nodes, k * seconds / max(dt, 1e-3))))
    sel = rng.choice(net.n_nodes, k, replace=False)
    t0 = time.perf_counter()
    oracle.nodal_forces_subset(mat, net, sel)
    dt = time.perf_counter() - t0
    pairs = 2 * k * net.n_nodes  # two target segments per node, every source
    return pairs / dt, oracle.num_threads(), k, dt


def emit(obj):
    print(json.dumps(obj), flush=True)


def arm_config(args, n_segments, world):
    """The workload description both arms report."""
    return {"workload": WORKLOAD, "precision": args.precision, "dd_steps_per_step": args.dd_steps,
            "pairs_per_step": n_segments * n_segments * args.dd_steps, "segments": n_segments,
            "l2": "flushed between timed steps (256 MB device write)",
            "parallelism": "one independent realisation per GPU" if world > 1 else "single GPU"}


# ------------------------------------------------------ closure legs
BATCH_WORKLOAD = ("256 independent realisations, N_r ~ U{1024..16384} segments in loops of 32, every stress "
                  "component ~ U(-200, 200) MPa, sessile loop fraction ~ U(0.1, 0.9), 16 loops per um^3, "
                  "dt 1e-11 s, 2000-step bursts, seed 1003")
SWEEP_WORKLOAD = ("16^3 material points, 100 load steps of smooth random stress fields up to 200 MPa and density "
                  "fields of the training marginals (seed 1005); surrogate inside its trust region, 64-realisation "
                  "DD ensembles of 4096-segment closures (128 loops, 100 steps at dt 5e-13 s) outside it")


def closure_legs(args, device):
    """PTA closures/s on the batched workloads, against plain FP64 DD on the
    same GPU: (1) the 256-realisation ensemble, mixed precision, timed steps
    extrapolated to its 2000-step bursts, with plain FP64 on a subsample
    extrapolated per segment pair; (2) the closure sweep: a surrogate fitted
    here on DD-labelled closures answers inside its trust region, DD
    ensembles outside it, on evenly spaced load steps of the 100-step load
    path (extrapolated), its answers checked against FP64 DD ensemble means
    on a sample of (point, step) pairs.  Wall-clock timing of synchronous
    calls (each call ends with a device-to-host copy of its results)."""
    import torch

    from paper_2005_02498_gb300 import closure_sweep as CS
    from paper_2005_02498_gb300 import ptadd
    from paper_2005_02498_gb300 import surrogate as SU

    mat = W.Material().as_tuple()
    out = {}
    # (1) batched ensemble
    batch = W.batch_ensemble(1003, R=256)
    dt3, burst = 1e-11, 2000
    with ptadd.Context(mat, ptadd.PTADD_MIXED, device) as c:
        c.batch_set(batch)
        c.batch_autotune()
        info = c.batch_info()
        c.batch_advance(2, dt3)  # warm-up: captures the two-step graph
        c.batch_set_nodes(batch.xyz)
        t0 = time.perf_counter()
        c.batch_advance(args.c3_steps, dt3)
        el = time.perf_counter() - t0
    ms = 1e3 * el / args.c3_steps
    sub = W.batch_from_networks([batch.realisation(r) for r in range(args.c3_fp64_R)])
    with ptadd.Context(mat, ptadd.PTADD_FP64, device) as c:
        c.batch_set(sub)
        pairs_sub = c.batch_info()["pairs_per_step"]
        c.batch_advance(1, dt3)
        c.batch_set_nodes(sub.xyz)
        t0 = time.perf_counter()
        c.batch_advance(2, dt3)
        el64 = time.perf_counter() - t0
    rate64 = pairs_sub * 2 / el64
    cps = batch.R / (ms * 1e-3 * burst)
    cps64 = batch.R / (info["pairs_per_step"] / rate64 * burst)
    out["batched_ensemble"] = {
        "workload": BATCH_WORKLOAD, "segments": int(batch.xyz.shape[0]), "pairs_per_step": info["pairs_per_step"],
        "tile_targets": info["tile_targets"], "chunk_sources": info["chunk_sources"],
        "timed_steps": args.c3_steps, "ms_per_step": ms, "pair_evals_per_s": info["pairs_per_step"] / (ms * 1e-3),
        "closures_per_s": cps, "closures_per_s_note": "timed steps extrapolated to the 2000-step bursts",
        "fp64_dd": {"realisations": args.c3_fp64_R, "steps": 2, "pair_evals_per_s": rate64,
                    "closures_per_s": cps64, "note": "plain FP64 on the first realisations, extrapolated per "
                                                     "segment pair to the whole batch"},
        "speedup_vs_fp64_dd": cps / cps64}

    # (2) surrogate fitted on DD closures, then the sweep slice
    steps, dt, loops, members = 100, 5e-13, 128, 64
    rng = np.random.default_rng(1004)
    nval = max(64, args.sur_train // 10)
    X = SU.feature_points(rng, args.sur_train + nval)
    pts, S, rho = CS.material_points(1005, 16)
    K = 100
    ks_run = CS.load_steps_run(K, args.sweep_steps)
    with ptadd.Context(mat, ptadd.PTADD_MIXED, device) as c:
        Y, t_lab, _ = SU.generate(c, X, 1, 1005, steps, dt, loops)
        t0 = time.perf_counter()
        val_err, curve, nfit = SU.fit_early_stopping(c, X[:args.sur_train], Y[:args.sur_train],
                                                     X[args.sur_train:], Y[args.sur_train:], epochs=40, seed=1004)
        t_fit = time.perf_counter() - t0
        # fused inference on 1M device-resident points resampled from the training inputs
        feats = torch.from_numpy(X[rng.integers(0, X.shape[0], size=1 << 20)]).cuda(device)
        yd = torch.empty((1 << 20, 6), dtype=torch.float64, device=feats.device)
        rd = torch.empty(1 << 20, dtype=torch.uint8, device=feats.device)
        st = torch.cuda.Stream(device=feats.device)
        torch.cuda.synchronize()
        c.set_stream(st.cuda_stream)
        c.surrogate_predict_dev(1 << 20, feats.data_ptr(), yd.data_ptr(), rd.data_ptr())
        st.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(10):
            c.surrogate_predict_dev(1 << 20, feats.data_ptr(), yd.data_ptr(), rd.data_ptr())
        e1.record(st)
        st.synchronize()
        inf_ms = e0.elapsed_time(e1) / 10
        c.set_stream(None)
        del feats, yd, rd
        r = CS.sweep(c, S, rho, K, ks_run, members, steps, dt, loops, 1005, True, device)
    # FP64 DD reference means on a random sample of (point, step) pairs of the run steps
    n = S.shape[0]
    rs = np.random.default_rng(1006)
    kr = np.asarray(ks_run) - 1
    pick = rs.choice(len(kr) * n, size=min(args.ref_points, len(kr) * n), replace=False)
    ks, ps = kr[pick // n], pick % n
    fref = np.hstack([S[ps] * ((ks + 1) / K)[:, None], rho[ps]])
    singles = np.zeros((pick.size, args.ref_members, 6))
    with ptadd.Context(mat, ptadd.PTADD_FP64, device) as c:
        t0 = time.perf_counter()
        ref, _, _ = SU.generate(c, fref, args.ref_members, 1007, steps, dt, loops, singles=singles)
        t_ref = time.perf_counter() - t0
    got = r["answers"][ks, ps]
    # noise of the reference means: spread of single realisations / sqrt(members)
    M = args.ref_members
    spread = float(np.linalg.norm(singles - ref[:, None, :]) / np.sqrt(M - 1) / np.linalg.norm(ref) / np.sqrt(M))
    fp64_real_per_s = pick.size * args.ref_members / t_ref
    total = r["wall_s"] * K / len(ks_run)
    sweep_cps = n * K / total
    fp64_cps = fp64_real_per_s / members  # an all-DD sweep answers each point with a 64-member ensemble
    run = np.asarray(ks_run) - 1
    flops = 2.0 * (30 * 256 + 256 * 256 * 2 + 256 * 6) * (1 << 20)
    out["surrogate"] = {
        "training_closures": args.sur_train, "validation_closures": nval, "fit_samples_with_images": nfit,
        "dd_label_closures_per_s_mixed": (args.sur_train + nval) / t_lab, "fit_s": t_fit,
        "validation_rel_err": val_err,
        "inference": {"points": 1 << 20, "ms": inf_ms, "closures_per_s": (1 << 20) / (inf_ms * 1e-3),
                      "tflops_algorithmic": flops / (inf_ms * 1e-3) / 1e12,
                      "frac_of_bf16_peak": flops / (inf_ms * 1e-3) / 1e12 / BF16_PEAK_TFLOPS,
                      "bf16_peak_tflops": BF16_PEAK_TFLOPS, "peak_source": BF16_PEAK_SOURCE}}
    out["closure_sweep"] = {
        "workload": SWEEP_WORKLOAD, "load_steps_run": len(ks_run), "closures": n * K,
        "closures_per_s": sweep_cps, "closures_per_s_note": "run load steps extrapolated to all 100",
        "fallback_fraction": float(r["used_dd"][run].mean()), "fallback_closures": int(r["fallback_closures"]),
        "rel_err_vs_fp64_dd": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
        "reference": {"pairs": int(pick.size), "members": args.ref_members, "precision": "fp64",
                      "noise_floor_rel": spread},
        "fp64_dd_closures_per_s": fp64_cps,
        "speedup_vs_fp64_dd": sweep_cps / fp64_cps}
    return out


# --------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    net = W.large_loop_network()
    mat = W.Material().as_tuple()
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_sample(net, per_step / 4, mat)
    vals, cores, ks, secs = [], 0, [], 0.0
    for _ in range(args.steps):
        v, cores, k, dt = cpu_sample(net, per_step, mat)
        vals.append(v)
        ks.append(k)
        secs += dt
    value = float(np.mean(vals))
    sample = ("FP64 CPU oracle (the reference arm computes in FP64 whatever the precision of the other arm): "
              "nodal forces of %d-%d randomly sampled nodes (2 target segments each) against all 32768 source "
              "segments per step" % (min(ks), max(ks)))
    emit({"impl": "reference", "metric": "segment-pair evals/s", "value": value, "unit": "pair-evals/s",
          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
          "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
          "config": arm_config(args, net.n_nodes, world),
          "cpu_baseline": {"value": value, "unit": "pair-evals/s", "cores": cores, "kind": "oracle",
                           "sample": sample},
          "e2e": {"value": value, "unit": "pair-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})
    return 0


# -------------------------------------------------------------- our arm
def run_ours(args):
    import torch

    from paper_2005_02498_gb300 import ptadd

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    ptadd.load()
    prec = ptadd.PTADD_FP64 if args.precision == "fp64" else ptadd.PTADD_MIXED
    mat = W.Material()
    net = W.large_loop_network(seed=rank_seed(rank))
    dt = W.LARGE_LOOPS["dt"]
    stream = torch.cuda.Stream()  # a real stream shared by the library and the timing events
    torch.cuda.set_stream(stream)
    ctx = ptadd.Context(mat.as_tuple(), prec, local)
    ctx.set_stream(stream.cuda_stream)
    ctx.set_network(net)
    info = ctx.info()
    pairs_per_bench_step = info["pairs_per_step"] * args.dd_steps

    meas_fp64 = ptadd.fma_peak(local, fp64=True, seconds=2.0)
    meas_fp32 = ptadd.fma_peak(local, fp64=False, seconds=2.0)
    meas_fp32x2 = ptadd.fma_peak(local, fp64=False, packed=True, seconds=2.0)
    sms = torch.cuda.get_device_properties(local).multi_processor_count

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        ctx.advance(args.dd_steps, dt)
    torch.cuda.synchronize()

    # ---- device-timed region
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ctx.profile_reset(timing=True)
    evs = []
    for _ in range(args.steps):
        flush.fill_(1.0)  # evict L2 between timed steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.advance(args.dd_steps, dt)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    elapsed_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), dist, "cuda")
    value = whole_job_rate(pairs_per_bench_step * args.steps, world, elapsed_ms * 1e-3)

    # ---- plain FP64 DD on the same GPU and workload, for the ratio
    fp64_cmp = None
    if args.precision == "mixed" and args.fp64_steps > 0:
        ctx.set_precision(ptadd.PTADD_FP64)
        ctx.advance(args.dd_steps, dt)  # warm-up
        torch.cuda.synchronize()
        ctx.profile_reset(timing=True)
        evs64 = []
        for _ in range(args.fp64_steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.advance(args.dd_steps, dt)
            e1.record(stream)
            evs64.append((e0, e1))
        torch.cuda.synchronize()
        p64 = ctx.profile_read()
        ms64 = sum(a.elapsed_time(b) for a, b in evs64)
        ms64 = max_over_ranks(ms64, dist, "cuda")
        v64 = whole_job_rate(pairs_per_bench_step * args.fp64_steps, world, ms64 * 1e-3)
        fp64_cmp = {"value": v64, "unit": "pair-evals/s", "steps": args.fp64_steps,
                    "ms_per_step": ms64 / args.fp64_steps, "speedup_of_mixed": value / v64,
                    "pair_kernel_tflops": FLOPS_PER_PAIR * p64["pair_evals"] / (p64["pair_ms"] * 1e-3) / 1e12}
        ctx.set_precision(prec)

    # ---- end to end through the C ABI with pinned host buffers
    n = info["n_nodes"]
    host_in = torch.from_numpy(net.xyz.copy()).pin_memory()
    host_out = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    ctx.profile_reset(timing=False)
    e2e_times = []
    for i in range(args.e2e_steps + 1):
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        ctx.set_nodes(host_in.data_ptr())
        ctx.advance(args.dd_steps, dt)
        ctx.get_nodes_into(host_out.data_ptr())
        t1 = time.perf_counter()
        if i > 0:  # the first round trip is a warm-up
            e2e_times.append(t1 - t0)
    e2e_s = max_over_ranks(float(np.sum(e2e_times)), dist, "cuda")
    e2e_value = whole_job_rate(pairs_per_bench_step * len(e2e_times), world, e2e_s)
    h2d = 3 * n * 8
    d2h = 3 * n * 8 + 10 * 8 + 4

    # ---- roofline of the dominant kernel (pair stress)
    avg_ms = prof["pair_ms"] / max(1, prof["pair_launches"])
    evals_per_launch = prof["pair_evals"] / max(1, prof["pair_launches"])
    achieved = FLOPS_PER_PAIR * evals_per_launch / (avg_ms * 1e-3)
    max_mhz = clk.get("sm_max_mhz") if clk and clk.get("sm_max_mhz") == clk.get("sm_max_mhz") else None
    max_mhz = max_mhz or 2070.0
    lanes = 2 if args.precision == "fp64" else 128  # FMA lanes per SM per clock
    peak = sms * lanes * 2 * max_mhz * 1e6
    if fp64_cmp:
        peak64 = sms * 2 * 2 * max_mhz * 1e6
        fp64_cmp["pair_kernel_frac_of_fp64_peak"] = fp64_cmp["pair_kernel_tflops"] * 1e12 / peak64
        x64 = recorded_capture("fp64").get("executed_fp64_flops_per_pair")
        if x64 is not None:
            t64 = fp64_cmp["pair_kernel_tflops"] * x64 / FLOPS_PER_PAIR
            fp64_cmp["executed"] = {"flops_per_pair": x64, "achieved": t64, "frac": t64 * 1e12 / peak64,
                                    "unit": "TFLOP/s"}
    roof = {"kernel": "pair_fp64_kernel" if args.precision == "fp64" else "pair_mixed_kernel",
            "bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": recorded_traffic(args.precision),
            "flops_per_pair": FLOPS_PER_PAIR, "pair_evals_per_launch": evals_per_launch,
            "avg_launch_ms": avg_ms,
            "peak_source": "%s FMA peak from unit counts: %d SMs x %d FMA lanes x 2 FLOP x %.0f MHz (maximum SM "
                           "clock); MEASURED_PEAKS.json has no FP32/FP64 figure"
                           % ("FP64" if args.precision == "fp64" else "FP32", sms, lanes, max_mhz),
            "measured_fma_chain_tflops": {"fp64": meas_fp64 / 1e12, "fp32": meas_fp32 / 1e12,
                                          "fp32_packed_pairs": meas_fp32x2 / 1e12}}
    # the same launch in executed operations (ncu instruction counters of the
    # recorded capture): the mixed kernel's coefficient form needs fewer than
    # the formulation that defines the unit
    cap = recorded_capture(args.precision)
    xkey = "executed_fp64_flops_per_pair" if args.precision == "fp64" else "executed_fp32_flops_per_pair"
    if cap.get(xkey) is not None and avg_ms > 0:
        executed = cap[xkey] * evals_per_launch / (avg_ms * 1e-3)
        roof["executed"] = {"flops_per_pair": cap[xkey], "achieved": executed / 1e12, "frac": executed / peak,
                            "unit": "TFLOP/s", "counted_on": cap.get("executed_counted_on")}
    else:
        roof["executed"] = None

    out = {"metric": "segment-pair evals/s", "value": value, "unit": "pair-evals/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if args.precision == "fp64" else "f32+f64",
           "data": "synthetic",
           "config": arm_config(args, n, world),
           "roofline": roof,
           "e2e": {"value": e2e_value, "unit": "pair-evals/s", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h},
           "gpu_launches": int(prof["kernel_launches"]),
           "fp64_dd": fp64_cmp,
           "near_field_point_pairs_per_step": prof.get("near_point_pairs", 0) / max(1, args.steps),
           "clocks": clk}
    ctx.close()
    del flush
    torch.cuda.empty_cache()

    if rank == 0 and world == 1 and not args.no_closures:
        out["closures"] = closure_legs(args, local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, k, secs = cpu_sample(net, args.cpu_seconds, mat.as_tuple())
        out["cpu_baseline"] = {"value": v, "unit": "pair-evals/s", "cores": cores, "kind": "oracle",
                               "sample": "FP64 CPU oracle, nodal forces of %d random nodes (%d target segments) "
                                         "against all %d sources, %.1f s" % (k, 2 * k, n, secs)}
    if rank == 0:
        emit(out)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
