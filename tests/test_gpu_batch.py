"""GPU parity of the batched ensemble (persistent pair kernel over a
cost-sorted work list, CUDA-graph step loop) against the FP64 CPU oracle run
on every realisation separately, plus the autotuner and its cache."""

import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2005_02498_gb300 import ptadd
from paper_2005_02498_gb300 import workloads as W

pytestmark = pytest.mark.gpu
MAT = W.Material().as_tuple()


def relmax(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(b)))


def relfro(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def uneven_networks():
    """Six realisations of uneven size: 1-5 loops, 23 or 32 nodes, pinned loops, own stresses."""
    rng = np.random.default_rng(77)
    nets = []
    for r, (nl, npl) in enumerate([(1, 32), (5, 32), (3, 23), (2, 32), (4, 23), (1, 23)]):
        nt = W.loop_ensemble(500 + r, nl, 0.5e-6, rng.uniform(-150e6, 150e6, size=6), nodes_per_loop=npl)
        if nl >= 3:
            nt.pinned[:npl] = 1  # first loop sessile
        nets.append(nt)
    return nets


@pytest.mark.parametrize("steps", [1, 4, 5])
def test_batch_fp64_matches_oracle_per_realisation(steps):
    nets = uneven_networks()
    batch = W.batch_from_networks(nets)
    dt = 5e-13
    with ptadd.Context(MAT, ptadd.PTADD_FP64, 0) as c:
        c.batch_set(batch)
        Lp, rho = c.batch_advance(steps, dt)
        x = c.batch_get_nodes()
    for r, nt in enumerate(nets):
        ref = O.burst(MAT, nt, steps, dt)
        n0, n1 = batch.node_off[r], batch.node_off[r + 1]
        assert relmax(x[n0:n1], ref["xyz"]) <= 1e-9
        assert relmax(x[n0:n1] - nt.xyz, ref["xyz"] - nt.xyz) <= 1e-9
        assert relmax(Lp[r], ref["Lp_avg"]) <= 1e-9
        assert abs(rho[r] / ref["rho_avg"] - 1) <= 1e-12


def test_batch_mixed_rates_within_one_percent():
    nets = uneven_networks()
    batch = W.batch_from_networks(nets)
    dt = 5e-13
    with ptadd.Context(MAT, ptadd.PTADD_MIXED, 0) as c:
        c.batch_set(batch)
        Lp, rho = c.batch_advance(20, dt)
    for r, nt in enumerate(nets):
        ref = O.burst(MAT, nt, 20, dt)
        assert relfro(Lp[r], ref["Lp_avg"]) <= 1e-2
        assert abs(rho[r] / ref["rho_avg"] - 1) <= 1e-6


def test_batch_graph_replay_is_deterministic_and_resumable():
    nets = uneven_networks()
    batch = W.batch_from_networks(nets)
    dt = 1e-12
    with ptadd.Context(MAT, ptadd.PTADD_MIXED, 0) as c:
        c.batch_set(batch)
        c.batch_advance(7, dt)
        x7 = c.batch_get_nodes()
        c.batch_set_nodes(batch.xyz)
        c.batch_advance(2, dt)
        c.batch_advance(5, dt)
        x25 = c.batch_get_nodes()
    assert np.array_equal(x7, x25)


def test_batch_autotune_writes_cache_and_keeps_results(tmp_path):
    bt = W.batch_ensemble(1003, R=6, n_min=256, n_max=2048, loops_per_um3=16.0)
    cache = str(tmp_path / "tune.jsonl")
    dt = 5e-13
    with ptadd.Context(MAT, ptadd.PTADD_MIXED, 0) as c:
        c.batch_set(bt)
        Lp0, _ = c.batch_advance(3, dt)
        assert c.batch_info()["tuned"] in (0, 1)
        c.batch_set_nodes(bt.xyz)
        c.batch_autotune(cache, force=True)
        info = c.batch_info()
        assert info["tuned"] == 1 and info["tile_targets"] in (64, 128)
        assert info["chunk_sources"] in (1024, 2048, 4096)
        Lp1, _ = c.batch_advance(3, dt)
    lines = [json.loads(l) for l in open(cache)]
    assert len(lines) == 1 and lines[0]["tpb"] == info["tile_targets"]
    for r in range(bt.R):
        assert relfro(Lp1[r], Lp0[r]) <= 1e-5
    # a second batch of the same size class picks the cached entry up at set time
    os.environ["PTADD_TUNE_CACHE"] = cache
    try:
        with ptadd.Context(MAT, ptadd.PTADD_MIXED, 0) as c:
            c.batch_set(bt)
            assert c.batch_info()["tuned"] == 1
    finally:
        del os.environ["PTADD_TUNE_CACHE"]


def test_batch_set_stress_and_errors():
    nets = uneven_networks()
    batch = W.batch_from_networks(nets)
    with ptadd.Context(MAT, ptadd.PTADD_FP64, 0) as c:
        with pytest.raises(ptadd.PtaddError) as e:
            ptadd._check(c._lib.ptadd_batch_advance(c._h, 1, 1e-12, None, None))
        assert e.value.status == 5
        bad = W.batch_from_networks(nets)
        bad.loop_off = bad.loop_off.copy()
        bad.loop_off[1] = bad.node_off[1] + 1  # first loop runs into realisation 1
        with pytest.raises(ptadd.PtaddError):
            c.batch_set(bad)
        c.batch_set(batch)
        sig = np.zeros((batch.R, 6))
        c.batch_set_stress(sig)
        Lp, _ = c.batch_advance(2, 1e-12)
    # zero applied stress: only self/interaction stresses drive the loops
    ref = O.burst(MAT, W.Network(nets[1].xyz, nets[1].loop_off, nets[1].burgers, nets[1].normal,
                                 nets[1].pinned, nets[1].volume, np.zeros(6)), 2, 1e-12)
    assert relmax(Lp[1], ref["Lp_avg"]) <= 1e-9
