"""GPU parity of the batched ensemble at the sizes of the batched workload
(realisations of 1k-16k segments, uneven, each with its own applied stress
and its own sessile loops), against the FP64 CPU oracle run on every
realisation separately.

The pair stage is forced to split every realisation into source chunks of
1024 segments (tiles of 64 or 128 targets), so the per-chunk offsets of the
work items and the node stage's sum over chunks are exercised: up to 16
chunks per realisation, with a ragged last chunk.  Forces are compared at
sampled nodes (chunk boundaries, loop ends and random ones); positions and
averaged rates after a short burst on the two smaller realisations.
"""

import functools

import numpy as np
import pytest

import oracle as O
from paper_2005_02498_gb300 import ptadd
from paper_2005_02498_gb300 import workloads as W

pytestmark = pytest.mark.gpu
MAT = W.Material().as_tuple()
SIZES = [1024, 4256, 8192, 16384]  # segments; 4256 = 4 chunks of 1024 and a ragged one of 160
CHUNK = 1024
STEPS = 3
DT = 5e-13


def relmax(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(b)))


def relfro(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def n_targets(nt):
    """Segments i -> nxt[i] with at least one unpinned node (the burst's targets)."""
    pin = nt.pinned.astype(bool)
    count = 0
    for k in range(nt.n_loops):
        idx = np.arange(nt.loop_off[k], nt.loop_off[k + 1])
        count += int(np.sum(~(pin[idx] & pin[np.roll(idx, -1)])))
    return count


@functools.lru_cache(maxsize=None)
def networks():
    nets = []
    for r, n in enumerate(SIZES):
        # the batched-workload recipe, one realisation of a fixed size per seed
        bt = W.batch_ensemble(2100 + r, R=1, n_min=n, n_max=n, sessile_min=0.3, sessile_max=0.5)
        nt = bt.realisation(0)
        assert nt.n_nodes == n and 0 < nt.pinned.sum() < n
        nets.append(nt)
    return nets


@functools.lru_cache(maxsize=None)
def samples():
    """Per realisation: unpinned nodes at chunk boundaries, loop ends and random."""
    rng = np.random.default_rng(2099)
    out = []
    for nt in networks():
        n = nt.n_nodes
        cand = set()
        for c in range(0, n, CHUNK):
            cand.update({c - 1, c, c + 1})
        cand.update(int(v) for v in nt.loop_off[:-1])
        cand.update(int(v) for v in rng.integers(0, n, size=40))
        sel = np.array(sorted(i for i in cand if 0 <= i < n and not nt.pinned[i]), np.int64)
        assert sel.size >= 30
        out.append(sel)
    return out


@functools.lru_cache(maxsize=None)
def oracle_forces():
    return [O.nodal_forces_subset(MAT, nt, sel) for nt, sel in zip(networks(), samples())]


@functools.lru_cache(maxsize=None)
def oracle_bursts():
    return [O.burst(MAT, nt, STEPS, DT) for nt in networks()[:2]]


@pytest.mark.parametrize("precision,tpb", [(ptadd.PTADD_FP64, 64), (ptadd.PTADD_FP64, 128),
                                           (ptadd.PTADD_MIXED, 64), (ptadd.PTADD_MIXED, 128)])
def test_full_size_batch_matches_oracle(precision, tpb):
    nets = networks()
    batch = W.batch_from_networks(nets)
    fp64 = precision == ptadd.PTADD_FP64
    with ptadd.Context(MAT, precision, 0) as c:
        c.batch_set(batch)
        c.batch_configure(tpb, CHUNK)
        info = c.batch_info()
        assert info["tile_targets"] == tpb and info["chunk_sources"] == CHUNK and info["tuned"] == 0
        # every realisation beyond the first spans several source chunks
        n_t = [n_targets(nt) for nt in nets]
        expect_items = sum(-(-t // tpb) * -(-nt.n_nodes // CHUNK) for t, nt in zip(n_t, nets))
        assert info["work_items"] == expect_items
        F = c.batch_get_forces()
        Lp, rho = c.batch_advance(STEPS, DT)
        x = c.batch_get_nodes()
    for r, (nt, sel, Fo) in enumerate(zip(nets, samples(), oracle_forces())):
        n0 = batch.node_off[r]
        ef = relmax(F[n0 + sel], Fo)
        assert ef <= (1e-11 if fp64 else 1e-4), (r, ef)
        assert np.all(F[n0:n0 + nt.n_nodes][nt.pinned.astype(bool)] == 0.0)
    for r, ref in enumerate(oracle_bursts()):
        nt = nets[r]
        n0, n1 = batch.node_off[r], batch.node_off[r + 1]
        if fp64:
            assert relmax(x[n0:n1], ref["xyz"]) <= 1e-9
            assert relmax(x[n0:n1] - nt.xyz, ref["xyz"] - nt.xyz) <= 1e-9
            assert relmax(Lp[r], ref["Lp_avg"]) <= 1e-9
            assert abs(rho[r] / ref["rho_avg"] - 1) <= 1e-12
        else:
            assert relfro(Lp[r], ref["Lp_avg"]) <= 1e-2
            assert relmax(x[n0:n1] - nt.xyz, ref["xyz"] - nt.xyz) <= 1e-4
            assert abs(rho[r] / ref["rho_avg"] - 1) <= 1e-6


def test_batch_configure_rejects_unsupported_tiles():
    nets = networks()[:1]
    with ptadd.Context(MAT, ptadd.PTADD_FP64, 0) as c:
        with pytest.raises(ptadd.PtaddError) as e:
            c.batch_configure(128, CHUNK)
        assert e.value.status == 5  # no batch loaded
        c.batch_set(W.batch_from_networks(nets))
        for tpb, ch in [(96, CHUNK), (128, 512), (64, 1000)]:
            with pytest.raises(ptadd.PtaddError) as e:
                c.batch_configure(tpb, ch)
            assert e.value.status == 1
