"""GPU parity of the polar dislocation velocity (Sec. 2.4, Eq. 2.11), summed
in the same reduction as Lp and rho in every DD step and averaged over the
burst (Eq. 2.5), against the FP64 CPU oracle.

Bars as for the averaged rates: <= 1e-9 relative (max-norm of the 3-vector,
against max |V| of the oracle) in FP64, <= 1 % in the mixed path.  The core
cross-section A is a caller parameter (the paper takes it as |b|^2 up to a
constant); V is linear in it.
"""

import numpy as np
import pytest

import oracle as O
from paper_2005_02498_gb300 import ptadd
from paper_2005_02498_gb300 import workloads as W

pytestmark = pytest.mark.gpu
MAT = W.Material().as_tuple()
CORE = W.Material().b ** 2


def relmax(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(b)))


def net_with_drift(seed=41):
    """Loops with some pinned nodes (partly pinned loops move off-centre, so V is not 0)."""
    net = W.loop_ensemble(seed, 9, 0.6e-6, np.array([40e6, -25e6, 60e6, 15e6, -10e6, 30e6]), nodes_per_loop=23)
    for k in range(9):
        net.pinned[23 * k:23 * k + 6 + k] = 1
    return net


@pytest.mark.parametrize("prec,tol", [(ptadd.PTADD_FP64, 1e-9), (ptadd.PTADD_MIXED, 1e-2)])
def test_burst_polar_velocity_matches_oracle(prec, tol):
    net = net_with_drift()
    dt, steps = 5e-13, 20
    ref = O.burst(MAT, net, steps, dt, core_area=CORE)
    with ptadd.Context(MAT, prec, 0) as c:
        c.set_network(net)
        with pytest.raises(ptadd.PtaddError) as e:
            c.get_polar_velocity(CORE)
        assert e.value.status == 5  # no burst yet
        c.advance(steps, dt)
        V = c.get_polar_velocity(CORE)
        V2 = c.get_polar_velocity(3 * CORE)
        with pytest.raises(ptadd.PtaddError):
            c.get_polar_velocity(-1.0)
    assert np.linalg.norm(ref["V_avg"]) > 0
    assert relmax(V, ref["V_avg"]) <= tol
    assert np.array_equal(V2, 3 * V) or relmax(V2, 3 * V) <= 1e-15


def test_batch_polar_velocity_matches_oracle_per_realisation():
    nets = [net_with_drift(50 + r) for r in range(4)]
    batch = W.batch_from_networks(nets)
    dt, steps = 5e-13, 6
    with ptadd.Context(MAT, ptadd.PTADD_FP64, 0) as c:
        c.batch_set(batch)
        with pytest.raises(ptadd.PtaddError):
            c.batch_get_polar_velocity(CORE)
        c.batch_advance(steps, dt)
        V = c.batch_get_polar_velocity(CORE)
    for r, nt in enumerate(nets):
        ref = O.burst(MAT, nt, steps, dt, core_area=CORE)
        assert relmax(V[r], ref["V_avg"]) <= 1e-9


def test_dissipation_projection_on_the_device_equals_the_host_function():
    """The device kernel over many material points against the host entry
    point point by point (the host one is pinned by tests/test_projection.py);
    a point with a non-finite value is left as it is and counted."""
    import torch
    rng = np.random.default_rng(9)
    n = 5000
    T6 = rng.normal(size=(n, 6)) * 1e8
    Lp = rng.normal(size=(n, 9)) * 1e3
    alpha = rng.normal(size=(n, 9)) * 1e12
    V = rng.normal(size=(n, 3))
    T6[17, 2] = np.nan
    dev = torch.device("cuda", 0)
    tT, tL, ta, tV = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (T6, Lp, alpha, V))
    bad = torch.zeros(1, dtype=torch.int32, device=dev)
    ptadd.dissipation_projection_dev(n, tT.data_ptr(), tL.data_ptr(), ta.data_ptr(), tV.data_ptr(), bad.data_ptr())
    torch.cuda.synchronize()
    Lg, Vg = tL.cpu().numpy(), tV.cpu().numpy()
    assert int(bad.item()) == 1
    assert np.array_equal(Lg[17], Lp[17]) and np.array_equal(Vg[17], V[17])
    changed = 0
    for p in range(n):
        if p == 17:
            continue
        Lh, Vh = ptadd.dissipation_projection(T6[p], Lp[p].reshape(3, 3), V[p], alpha[p].reshape(3, 3))
        assert np.allclose(Lg[p], Lh.reshape(9), rtol=1e-13, atol=1e-13 * np.abs(Lp[p]).max())
        assert np.allclose(Vg[p], Vh, rtol=1e-13, atol=1e-13 * np.abs(V[p]).max())
        changed += int(not np.array_equal(Lh.reshape(9), Lp[p]))
    assert 1000 < changed < n  # about half the random points dissipate negatively
