"""Failure paths through the C ABI, made on the host (no GPU fault):
non-finite inputs are refused before they reach the device, a burst whose
positions overflow reports PTADD_ERR_NONFINITE, a tensor-core wait that can
never complete gives up within its limit and reports PTADD_ERR_TIMEOUT, and
after each of them the context (or the library) keeps giving the results
of a fresh one."""

import numpy as np
import pytest

from paper_2005_02498_gb300 import ptadd
from paper_2005_02498_gb300 import workloads as W

pytestmark = pytest.mark.gpu
MAT = W.Material().as_tuple()
DT = 5e-13
HUGE_DT = 1e300  # finite and positive, so accepted; x + v dt overflows in the first step


def fresh_burst(prec, net, steps):
    with ptadd.Context(MAT, prec, 0) as c:
        c.set_network(net)
        Lp, rho = c.advance(steps, DT)
        return Lp, rho, c.get_nodes()


@pytest.mark.parametrize("prec", [ptadd.PTADD_FP64, ptadd.PTADD_MIXED])
def test_nonfinite_inputs_and_bursts_are_reported_and_the_context_recovers(prec):
    net = W.small_loop_network()
    with ptadd.Context(MAT, prec, 0) as c:
        c.set_network(net)
        bad = net.xyz.copy()
        bad[5, 1] = np.nan
        with pytest.raises(ptadd.PtaddError) as e:
            c.set_nodes(bad)
        assert e.value.status == 1
        with pytest.raises(ptadd.PtaddError) as e:
            c.advance(2, HUGE_DT)
        assert e.value.status == 3
        assert not np.all(np.isfinite(c.get_nodes()))
        c.set_nodes(net.xyz)
        Lp, rho = c.advance(5, DT)
        x = c.get_nodes()
    Lp0, rho0, x0 = fresh_burst(prec, net, 5)
    assert np.array_equal(x, x0) and np.array_equal(Lp, Lp0) and rho == rho0


def test_nonfinite_batch_burst_is_reported_and_the_batch_recovers():
    nets = [W.loop_ensemble(900 + r, 2 + r, 0.5e-6, np.array([50e6, 0, -20e6, 10e6, 0, 30e6])) for r in range(3)]
    batch = W.batch_from_networks(nets)
    with ptadd.Context(MAT, ptadd.PTADD_MIXED, 0) as c:
        c.batch_set(batch)
        bad = batch.xyz.copy()
        bad[0, 0] = np.inf
        with pytest.raises(ptadd.PtaddError) as e:
            c.batch_set_nodes(bad)
        assert e.value.status == 1
        with pytest.raises(ptadd.PtaddError) as e:
            c.batch_advance(3, HUGE_DT)
        assert e.value.status == 3
        c.batch_set_nodes(batch.xyz)
        Lp, rho = c.batch_advance(4, DT)
    with ptadd.Context(MAT, ptadd.PTADD_MIXED, 0) as c:
        c.batch_set(batch)
        Lp0, rho0 = c.batch_advance(4, DT)
    assert np.array_equal(Lp, Lp0) and np.array_equal(rho, rho0)


def test_tensor_core_wait_gives_up_and_the_library_stays_usable():
    assert ptadd.gemm_timeout_selftest(0) == 4  # PTADD_ERR_TIMEOUT
    rng = np.random.default_rng(5)
    A = ptadd.to_bf16_bits(rng.normal(size=(130, 64)).astype(np.float32))
    B = ptadd.to_bf16_bits(rng.normal(size=(32, 64)).astype(np.float32))
    C = ptadd.gemm_bf16(A, B)
    ref = ptadd.from_bf16_bits(A).astype(np.float64) @ ptadd.from_bf16_bits(B).astype(np.float64).T
    assert np.max(np.abs(C - ref)) / np.max(np.abs(ref)) <= 1e-5
