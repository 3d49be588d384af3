"""ptadd_forces_noalloc: nodal forces computed without any device allocation.

Some callers cannot call cudaMalloc: code running under another framework's
memory pool (which owns the device memory budget) and latency-critical loops
where cudaMalloc's implicit device synchronisation would stall other streams.
For them the library offers one entry point whose scratch is a fixed array in
the library's own device memory.  Here it is called through the C ABI on
device buffers the test owns, and compared with the context-based
ptadd_get_forces within the force tolerance of the parity tests (1e-11
relative max-norm), on two different networks in a row and once more on the
first (the shared scratch must carry nothing over between calls).

This file is named so pytest collects it last.
"""

import numpy as np
import pytest

from paper_2005_02498_gb300 import ptadd
from paper_2005_02498_gb300 import workloads as W

pytestmark = pytest.mark.gpu
MAT = W.Material().as_tuple()


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def ring_tables(net):
    n = net.n_nodes
    nxt = np.empty(n, np.int32)
    prv = np.empty(n, np.int32)
    for k in range(net.n_loops):
        idx = np.arange(net.loop_off[k], net.loop_off[k + 1])
        nxt[idx] = np.roll(idx, -1)
        prv[idx] = np.roll(idx, 1)
    counts = np.diff(net.loop_off)
    bseg = np.repeat(net.burgers, counts, axis=0)
    return nxt, prv, np.ascontiguousarray(bseg)


def forces_noalloc(net):
    import torch
    dev = torch.device("cuda", 0)
    nxt, prv, bseg = ring_tables(net)
    x = torch.from_numpy(np.ascontiguousarray(net.xyz)).to(dev)
    tn = torch.from_numpy(nxt).to(dev)
    tp = torch.from_numpy(prv).to(dev)
    tb = torch.from_numpy(bseg).to(dev)
    F = torch.full((net.n_nodes, 3), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    ptadd.forces_noalloc(MAT, net.n_nodes, x.data_ptr(), tn.data_ptr(), tp.data_ptr(), tb.data_ptr(),
                         net.sig_app, F.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    return F.cpu().numpy()


def forces_context(net):
    with ptadd.Context(MAT, ptadd.PTADD_FP64, 0) as c:
        c.set_network(net)
        return c.get_forces()


def test_noalloc_forces_match_context_forces_on_consecutive_calls():
    a = W.medium_loop_network()
    b = W.loop_ensemble(33, 13, 0.6e-6, np.array([20e6, -35e6, 50e6, 10e6, -5e6, 25e6]), nodes_per_loop=23)
    Fa1 = forces_noalloc(a)
    Fb = forces_noalloc(b)
    Fa2 = forces_noalloc(a)
    assert np.all(np.isfinite(Fa1)) and np.all(np.isfinite(Fb))
    assert relmax(Fa1, forces_context(a)) <= 1e-11
    assert relmax(Fb, forces_context(b)) <= 1e-11
    assert np.array_equal(Fa1, Fa2)


def test_noalloc_rejects_networks_beyond_its_scratch():
    import torch
    dev = torch.device("cuda", 0)
    small = torch.zeros(16, dtype=torch.float64, device=dev)
    idx = torch.zeros(16, dtype=torch.int32, device=dev)
    with pytest.raises(ptadd.PtaddError) as e:
        ptadd.forces_noalloc(MAT, ptadd.NOALLOC_MAX_SEGMENTS + 1, small.data_ptr(), idx.data_ptr(),
                             idx.data_ptr(), small.data_ptr(), np.zeros(6), small.data_ptr())
    assert e.value.status == 1
    assert "scratch" in str(e.value)


def test_noalloc_rejects_broken_loop_tables_without_touching_memory_outside_them():
    # The tables are checked on the device before any kernel indexes with
    # them: an entry outside [0, n) or one that breaks prv[nxt[i]] == i is
    # never used as an index, and the call writes NaN to every output force.
    # A valid call afterwards is unaffected.
    import torch
    dev = torch.device("cuda", 0)
    net = W.small_loop_network()
    nxt, prv, bseg = ring_tables(net)
    x = torch.from_numpy(np.ascontiguousarray(net.xyz)).to(dev)
    tb = torch.from_numpy(bseg).to(dev)
    stream = torch.cuda.current_stream()
    for bad_nxt, bad_prv in [(7, None), (None, 2), (None, None)]:
        n2, p2 = nxt.copy(), prv.copy()
        if bad_nxt is not None:
            n2[bad_nxt] = net.n_nodes + 1000  # out of range
        if bad_prv is not None:
            p2[bad_prv] = -5  # out of range
        if bad_nxt is None and bad_prv is None:
            n2[3], n2[4] = n2[4], n2[3]  # in range, but prv[nxt[i]] != i
        tn = torch.from_numpy(n2).to(dev)
        tp = torch.from_numpy(p2).to(dev)
        F = torch.zeros((net.n_nodes, 3), dtype=torch.float64, device=dev)
        ptadd.forces_noalloc(MAT, net.n_nodes, x.data_ptr(), tn.data_ptr(), tp.data_ptr(), tb.data_ptr(),
                             net.sig_app, F.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        assert torch.isnan(F).all()
    F_ok = forces_noalloc(net)
    assert relmax(F_ok, forces_context(net)) <= 1e-11
