"""Argument and state checks of the closure sweep (ptadd_closure_sweep).
Its dispatch (surrogate inside the trust region, DD ensembles outside it) is
checked with a surrogate fitted on DD closures in
tests/test_gpu_surrogate_closure.py."""

import numpy as np
import pytest

from paper_2005_02498_gb300 import ptadd
from paper_2005_02498_gb300 import workloads as W

pytestmark = pytest.mark.gpu
MAT = W.Material().as_tuple()


def test_closure_sweep_needs_a_fitted_surrogate_and_valid_sizes():
    with ptadd.Context(MAT, ptadd.PTADD_MIXED, 0) as c:
        with pytest.raises(ptadd.PtaddError):
            c.closure_sweep(np.zeros((1, 6)), np.ones((1, 24)) * 1e12, 2, 256, 4, 5e-13, 1)
        with pytest.raises(ptadd.PtaddError):
            c.closure_sweep(np.zeros((1, 6)), np.ones((1, 24)) * 1e12, 2, 100, 4, 5e-13, 1)  # not a multiple of 32
