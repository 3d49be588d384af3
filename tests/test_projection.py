"""The non-negative-dissipation correction (Sec. 4): checked against what the
paper states about it (host only, no GPU): the corrected Lp does not
dissipate along T, the removed part is parallel to T, everything orthogonal
to T is untouched, and likewise for V with X(T alpha)."""

import numpy as np
import pytest

from paper_2005_02498_gb300 import ptadd

EPS = np.zeros((3, 3, 3))
for i, j, k in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
    EPS[i, j, k], EPS[i, k, j] = 1.0, -1.0


def _full(t6):
    return np.array([[t6[0], t6[5], t6[4]], [t6[5], t6[1], t6[3]], [t6[4], t6[3], t6[2]]])


def test_lp_projection():
    rng = np.random.default_rng(2)
    for _ in range(200):
        t6 = rng.normal(size=6)
        T = _full(t6)
        Lp = rng.normal(size=(3, 3))
        d = np.sum(T * Lp)
        out, _ = ptadd.dissipation_projection(t6, Lp)
        if d >= 0:
            assert np.array_equal(out, Lp)
            continue
        assert abs(np.sum(T * out)) <= 1e-12 * np.linalg.norm(T) * np.linalg.norm(Lp)
        removed = Lp - out
        assert np.allclose(removed, d * T / np.sum(T * T), rtol=1e-12, atol=1e-15)
        Y = rng.normal(size=(3, 3))
        Y -= np.sum(Y * T) / np.sum(T * T) * T  # orthogonal to T
        assert abs(np.sum(Y * out) - np.sum(Y * Lp)) <= 1e-12 * np.linalg.norm(Y) * np.linalg.norm(Lp)
        again, _ = ptadd.dissipation_projection(t6, out)  # idempotent: no negative dissipation left
        assert np.allclose(again, out, rtol=0, atol=1e-15 * np.linalg.norm(Lp))


def test_v_projection_uses_the_alternating_tensor():
    rng = np.random.default_rng(3)
    hits = 0
    for _ in range(200):
        t6 = rng.normal(size=6)
        alpha = rng.normal(size=(3, 3))
        V = rng.normal(size=3)
        w = np.einsum("ijk,jk->i", EPS, _full(t6) @ alpha)  # X(T alpha)
        beta = V @ w
        _, out = ptadd.dissipation_projection(t6, np.zeros((3, 3)), V, alpha)
        if beta >= 0:
            assert np.array_equal(out, V)
            continue
        hits += 1
        assert abs(out @ w) <= 1e-12 * np.linalg.norm(V) * np.linalg.norm(w)
        assert np.allclose(V - out, beta * w / (w @ w), rtol=1e-12, atol=1e-15)
    assert hits > 50


def test_degenerate_and_bad_inputs():
    Lp = np.arange(9.0).reshape(3, 3) - 4
    out, _ = ptadd.dissipation_projection(np.zeros(6), Lp)
    assert np.array_equal(out, Lp)  # zero stress: nothing to project on
    with pytest.raises(ptadd.PtaddError):
        ptadd.dissipation_projection(np.ones(6), Lp, V=np.ones(3))  # V needs alpha
    with pytest.raises(ptadd.PtaddError):
        ptadd.dissipation_projection(np.array([np.nan, 0, 0, 0, 0, 0]), Lp)
