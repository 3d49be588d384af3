"""Plain reference of the block-level front end of the DD-continuum coupling
(Sec. 4.2 and 4.2.1), on top of the oracle's FP64 burst.

TEST INFRASTRUCTURE, like the rest of this package: only the test suite may
use it.  It shares no code with the product's block driver.  Tensors are
handled as full 3x3 matrices here (the product works on Voigt vectors).

Readings, the same as the product's:
  * <T>_r is the quadrature of the volume integral over the block divided by
    the block's volume, both with the same Gauss weights;
  * |.| of a stress is the Frobenius norm of the full tensor;
  * a zero stress gap has no direction to inflate along: T^_t = T^_{t-Delta}
    and mag = inf, so the rescaled rates are 0;
  * every block's DD box runs in lock step: a phase (the burst at
    T^_{t-Delta}, then the one at T^_t, which starts where the first ended)
    ends after the first chunk at which every block's running averages moved
    by less than the tolerances, or after max_chunks chunks;
  * Lpdot_r = (R^Lp_{r,t} - R^Lp_{r,t-Delta}) / Delta* / mag_r (Eq. 2.8 with
    Delta = Delta*, then the rescale);
  * Lp^k_r = Lp^{k-1}_r + Lpdot^{k-1}_r dt^{k-1}; a block with
    |Lp^k_r| Delta* >= 0.002 (the limit condition without the polar part,
    which the burst does not compute) keeps Lp: its Lpdot^k is set to 0, and
    the load stops rising.
`p` is any object with the attributes delta_star, gap_min, dt, chunk,
tol_lp, tol_rho, max_chunks, strain_step.
"""

from __future__ import annotations

import numpy as np

from . import burst


def _full(v):
    return np.array([[v[0], v[5], v[4]], [v[5], v[1], v[3]], [v[4], v[3], v[2]]], dtype=float)


def _voigt(T):
    return np.array([T[0, 0], T[1, 1], T[2, 2], T[1, 2], T[0, 2], T[0, 1]])


def block_average(T6, w, block, n_blocks):
    """<T>_r = (integral of T over block r) / |block r| (Sec. 4.2), both by
    the Gauss rule sum_g w_g f(x_g) over the points of the block."""
    out = np.zeros((n_blocks, 6))
    for r in range(n_blocks):
        integral = np.zeros((3, 3))
        volume = 0.0
        for g in range(len(w)):
            if block[g] == r:
                integral += w[g] * _full(T6[g])
                volume += w[g]
        out[r] = _voigt(integral / volume)
    return out


def stress_pair(T_k, T_km1, delta_star, dt_prev, gap_min):
    """The stresses of one block's PTA at increment k (Sec. 4.2.1): the
    extrapolated pair and the minimum-gap rule.  Returns (T_prev, T_t, mag)."""
    R = len(T_k)
    T_prev, T_t, mag = np.zeros((R, 6)), np.zeros((R, 6)), np.ones(R)
    for r in range(R):
        A = _full(T_k[r])
        if T_km1 is not None and dt_prev > 0:
            B = A + delta_star / dt_prev * (A - _full(T_km1[r]))
        else:
            B = A.copy()
        gap = np.linalg.norm(B - A)  # Frobenius
        if gap < gap_min:
            if gap == 0.0:
                mag[r] = np.inf
            else:
                mag[r] = gap_min / gap
                B = A + mag[r] * (B - A)
        T_prev[r], T_t[r] = _voigt(A), _voigt(B)
    return T_prev, T_t, mag


def _phase(mat, net, xyz, sig, p, burst_fn):
    """Lock-step chunks of p.chunk DD steps for every block from positions
    xyz[r] under stress sig[r].  Returns (averages Lp [R,3,3], rho [R],
    chunks, end positions)."""
    R = len(xyz)
    sum_lp, sum_rho = np.zeros((R, 3, 3)), np.zeros(R)
    n, last = 0, None
    while n < p.max_chunks:
        for r in range(R):
            m = net.copy()
            m.xyz, m.sig_app = xyz[r].copy(), np.array(sig[r], float)
            b = burst_fn(mat, m, p.chunk, p.dt)
            xyz[r] = b["xyz"]
            sum_lp[r] += b["Lp_avg"]
            sum_rho[r] += b["rho_avg"]
        n += 1
        cur_lp, cur_rho = sum_lp / n, sum_rho / n
        if last is not None:
            done = all(np.linalg.norm(cur_lp[r] - last[0][r]) <= p.tol_lp * np.linalg.norm(cur_lp[r])
                       and abs(cur_rho[r] - last[1][r]) <= p.tol_rho * abs(cur_rho[r]) for r in range(R))
            if done:
                break
        last = (cur_lp, cur_rho)
    return sum_lp / n, sum_rho / n, n, xyz


def increment(mat, net, xyz, state, T_k, T_km1, dt_prev, p, burst_fn=burst):
    """One coupling increment at every block.  xyz: list of the blocks'
    node positions (updated in place); state: dict with Lp [R,3,3] and
    Lpdot [R,3,3] of the previous increment (updated in place).  Returns
    the record of the increment."""
    T_prev, T_t, mag = stress_pair(T_k, T_km1, p.delta_star, dt_prev, p.gap_min)
    R1, r1, n1, xyz = _phase(mat, net, xyz, T_prev, p, burst_fn)
    R2, r2, n2, xyz = _phase(mat, net, xyz, T_t, p, burst_fn)
    R = len(T_k)
    lpdot = np.zeros((R, 3, 3))
    rhodot = np.zeros(R)
    for r in range(R):
        lpdot[r] = (R2[r] - R1[r]) / p.delta_star / mag[r]
        rhodot[r] = (r2[r] - r1[r]) / p.delta_star / mag[r]
    Lp = state["Lp"] + state["Lpdot"] * dt_prev
    limit = np.array([np.linalg.norm(Lp[r]) * p.delta_star >= p.strain_step for r in range(R)])
    for r in range(R):
        if limit[r]:
            lpdot[r] = 0.0
            rhodot[r] = 0.0
    state["Lp"], state["Lpdot"] = Lp, lpdot
    return {"T_prev": T_prev, "T_t": T_t, "mag": mag, "R_prev": R1, "R_t": R2, "rho_prev": r1, "rho_t": r2,
            "Lpdot": lpdot, "rhodot": rhodot, "Lp": Lp, "limit": limit, "load_on": not limit.any(),
            "chunks": [n1, n2]}
