"""Plain reference of Practical Time Averaging of one DD box (Sec. 3.1),
on top of the oracle's FP64 burst.

TEST INFRASTRUCTURE, like the rest of this package: only the test suite may
use it.  It shares no code with the product's PTA driver; it runs the
single-box slow-time loop of Sec. 3.1 with the same readings (load
l(t) = c1 (t + Delta) along a unit pattern; a running average converges when
one more chunk of DD steps moves it by less than the tolerance; Frobenius
norms; next slow step 0.002 / |R^Lp_t|, at most h_max).

`p` is any object with the attributes rate, pattern, delta, h0, h_max, dt,
chunk, tol_lp, tol_rho, max_chunks, extend_chunks, lpdot_max, max_jumps,
strain_step.  Returns one record per slow step (t, load, Lp, rho, Lp_prev,
Lpdot, rhodot, jumps, chunks, extended).
"""

from __future__ import annotations

import numpy as np

from . import burst


def _stress(p, t):
    return p.rate * (t + p.delta) * np.asarray(p.pattern, float)


def _net_at(net, xyz, sig):
    m = net.copy()
    m.xyz = xyz.copy()
    m.sig_app = sig
    return m


def _average_until_converged(mat, net, xyz, sig, p):
    """Chunks of p.chunk steps from positions xyz under stress sig; stops when
    a chunk changes the running averages by less than the tolerances, or
    after p.max_chunks chunks.  Returns (sum of chunk Lp, sum of chunk rho,
    chunks, end positions)."""
    sL, sr, n = np.zeros((3, 3)), 0.0, 0
    last = None
    while n < p.max_chunks:
        r = burst(mat, _net_at(net, xyz, sig), p.chunk, p.dt)
        xyz = r["xyz"]
        sL, sr, n = sL + r["Lp_avg"], sr + r["rho_avg"], n + 1
        RL, Rr = sL / n, sr / n
        if last is not None:
            if (np.linalg.norm(RL - last[0]) <= p.tol_lp * np.linalg.norm(RL)
                    and abs(Rr - last[1]) <= p.tol_rho * abs(Rr)):
                break
        last = (RL, Rr)
    return sL, sr, n, xyz


def run(mat, net, p, slow_steps):
    xyz = net.xyz.copy()
    t = 0.0
    h = p.h0
    records = []
    for _ in range(slow_steps):
        jumps = 0
        while True:
            # converged averages at l(t - Delta) from the carried microstructure
            sL1, sr1, n1, x1 = _average_until_converged(mat, net, xyz, _stress(p, t - p.delta), p)
            # then at l(t), from where that burst stopped
            sL2, sr2, n2, x2 = _average_until_converged(mat, net, x1, _stress(p, t), p)
            # difference quotient of the two averages
            lpdot = (sL2 / n2 - sL1 / n1) / p.delta
            # a jump restarts the pair from the state the l(t) burst ended in
            if np.linalg.norm(lpdot) > p.lpdot_max and jumps < p.max_jumps:
                xyz = x2
                jumps += 1
                continue
            break
        # extend the t - Delta average while it exceeds the t average
        ext = 0
        xe = x1
        while np.linalg.norm(sL1 / n1) > np.linalg.norm(sL2 / n2) and ext < p.extend_chunks:
            r = burst(mat, _net_at(net, xe, _stress(p, t - p.delta)), p.chunk, p.dt)
            xe = r["xyz"]
            sL1, sr1, n1 = sL1 + r["Lp_avg"], sr1 + r["rho_avg"], n1 + 1
            ext += 1
        lpdot = (sL2 / n2 - sL1 / n1) / p.delta
        rhodot = (sr2 / n2 - sr1 / n1) / p.delta
        records.append({"t": t, "load": float(p.rate * (t + p.delta)), "Lp": sL2 / n2, "rho": sr2 / n2,
                        "Lp_prev": sL1 / n1, "Lpdot": lpdot, "rhodot": rhodot, "jumps": jumps,
                        "chunks": [n1 - ext, n2], "extended": ext})
        # slow time step from the strain-step bound
        h = min(p.h_max, p.strain_step / max(np.linalg.norm(sL2 / n2), 1e-300))
        xyz = x2
        t += h
    return records
