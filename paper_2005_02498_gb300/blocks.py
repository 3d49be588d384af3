"""Block-level front end of the DD-continuum coupling (Sec. 4.2, 4.2.1):
one DD box per stress-averaging block, all advanced together as one batch.

    python -m paper_2005_02498_gb300.blocks --side 3 --increments 4

The continuum solver hands over, at increment k, the Gauss-point stresses;
per block r:
  * <T>^k_r, their volume average over the block (ptadd_block_average);
  * the PTA stress pair T^_{r,t-Delta} = <T>^k_r and the extrapolation
    T^_{r,t} = <T>^k_r + (Delta*/dt^{k-1})(<T>^k_r - <T>^{k-1}_r), with the
    gap raised to 0.5 MPa when it is smaller, mag > 1 recording by how much
    (ptadd_block_stress_pair);
  * a burst at T^_{t-Delta} until the running averages converge, then one
    at T^_t from where it ended (all blocks in lock step: a phase ends at the
    first chunk after which every block's averages moved by less than the
    tolerances, or at the cap);
  * Lpdot_r = (R^Lp_t - R^Lp_{t-Delta}) / Delta* / mag_r, rhodot likewise;
  * Lp^k_r = Lp^{k-1}_r + Lpdot^{k-1}_r dt^{k-1}; a block at the limit
    condition |Lp^k_r| Delta* >= 0.002 keeps its Lp (Lpdot^k_r = 0) and the
    load stops rising.  The polar-velocity part of that condition is left
    out: the burst does not compute V.
The continuum solve itself (alpha, chi, z, u) is not part of this package;
`stress_step_control` takes it as a callback for the paper's stress-based
time step rule, and `run_synthetic` stands in for it with a prescribed
stress field.
"""

from __future__ import annotations

import argparse
import dataclasses
import json

import numpy as np

from . import ptadd
from . import workloads as W


@dataclasses.dataclass
class BlockParams:
    delta_star: float = 0.1      # Delta* = n a with n = 100, a = 1e-3 s
    gap_min: float = 0.5e6       # Pa, smallest stress gap handed to PTA
    stress_jump: float = 3e6     # Pa, largest block stress change per increment
    strain_step: float = 0.002   # plastic strain bound of one increment
    dt: float = 5e-13            # DD time step, s
    chunk: int = 20              # DD steps between convergence checks
    tol_lp: float = 2e-2
    tol_rho: float = 1e-3
    max_chunks: int = 10


def _norms(Lp):
    return np.sqrt(np.einsum("rij,rij->r", Lp, Lp))


class BlockPTA:
    """The DD boxes of n_blocks blocks, all starting from the microstructure
    `net`, in one batch of `ctx`."""

    def __init__(self, ctx, net, n_blocks, p):
        self.ctx, self.p, self.R = ctx, p, int(n_blocks)
        ctx.batch_set(W.batch_from_networks([net.copy() for _ in range(self.R)]))
        self.Lp = np.zeros((self.R, 3, 3))
        self.Lpdot = np.zeros((self.R, 3, 3))

    def _phase(self, sig):
        p, ctx = self.p, self.ctx
        ctx.batch_set_stress(sig)
        sum_lp, sum_rho, n, prev = np.zeros((self.R, 3, 3)), np.zeros(self.R), 0, None
        while n < p.max_chunks:
            lp, rho = ctx.batch_advance(p.chunk, p.dt)
            sum_lp += lp
            sum_rho += rho
            n += 1
            cur = (sum_lp / n, sum_rho / n)
            if prev is not None:
                ok_lp = _norms(cur[0] - prev[0]) <= p.tol_lp * _norms(cur[0])
                ok_rho = np.abs(cur[1] - prev[1]) <= p.tol_rho * np.abs(cur[1])
                if np.all(ok_lp & ok_rho):
                    break
            prev = cur
        return sum_lp / n, sum_rho / n, n

    def increment(self, T_k, T_km1, dt_prev):
        """One coupling increment.  T_k, T_km1: block stresses [R, 6] (Pa,
        Voigt) at increments k and k-1 (T_km1 None: no extrapolation);
        dt_prev: dt^{k-1} (s).  Returns the record of the increment."""
        p = self.p
        T_prev, T_t, mag = ptadd.block_stress_pair(T_k, T_km1, p.delta_star, dt_prev, p.gap_min)
        R1, rho1, n1 = self._phase(T_prev)
        R2, rho2, n2 = self._phase(T_t)
        lpdot = (R2 - R1) / p.delta_star / mag[:, None, None]
        rhodot = (rho2 - rho1) / p.delta_star / mag
        self.Lp = self.Lp + self.Lpdot * dt_prev
        limit = _norms(self.Lp) * p.delta_star >= p.strain_step
        lpdot[limit] = 0.0
        rhodot[limit] = 0.0
        self.Lpdot = lpdot
        return {"T_prev": T_prev, "T_t": T_t, "mag": mag, "R_prev": R1, "R_t": R2, "rho_prev": rho1,
                "rho_t": rho2, "Lpdot": lpdot, "rhodot": rhodot, "Lp": self.Lp.copy(), "limit": limit,
                "load_on": not limit.any(), "chunks": [n1, n2]}


def stress_step_control(solve, T_k, dt, p):
    """The stress-based time step rule of the coupling: solve(dt) returns the
    block stresses [R, 6] at the end of an increment of length dt; while
    some block's stress changes by more than p.stress_jump, the increment is
    redone with half the step, but never below Delta*.  Returns (dt, T_next).
    The DD bursts of an increment do not depend on its own dt, so only the
    solve is repeated."""
    while True:
        T_next = solve(dt)
        change = np.sqrt(np.sum((T_next - T_k)[:, :3] ** 2, 1) + 2 * np.sum((T_next - T_k)[:, 3:] ** 2, 1))
        if change.max() <= p.stress_jump or dt <= p.delta_star:
            return dt, T_next
        dt = max(0.5 * dt, p.delta_star)


def synthetic_mesh(side, elems=4, block_edge=1e-6, thickness=1e-6):
    """A side x side array of square blocks (edge block_edge, the sample's
    thickness), each split into elems x elems square elements with 2 x 2
    Gauss points.  Returns (points [n, 2], weights [n], block [n])."""
    g = 0.5 / np.sqrt(3.0)
    h = block_edge / elems
    pts, w, blk = [], [], []
    for by in range(side):
        for bx in range(side):
            for ey in range(elems):
                for ex in range(elems):
                    cx, cy = bx * block_edge + (ex + 0.5) * h, by * block_edge + (ey + 0.5) * h
                    for sy in (-g, g):
                        for sx in (-g, g):
                            pts.append((cx + sx * h, cy + sy * h))
                            w.append(0.25 * h * h * thickness)
                            blk.append(by * side + bx)
    return np.array(pts), np.array(w), np.array(blk, np.int32)


def bending_field(points, load, gradient, height):
    """Uniaxial stress along x that varies linearly across the sample's
    height: sigma_xx = load (1 + gradient (y / height - 1/2)); Voigt [n, 6]."""
    out = np.zeros((len(points), 6))
    out[:, 0] = load * (1.0 + gradient * (points[:, 1] / height - 0.5))
    return out


def run_synthetic(ctx, net, p, side=3, increments=4, rate=1e6, gradient=0.5, dt0=1.0, load0=20e6):
    """Coupling increments on a side x side block array under a prescribed
    stress field that rises at `rate` (Pa/s) while the load is on; the
    prescribed field stands in for the continuum solve."""
    pts, w, blk = synthetic_mesh(side)
    height = side * 1e-6
    n_blocks = side * side
    box = BlockPTA(ctx, net, n_blocks, p)
    load = load0
    T_k = ptadd.block_average(bending_field(pts, load, gradient, height), w, blk, n_blocks)
    T_km1, dt_prev, t, out = None, 0.0, 0.0, []
    for _ in range(increments):
        rec = box.increment(T_k, T_km1, dt_prev)
        step = p.delta_star if not rec["load_on"] else dt0
        rise = rate if rec["load_on"] else 0.0
        dt, T_next = stress_step_control(
            lambda h: ptadd.block_average(bending_field(pts, load + rise * h, gradient, height), w, blk, n_blocks),
            T_k, step, p)
        out.append({"t": t, "dt": dt, "load": load, "chunks": rec["chunks"],
                    "mag": [float(m) if np.isfinite(m) else None for m in rec["mag"]],  # None: no gap
                    "Lpdot_norm": _norms(rec["Lpdot"]).tolist(), "Lp_norm": _norms(rec["Lp"]).tolist(),
                    "limit": rec["limit"].tolist()})
        load += rise * dt
        t += dt
        T_km1, T_k, dt_prev = T_k, T_next, dt
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--side", type=int, default=3)
    ap.add_argument("--increments", type=int, default=4)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--device", type=int, default=0)
    a = ap.parse_args(argv)
    prec = ptadd.PTADD_FP64 if a.precision == "fp64" else ptadd.PTADD_MIXED
    with ptadd.Context(W.Material().as_tuple(), prec, a.device) as ctx:
        recs = run_synthetic(ctx, W.small_loop_network(), BlockParams(), a.side, a.increments)
    print(json.dumps({"workload": "%d x %d blocks, 16 loops (512 segments) each" % (a.side, a.side),
                      "precision": a.precision, "increments": recs}))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
