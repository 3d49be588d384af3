"""Seeded synthetic inputs for the dislocation-dynamics burst.

This module only *draws inputs*: node positions of closed glide loops, their
Burgers vectors and glide normals, pinned flags, applied stress tensors and
volumes.  It holds none of the method's arithmetic (no stress field, force,
mobility or averaging), so both the CUDA path and the CPU oracle may take
their inputs from here.

The paper builds its microstructures from boundary-to-boundary segment pairs
(Sec. 3.2.1) with MoDELib; those microstructures are not published.  The
workloads here are ensembles of circular glide loops on the 12 FCC
{111}<110> slip systems:

* node k of a loop sits at c + R (cos phi_k e1 + sin phi_k e2), with
  e1 = b_hat, e2 = n x b_hat, phi_k = 2 pi k / n_nodes + phi_0;
* the line sense is drawn as +-1 (a -1 reverses the node order);
* all lengths are SI metres, stresses Pa, volumes m^3.

Every generator takes an explicit integer seed and uses numpy's PCG64 stream,
so a (seed, arguments) pair fixes the workload bit for bit on any host.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

# --------------------------------------------------------------------------
# Material (the loop-ensemble workloads: isotropic FCC, mu = 48 GPa,
# nu = 0.34, |b| = 0.2556 nm, core width a = |b|, drag B = 1e-4 Pa s).
# --------------------------------------------------------------------------
MU = 48.0e9
NU = 0.34
BURGERS = 2.556e-10
CORE_A = BURGERS
DRAG_B = 1.0e-4
MICRON = 1.0e-6


@dataclasses.dataclass(frozen=True)
class Material:
    mu: float = MU
    nu: float = NU
    b: float = BURGERS
    a: float = CORE_A
    B: float = DRAG_B

    def as_tuple(self):
        return (self.mu, self.nu, self.b, self.a, self.B)


def fcc_slip_systems():
    """The 12 FCC {111}<110> slip systems as unit vectors.

    Returns (b_hat[12,3], n_hat[12,3]); every b_hat lies in its plane
    (b_hat . n_hat = 0).  Order: plane (111), (-111), (1-11), (11-1), and in
    each plane the three <110> directions perpendicular to its normal.
    """
    normals = np.array([[1, 1, 1], [-1, 1, 1], [1, -1, 1], [1, 1, -1]], dtype=np.float64)
    cands = np.array([[0, 1, -1], [1, 0, -1], [1, -1, 0],
                      [0, 1, 1], [1, 0, 1], [1, 1, 0]], dtype=np.float64)
    bs, ns = [], []
    for n in normals:
        for c in cands:
            if c @ n == 0.0:
                bs.append(c / math.sqrt(2.0))
                ns.append(n / math.sqrt(3.0))
    b = np.array(bs)
    n = np.array(ns)
    assert b.shape == (12, 3)
    return b, n


@dataclasses.dataclass
class Network:
    """One realisation: closed loops of straight segments (SI units).

    Loop k owns nodes [loop_off[k], loop_off[k+1]); segment i runs from node i
    to the next node of its loop (wrapping at the loop end).
    """
    xyz: np.ndarray        # [n_nodes, 3] float64, m
    loop_off: np.ndarray   # [n_loops + 1] int64
    burgers: np.ndarray    # [n_loops, 3] float64, m
    normal: np.ndarray     # [n_loops, 3] float64, unit
    pinned: np.ndarray     # [n_nodes] uint8
    volume: float          # m^3
    sig_app: np.ndarray    # [6] Pa, Voigt order xx, yy, zz, yz, xz, xy

    @property
    def n_nodes(self):
        return int(self.xyz.shape[0])

    @property
    def n_loops(self):
        return int(self.loop_off.shape[0] - 1)

    def copy(self):
        return Network(self.xyz.copy(), self.loop_off.copy(), self.burgers.copy(),
                       self.normal.copy(), self.pinned.copy(), float(self.volume),
                       self.sig_app.copy())


def uniaxial_stress(value_pa, axis=2):
    """Voigt stress vector of a uniaxial stress along a cube axis."""
    s = np.zeros(6)
    s[axis] = value_pa
    return s


def circular_loops(rng, n_loops, box_edge, r_min=0.05 * MICRON, r_max=0.2 * MICRON,
                   nodes_per_loop=32, b_mag=BURGERS, systems=None):
    """Draw n_loops circular glide loops (each a regular nodes_per_loop-gon).

    Radius ~ U(r_min, r_max), centre ~ U[0, box_edge)^3, slip system ~ U{12}
    (or drawn from `systems`), phase phi_0 ~ U[0, 2 pi), line sense ~ +-1.
    Returns (xyz, loop_off, burgers, normal).
    """
    bh, nh = fcc_slip_systems()
    if systems is None:
        systems = np.arange(12)
    sys_idx = rng.choice(np.asarray(systems), size=n_loops)
    radius = rng.uniform(r_min, r_max, size=n_loops)
    centre = rng.uniform(0.0, box_edge, size=(n_loops, 3))
    phi0 = rng.uniform(0.0, 2.0 * math.pi, size=n_loops)
    sense = rng.choice(np.array([-1.0, 1.0]), size=n_loops)

    e1 = bh[sys_idx]
    nrm = nh[sys_idx]
    e2 = np.cross(nrm, e1)
    k = np.arange(nodes_per_loop, dtype=np.float64)
    phi = phi0[:, None] + sense[:, None] * (2.0 * math.pi / nodes_per_loop) * k[None, :]
    xyz = (centre[:, None, :]
           + radius[:, None, None] * (np.cos(phi)[:, :, None] * e1[:, None, :]
                                      + np.sin(phi)[:, :, None] * e2[:, None, :]))
    xyz = xyz.reshape(-1, 3)
    loop_off = np.arange(n_loops + 1, dtype=np.int64) * nodes_per_loop
    burgers = b_mag * e1
    return np.ascontiguousarray(xyz), loop_off, np.ascontiguousarray(burgers), np.ascontiguousarray(nrm)


def loop_ensemble(seed, n_loops, box_edge, sig_app, nodes_per_loop=32,
                  r_min=0.05 * MICRON, r_max=0.2 * MICRON):
    """A single realisation of n_loops free glide loops in a cube of edge box_edge."""
    rng = np.random.default_rng(seed)
    xyz, off, bv, nv = circular_loops(rng, n_loops, box_edge, r_min, r_max, nodes_per_loop)
    return Network(xyz, off, bv, nv, np.zeros(xyz.shape[0], np.uint8),
                   box_edge ** 3, np.asarray(sig_app, dtype=np.float64).copy())


# --------------------------------------------------------------------------
# The named workloads.
# --------------------------------------------------------------------------
SMALL_LOOPS = dict(n_loops=16, box_edge=1.0 * MICRON, steps=100, dt=1e-11, seed=1001)
LARGE_LOOPS = dict(n_loops=1024, box_edge=5.0 * MICRON, steps=1000, dt=1e-11, seed=1002)
# same loop density as LARGE_LOOPS, a quarter of the loops (profiling-sized case)
MEDIUM_LOOPS = dict(n_loops=256, box_edge=5.0 * MICRON * 0.25 ** (1.0 / 3.0), dt=1e-11, seed=1006)


def small_loop_network(seed=SMALL_LOOPS["seed"]):
    """16 loops x 32 segments (512) in a 1 um cube, 50 MPa uniaxial along [001]."""
    return loop_ensemble(seed, SMALL_LOOPS["n_loops"], SMALL_LOOPS["box_edge"],
                         uniaxial_stress(50e6))


def large_loop_network(seed=LARGE_LOOPS["seed"]):
    """1024 loops x 32 segments (32768) in a 5 um cube, 50 MPa uniaxial along [001]."""
    return loop_ensemble(seed, LARGE_LOOPS["n_loops"], LARGE_LOOPS["box_edge"],
                         uniaxial_stress(50e6))


def medium_loop_network(seed=MEDIUM_LOOPS["seed"]):
    """256 loops x 32 segments (8192) at the loop density of the large workload."""
    return loop_ensemble(seed, MEDIUM_LOOPS["n_loops"], MEDIUM_LOOPS["box_edge"],
                         uniaxial_stress(50e6))


@dataclasses.dataclass
class Batch:
    """R realisations concatenated (SI units).

    Realisation r owns nodes [node_off[r], node_off[r+1]) and loops
    [loop_base[r], loop_base[r+1]); loop_off indexes the concatenated nodes.
    """
    xyz: np.ndarray
    loop_off: np.ndarray     # [total_loops + 1], global node indices
    loop_base: np.ndarray    # [R + 1]
    node_off: np.ndarray     # [R + 1]
    burgers: np.ndarray
    normal: np.ndarray
    pinned: np.ndarray
    sig6: np.ndarray         # [R, 6]
    volume: np.ndarray       # [R]

    @property
    def R(self):
        return int(self.node_off.shape[0] - 1)

    def realisation(self, r):
        n0, n1 = int(self.node_off[r]), int(self.node_off[r + 1])
        l0, l1 = int(self.loop_base[r]), int(self.loop_base[r + 1])
        return Network(self.xyz[n0:n1].copy(), self.loop_off[l0:l1 + 1] - n0,
                       self.burgers[l0:l1].copy(), self.normal[l0:l1].copy(),
                       self.pinned[n0:n1].copy(), float(self.volume[r]),
                       self.sig6[r].copy())


def batch_ensemble(seed, R=256, n_min=1024, n_max=16384, nodes_per_loop=32,
                   stress_max=200e6, sessile_min=0.1, sessile_max=0.9,
                   loops_per_um3=16.0):
    """Batched ensemble of R independent realisations.

    Per realisation: N_r ~ U{n_min..n_max} rounded to a multiple of
    nodes_per_loop; each of the 6 stress components ~ U(-stress_max,
    stress_max); sessile fraction f_r ~ U(sessile_min, sessile_max): whole
    loops, in random order, are marked pinned until the pinned line length
    reaches f_r of the total.  The cube edge keeps the loop density at
    loops_per_um3, i.e. edge = (n_loops / loops_per_um3)^(1/3) um.
    """
    rng = np.random.default_rng(seed)
    xs, bvs, nvs, pins, offs = [], [], [], [], []
    loop_base = [0]
    node_off = [0]
    sig6 = np.empty((R, 6))
    vol = np.empty(R)
    for r in range(R):
        n_r = int(rng.integers(n_min, n_max + 1))
        n_loops = max(1, int(round(n_r / nodes_per_loop)))
        edge = (n_loops / loops_per_um3) ** (1.0 / 3.0) * MICRON
        xyz, off, bv, nv = circular_loops(rng, n_loops, edge, nodes_per_loop=nodes_per_loop)
        sig6[r] = rng.uniform(-stress_max, stress_max, size=6)
        frac = rng.uniform(sessile_min, sessile_max)
        # pinned loops: random order until the pinned length fraction reaches frac
        seg = np.roll(xyz.reshape(n_loops, nodes_per_loop, 3), -1, axis=1) - xyz.reshape(n_loops, nodes_per_loop, 3)
        loop_len = np.sqrt((seg ** 2).sum(-1)).sum(-1)
        order = rng.permutation(n_loops)
        pinned_loop = np.zeros(n_loops, bool)
        acc, tot = 0.0, loop_len.sum()
        for k in order:
            if acc >= frac * tot:
                break
            pinned_loop[k] = True
            acc += loop_len[k]
        pin = np.repeat(pinned_loop, nodes_per_loop).astype(np.uint8)
        xs.append(xyz)
        bvs.append(bv)
        nvs.append(nv)
        pins.append(pin)
        offs.append(off[:-1] + node_off[-1])
        node_off.append(node_off[-1] + xyz.shape[0])
        loop_base.append(loop_base[-1] + n_loops)
        vol[r] = edge ** 3
    loop_off = np.concatenate(offs + [np.array([node_off[-1]], np.int64)]).astype(np.int64)
    return Batch(np.ascontiguousarray(np.concatenate(xs)), loop_off,
                 np.asarray(loop_base, np.int64), np.asarray(node_off, np.int64),
                 np.ascontiguousarray(np.concatenate(bvs)), np.ascontiguousarray(np.concatenate(nvs)),
                 np.concatenate(pins), sig6, vol)


def batch_from_networks(nets):
    """Concatenate single-realisation Networks into a Batch."""
    node_off = [0]
    loop_base = [0]
    offs = []
    for nt in nets:
        offs.append(np.asarray(nt.loop_off[:-1], np.int64) + node_off[-1])
        node_off.append(node_off[-1] + nt.n_nodes)
        loop_base.append(loop_base[-1] + nt.n_loops)
    loop_off = np.concatenate(offs + [np.array([node_off[-1]], np.int64)])
    return Batch(np.ascontiguousarray(np.concatenate([nt.xyz for nt in nets])), loop_off,
                 np.asarray(loop_base, np.int64), np.asarray(node_off, np.int64),
                 np.ascontiguousarray(np.concatenate([nt.burgers for nt in nets])),
                 np.ascontiguousarray(np.concatenate([nt.normal for nt in nets])),
                 np.concatenate([nt.pinned for nt in nets]).astype(np.uint8),
                 np.stack([nt.sig_app for nt in nets]), np.array([nt.volume for nt in nets], float))


# --------------------------------------------------------------------------
# Closure samples for the surrogate: realisations whose per-slip-system line
# densities vary, and the 30 closure features of each realisation.
# --------------------------------------------------------------------------
def slip_system_index(burgers, normal):
    """Index (0..11) of the FCC slip system of each loop, matching +-b_hat and +-n."""
    bh, nh = fcc_slip_systems()
    b = burgers / np.linalg.norm(burgers, axis=1, keepdims=True)
    sb = np.abs(b @ bh.T)
    sn = np.abs(normal @ nh.T)
    idx = np.argmax(sb * sn, axis=1)
    return idx


def closure_features(batch):
    """[R, 30]: applied stress (6, Pa), mobile (12) and sessile (12) line
    densities per FCC slip system (1/m^2) of every realisation."""
    sys_idx = slip_system_index(batch.burgers, batch.normal)
    feats = np.zeros((batch.R, 30))
    feats[:, :6] = batch.sig6
    for r in range(batch.R):
        l0, l1 = int(batch.loop_base[r]), int(batch.loop_base[r + 1])
        for k in range(l0, l1):
            a, b = int(batch.loop_off[k]), int(batch.loop_off[k + 1])
            x = batch.xyz[a:b]
            per = np.sum(np.linalg.norm(np.roll(x, -1, axis=0) - x, axis=1))
            col = 18 if batch.pinned[a] else 6
            feats[r, col + sys_idx[k]] += per / batch.volume[r]
    return feats


def closure_ensemble(seed, R, loops_min=16, loops_max=64, density_min=8.0, density_max=32.0,
                     stress_max=200e6, sessile_min=0.1, sessile_max=0.9, nodes_per_loop=32):
    """R independent realisations for closure samples.

    Per realisation: loop count ~ U{loops_min..loops_max}; loop density
    ~ U(density_min, density_max) per um^3 (sets the cube); slip-system
    weights ~ Dirichlet(1, ..., 1) and each loop's system drawn from them;
    radius ~ U(0.05, 0.2) um; every stress component ~ U(-stress_max,
    stress_max); whole loops pinned in random order until the pinned line
    fraction reaches f ~ U(sessile_min, sessile_max).
    Returns (Batch, features [R, 30]).
    """
    rng = np.random.default_rng(seed)
    nets = []
    for _ in range(R):
        nl = int(rng.integers(loops_min, loops_max + 1))
        dens = rng.uniform(density_min, density_max)
        edge = (nl / dens) ** (1.0 / 3.0) * MICRON
        w = rng.dirichlet(np.ones(12))
        systems = rng.choice(12, size=nl, p=w)
        xyz, off, bv, nv = _loops_with_systems(rng, systems, edge, nodes_per_loop)
        frac = rng.uniform(sessile_min, sessile_max)
        seg = np.roll(xyz.reshape(nl, nodes_per_loop, 3), -1, axis=1) - xyz.reshape(nl, nodes_per_loop, 3)
        loop_len = np.sqrt((seg ** 2).sum(-1)).sum(-1)
        pinned_loop = np.zeros(nl, bool)
        acc, tot = 0.0, loop_len.sum()
        for k in rng.permutation(nl):
            if acc >= frac * tot:
                break
            pinned_loop[k] = True
            acc += loop_len[k]
        pin = np.repeat(pinned_loop, nodes_per_loop).astype(np.uint8)
        nets.append(Network(xyz, off, bv, nv, pin, edge ** 3, rng.uniform(-stress_max, stress_max, size=6)))
    batch = batch_from_networks(nets)
    return batch, closure_features(batch)


def _loops_with_systems(rng, systems, edge, nodes_per_loop, r_min=0.05 * MICRON, r_max=0.2 * MICRON,
                        radius=None, sense=None):
    bh, nh = fcc_slip_systems()
    n = len(systems)
    if radius is None:
        radius = rng.uniform(r_min, r_max, size=n)
    centre = rng.uniform(0.0, edge, size=(n, 3))
    phi0 = rng.uniform(0.0, 2.0 * math.pi, size=n)
    if sense is None:
        sense = rng.choice(np.array([-1.0, 1.0]), size=n)
    e1 = bh[systems]
    nrm = nh[systems]
    e2 = np.cross(nrm, e1)
    k = np.arange(nodes_per_loop, dtype=np.float64)
    phi = phi0[:, None] + sense[:, None] * (2.0 * math.pi / nodes_per_loop) * k[None, :]
    xyz = (centre[:, None, :] + radius[:, None, None] * (np.cos(phi)[:, :, None] * e1[:, None, :]
                                                         + np.sin(phi)[:, :, None] * e2[:, None, :]))
    off = np.arange(n + 1, dtype=np.int64) * nodes_per_loop
    return (np.ascontiguousarray(xyz.reshape(-1, 3)), off, np.ascontiguousarray(BURGERS * e1),
            np.ascontiguousarray(nrm))


def realisation_for_densities(rng, sig6, rho_m, rho_s, n_loops=32, nodes_per_loop=32,
                              r_min=0.05 * MICRON, r_max=0.2 * MICRON, stratified=False):
    """One realisation whose mobile/sessile line densities per slip system
    follow rho_m[12], rho_s[12] (1/m^2): n_loops loops split over the 24
    (system, mobile/sessile) classes in proportion to their density.

    stratified=False: classes drawn independently per loop, radii ~
    U(r_min, r_max), line sense +-1, cube volume from the mean loop perimeter
    (densities match on average).
    stratified=True: class counts are floor or ceil of n_loops x share
    (systematic sampling of the remainders), radii are stratified over
    (r_min, r_max) within each class, line senses are balanced within each
    class, and the volume is set from the drawn loops' total length, so the
    total density matches exactly and each class's within one loop."""
    dens = np.concatenate([np.asarray(rho_m, float), np.asarray(rho_s, float)])
    tot = dens.sum()
    p = dens / tot if tot > 0 else np.full(24, 1.0 / 24)
    radius = sense = None
    if not stratified:
        cls = rng.choice(24, size=n_loops, p=p)
    else:
        e = n_loops * p
        counts = np.floor(e).astype(np.int64)
        extra = n_loops - int(counts.sum())
        if extra > 0:
            picks = np.searchsorted(np.cumsum(e - counts), rng.uniform() + np.arange(extra), side="right")
            counts += np.bincount(np.minimum(picks, 23), minlength=24)
        cls = np.repeat(np.arange(24), counts)
        radius = np.empty(cls.size)
        sense = np.empty(cls.size)
        for c in range(24):
            idx = np.flatnonzero(cls == c)
            k = idx.size
            if k == 0:
                continue
            radius[idx] = r_min + (r_max - r_min) * (rng.permutation(k) + rng.uniform(size=k)) / k
            sg = np.where(np.arange(k) < k // 2, 1.0, -1.0)
            if k % 2:
                sg[-1] = rng.choice(np.array([-1.0, 1.0]))
            sense[idx] = rng.permutation(sg)
    systems = cls % 12
    xyz_tmp_edge = 1.0 * MICRON
    chord = 2.0 * math.sin(math.pi / nodes_per_loop) * nodes_per_loop
    if stratified:
        length = chord * radius.sum()
    else:
        length = n_loops * chord * 0.5 * (r_min + r_max)
    volume = length / tot if tot > 0 else xyz_tmp_edge ** 3
    edge = volume ** (1.0 / 3.0)
    xyz, off, bv, nv = _loops_with_systems(rng, systems, edge, nodes_per_loop, r_min, r_max, radius, sense)
    pin = np.repeat((cls >= 12).astype(np.uint8), nodes_per_loop)
    return Network(xyz, off, bv, nv, pin, edge ** 3, np.asarray(sig6, float).copy())


# --------------------------------------------------------------------------
# The paper's microstructure recipe (Sec. 3.2.1) on glide loops: mobile line
# density shared among the slip systems in proportion to |Schmid factor|,
# sessile density spread evenly over the 12 systems (rho_s >> rho_m), every
# loop carrying both line senses (net density 0), sessile loops pinned.
# --------------------------------------------------------------------------
def schmid_factors(sig6):
    """f_i = b_i . (sigma n_i) / |sigma| for the 12 FCC systems (|sigma| the
    Frobenius norm of the full tensor), Sec. 3.2.1."""
    s = np.asarray(sig6, float)
    S = np.array([[s[0], s[5], s[4]], [s[5], s[1], s[3]], [s[4], s[3], s[2]]])
    bh, nh = fcc_slip_systems()
    return np.einsum("ki,ij,kj->k", bh, S, nh) / np.linalg.norm(S)


def junction_microstructure(seed, sig6, rho_m, rho_s, n_loops=64, nodes_per_loop=32,
                            r_min=0.05 * MICRON, r_max=0.2 * MICRON, sessile_case=2):
    """One realisation of the paper's recipe with n_loops glide loops:
    mobile density rho_m (1/m^2) per system in proportion to |f_i|, sessile
    density rho_s evenly over the systems; class counts, radii and senses
    stratified as in realisation_for_densities.

    sessile_case (the two cases of Sec. 3.2): 2, the sessile loops' Burgers
    vectors lie in their planes (b . n = 0); 1, Lomer-Cottrell-type locks,
    whose Burgers vectors lie out of their planes (lomer_cottrell_sessiles).
    Both cases share the geometry of a seed."""
    f = np.abs(schmid_factors(sig6))
    rho_mi = rho_m * f / f.sum()
    rho_si = np.full(12, rho_s / 12.0)
    rng = np.random.default_rng(seed)
    net = realisation_for_densities(rng, sig6, rho_mi, rho_si, n_loops, nodes_per_loop, r_min, r_max,
                                    stratified=True)
    if sessile_case == 1:
        return lomer_cottrell_sessiles(net, np.random.default_rng([seed, 1]))
    if sessile_case != 2:
        raise ValueError("sessile_case must be 1 or 2")
    return net


def lomer_cottrell_sessiles(net, rng):
    """Case 1 of Sec. 3.2: every sessile loop (all its nodes pinned) keeps
    its plane, line and |b| and takes a Burgers vector along one of the three
    <110> directions that do not lie in its plane (b . n = +-(2/sqrt 6)|b|),
    drawn uniformly, with a random sign; mobile loops are unchanged."""
    cands = np.array([[0, 1, -1], [1, 0, -1], [1, -1, 0], [0, 1, 1], [1, 0, 1], [1, 1, 0]], float) / math.sqrt(2.0)
    out = net.copy()
    bv = out.burgers.copy()
    for k in range(out.n_loops):
        a, b = out.loop_off[k], out.loop_off[k + 1]
        if not np.all(out.pinned[a:b]):
            continue
        off_plane = cands[np.abs(cands @ out.normal[k]) > 0.5]
        d = off_plane[rng.integers(off_plane.shape[0])] * rng.choice(np.array([-1.0, 1.0]))
        bv[k] = np.linalg.norm(bv[k]) * d
    out.burgers = bv
    return out


# --------------------------------------------------------------------------
# Crystal-to-global frames (Appendix): A_ki = e_k . e^_i, so that global
# components are g = A c; its rows are the unit crystallographic directions
# that lie along the global X, Y and Z = X x Y axes.  The DD box works in the
# crystal frame, so a stress given in the laboratory frame enters as
# sigma_crystal = A^T sigma_global A.
# --------------------------------------------------------------------------
C2G_TENSION = ((0, -1, 1), (2, 1, 1))   # symmetric double slip, uniaxial tension (Sec. 3.3.1)
C2G_SHEAR = ((0, 1, 1), (-1, 1, -1))    # simple shear orientation (Sec. 3.3.2)


def c2g_matrix(x_dir, y_dir):
    """C2G matrix with the crystal direction x_dir along global X and y_dir
    (perpendicular to it) along global Y."""
    x = np.asarray(x_dir, float)
    y = np.asarray(y_dir, float)
    if abs(x @ y) > 1e-12 * np.linalg.norm(x) * np.linalg.norm(y):
        raise ValueError("the two crystal directions must be perpendicular")
    x = x / np.linalg.norm(x)
    y = y / np.linalg.norm(y)
    return np.array([x, y, np.cross(x, y)])


def global_to_crystal_stress(sig6_global, A):
    """Voigt stress in the laboratory frame -> Voigt stress in the crystal
    frame of the C2G matrix A."""
    s = np.asarray(sig6_global, float)
    S = np.array([[s[0], s[5], s[4]], [s[5], s[1], s[3]], [s[4], s[3], s[2]]])
    C = A.T @ S @ A
    return np.array([C[0, 0], C[1, 1], C[2, 2], C[1, 2], C[0, 2], C[0, 1]])
