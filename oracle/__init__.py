"""Plain FP64 CPU oracle of the discrete-dislocation burst (ctypes binding).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_2005_02498_gb300``) never imports it and shares no code with it.

``build()`` compiles ``ptadd_oracle.c`` with gcc (OpenMP, no fused
multiply-add contraction so x86 and Arm hosts round alike) into
``oracle/_lib/liboracle.so``.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ptadd_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "mlp_oracle.c"), os.path.join(_HERE, "junction_oracle.c")]
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_U8 = ctypes.POINTER(ctypes.c_uint8)


def build(force=False):
    """Compile the oracle shared library if it is missing or stale."""
    os.makedirs(_LIBDIR, exist_ok=True)
    hdr = os.path.join(_HERE, "ptadd_oracle.h")
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max([os.path.getmtime(f) for f in _SRCS] + [os.path.getmtime(hdr)])):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
           "-std=c11", "-o", tmp, *_SRCS, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.orc_gauss4.argtypes = [_D, _D]
        lib.orc_seg_stress.argtypes = [_D, _D, _D, _D, _D, _D]
        lib.orc_seg_stress_quad.argtypes = [_D, _D, _D, _D, _D, ctypes.c_int, ctypes.c_int, _D]
        lib.orc_seg_stress_quad.restype = ctypes.c_int
        lib.orc_ra_derivs.argtypes = [_D, ctypes.c_double, _D, _D]
        lib.orc_stress_at.argtypes = [_D, ctypes.c_int64, _D, ctypes.c_int64, _I64, _D, _D,
                                      ctypes.c_int, ctypes.c_int64, _D, _D]
        lib.orc_nodal_forces.argtypes = [_D, ctypes.c_int64, _D, ctypes.c_int64, _I64, _D, _U8,
                                         _D, ctypes.c_int, ctypes.c_int, _D]
        lib.orc_nodal_forces_subset.argtypes = [_D, ctypes.c_int64, _D, ctypes.c_int64, _I64, _D,
                                                _D, ctypes.c_int, ctypes.c_int64, _I64, _D]
        lib.orc_velocities.argtypes = [_D, ctypes.c_int64, _D, ctypes.c_int64, _I64, _D, _U8, _D, _D]
        lib.orc_lp_rho.argtypes = [ctypes.c_int64, _D, ctypes.c_int64, _I64, _D, _D,
                                   ctypes.c_double, _D, _D]
        lib.orc_velocities_consistent.argtypes = [_D, ctypes.c_int64, _D, ctypes.c_int64, _I64, _D, _U8, _D, _D]
        lib.orc_burst.argtypes = [_D, ctypes.c_int64, _D, ctypes.c_int64, _I64, _D, _D, _U8,
                                  ctypes.c_double, _D, ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                                  _D, _D, _D, _D, _D, ctypes.c_double, _D, ctypes.c_int]
        lib.orc_polar_velocity.argtypes = [ctypes.c_int64, _D, ctypes.c_int64, _I64, _D, ctypes.c_double,
                                           ctypes.c_double, _D]
        lib.orc_burst.restype = ctypes.c_int
        _I32 = ctypes.POINTER(ctypes.c_int32)
        lib.orc_splitmix64_mix.argtypes = [ctypes.c_uint64]
        lib.orc_splitmix64_mix.restype = ctypes.c_uint64
        lib.orc_junction_fraction.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64]
        lib.orc_junction_fraction.restype = ctypes.c_double
        lib.orc_point_segment_dist2.argtypes = [_D, _D, _D]
        lib.orc_point_segment_dist2.restype = ctypes.c_double
        lib.orc_burst_junctions.argtypes = [_D, ctypes.c_int64, _D, ctypes.c_int64, _I64, _D, _D, _U8,
                                            ctypes.c_double, _D, ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                                            _D, ctypes.c_uint64, _I32, _I32, _I32, _D, _D, _I64, _D, _D, _D, _D]
        lib.orc_burst_junctions.restype = ctypes.c_int
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_gelu.argtypes = [ctypes.c_double]
        lib.orc_gelu.restype = ctypes.c_double
        lib.orc_gelu_grad.argtypes = [ctypes.c_double]
        lib.orc_gelu_grad.restype = ctypes.c_double
        lib.orc_mlp_param_count.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        lib.orc_mlp_param_count.restype = ctypes.c_int64
        lib.orc_mlp_forward.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), _D, ctypes.c_int64, _D, _D]
        lib.orc_mlp_loss_grad.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), _D, ctypes.c_int64, _D, _D, _D]
        lib.orc_mlp_loss_grad.restype = ctypes.c_double
        lib.orc_adam_step.argtypes = [ctypes.c_int64, _D, _D, _D, _D, ctypes.c_int64, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double]
        _lib = lib
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_D)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(_I64)


def _u8(a):
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a, a.ctypes.data_as(_U8)


def _mat(mat):
    return _d(np.asarray(tuple(mat), dtype=np.float64))


def num_threads():
    return int(_load().orc_num_threads())


def gauss4():
    xi = np.zeros(4)
    w = np.zeros(4)
    _load().orc_gauss4(xi.ctypes.data_as(_D), w.ctypes.data_as(_D))
    return xi, w


def seg_stress(mat, x1, x2, b, x):
    """Analytic nonsingular stress (Voigt 6) of segment x1->x2 at point x."""
    lib = _load()
    m, mp = _mat(mat)
    a1, p1 = _d(x1)
    a2, p2 = _d(x2)
    ab, pb = _d(b)
    ax, px = _d(x)
    out = np.zeros(6)
    lib.orc_seg_stress(mp, p1, p2, pb, px, out.ctypes.data_as(_D))
    return out


def seg_stress_quad(mat, x1, x2, b, x, panels=64, order=16):
    """Brute-force long-double quadrature of the same integrand (3x3)."""
    lib = _load()
    m, mp = _mat(mat)
    a1, p1 = _d(x1)
    a2, p2 = _d(x2)
    ab, pb = _d(b)
    ax, px = _d(x)
    out = np.zeros(9)
    rc = lib.orc_seg_stress_quad(mp, p1, p2, pb, px, int(panels), int(order), out.ctypes.data_as(_D))
    if rc != 0:
        raise ValueError("bad quadrature arguments")
    return out.reshape(3, 3)


def ra_derivs(R, a):
    lib = _load()
    aR, pR = _d(R)
    d3 = np.zeros(27)
    dl = np.zeros(3)
    lib.orc_ra_derivs(pR, float(a), d3.ctypes.data_as(_D), dl.ctypes.data_as(_D))
    return d3.reshape(3, 3, 3), dl


def stress_at(mat, net, pts, interactions=True, sig_app=None):
    lib = _load()
    m, mp = _mat(mat)
    x, px = _d(net.xyz)
    off, poff = _i(net.loop_off)
    bv, pb = _d(net.burgers)
    sa, ps = _d(net.sig_app if sig_app is None else sig_app)
    P, pP = _d(np.asarray(pts).reshape(-1, 3))
    out = np.zeros((P.shape[0], 6))
    lib.orc_stress_at(mp, net.n_nodes, px, net.n_loops, poff, pb, ps, int(bool(interactions)),
                      P.shape[0], pP, out.ctypes.data_as(_D))
    return out


def nodal_forces(mat, net, interactions=True, skip_pinned=False, xyz=None):
    lib = _load()
    m, mp = _mat(mat)
    x, px = _d(net.xyz if xyz is None else xyz)
    off, poff = _i(net.loop_off)
    bv, pb = _d(net.burgers)
    pin, ppin = _u8(net.pinned)
    sa, ps = _d(net.sig_app)
    F = np.zeros((net.n_nodes, 3))
    lib.orc_nodal_forces(mp, net.n_nodes, px, net.n_loops, poff, pb, ppin, ps,
                         int(bool(interactions)), int(bool(skip_pinned)), F.ctypes.data_as(_D))
    return F


def nodal_forces_subset(mat, net, sel, interactions=True, xyz=None):
    lib = _load()
    m, mp = _mat(mat)
    x, px = _d(net.xyz if xyz is None else xyz)
    off, poff = _i(net.loop_off)
    bv, pb = _d(net.burgers)
    sa, ps = _d(net.sig_app)
    s, psel = _i(sel)
    F = np.zeros((s.shape[0], 3))
    lib.orc_nodal_forces_subset(mp, net.n_nodes, px, net.n_loops, poff, pb, ps,
                                int(bool(interactions)), s.shape[0], psel, F.ctypes.data_as(_D))
    return F


def velocities(mat, net, F, xyz=None, consistent=False):
    """Glide mobility of Eq. 2.1: lumped (default) or with the consistent mass matrix."""
    lib = _load()
    m, mp = _mat(mat)
    x, px = _d(net.xyz if xyz is None else xyz)
    off, poff = _i(net.loop_off)
    nv, pn = _d(net.normal)
    pin, ppin = _u8(net.pinned)
    f, pf = _d(F)
    v = np.zeros((net.n_nodes, 3))
    fn = lib.orc_velocities_consistent if consistent else lib.orc_velocities
    fn(mp, net.n_nodes, px, net.n_loops, poff, pn, ppin, pf, v.ctypes.data_as(_D))
    return v


def lp_rho(net, v, xyz=None):
    lib = _load()
    x, px = _d(net.xyz if xyz is None else xyz)
    off, poff = _i(net.loop_off)
    bv, pb = _d(net.burgers)
    vv, pv = _d(v)
    Lp = np.zeros(9)
    rho = ctypes.c_double(0.0)
    lib.orc_lp_rho(net.n_nodes, px, net.n_loops, poff, pb, pv, float(net.volume),
                   Lp.ctypes.data_as(_D), ctypes.byref(rho))
    return Lp.reshape(3, 3), rho.value


def polar_velocity(net, v, core_area, xyz=None):
    """V = (core_area / |B|) sum_s L_s vbar_s (Eq. 2.11), from nodal velocities v [n, 3]."""
    lib = _load()
    x, px = _d(net.xyz if xyz is None else xyz)
    off, poff = _i(net.loop_off)
    vv, pv = _d(v)
    V = np.zeros(3)
    lib.orc_polar_velocity(net.n_nodes, px, net.n_loops, poff, pv, float(net.volume), float(core_area),
                           V.ctypes.data_as(_D))
    return V


def burst(mat, net, n_steps, dt, interactions=True, trace=False, core_area=None, consistent_mass=False):
    """Run n_steps Euler steps; returns dict(xyz, Lp_avg (3x3), rho_avg[, Lp_trace, rho_trace][, V_avg]).
    consistent_mass: the consistent mobility of Eq. 2.1 instead of the lumped one."""
    lib = _load()
    m, mp = _mat(mat)
    x, px = _d(net.xyz)
    off, poff = _i(net.loop_off)
    bv, pb = _d(net.burgers)
    nv, pn = _d(net.normal)
    pin, ppin = _u8(net.pinned)
    sa, ps = _d(net.sig_app)
    xo = np.zeros_like(x)
    Lp = np.zeros(9)
    rho = ctypes.c_double(0.0)
    tL = np.zeros((max(n_steps, 1), 9)) if trace else None
    tr = np.zeros(max(n_steps, 1)) if trace else None
    V = np.zeros(3)
    rc = lib.orc_burst(mp, net.n_nodes, px, net.n_loops, poff, pb, pn, ppin, float(net.volume), ps,
                       int(bool(interactions)), int(n_steps), float(dt), xo.ctypes.data_as(_D),
                       Lp.ctypes.data_as(_D), ctypes.byref(rho),
                       tL.ctypes.data_as(_D) if trace else None,
                       tr.ctypes.data_as(_D) if trace else None,
                       float(core_area or 0.0), V.ctypes.data_as(_D) if core_area is not None else None,
                       int(bool(consistent_mass)))
    out = dict(xyz=xo, Lp_avg=Lp.reshape(3, 3), rho_avg=rho.value, status=rc)
    if core_area is not None:
        out["V_avg"] = V
    if trace:
        out["Lp_trace"] = tL[:n_steps].reshape(-1, 3, 3)
        out["rho_trace"] = tr[:n_steps]
    return out


# ------------------------------------------------------------ junctions
def splitmix64_mix(z):
    return int(_load().orc_splitmix64_mix(ctypes.c_uint64(z & 0xFFFFFFFFFFFFFFFF)))


def junction_fraction(seed, node, k):
    return float(_load().orc_junction_fraction(ctypes.c_uint64(seed), int(node), int(k)))


def point_segment_dist2(x, x1, x2):
    x, px = _d(x)
    x1, p1 = _d(x1)
    x2, p2 = _d(x2)
    return float(_load().orc_point_segment_dist2(px, p1, p2))


def junction_state(n_nodes):
    """Fresh junction state: nothing held, clock 0."""
    return dict(seg=np.full(n_nodes, -1, np.int32), last=np.full(n_nodes, -1, np.int32),
                count=np.zeros(n_nodes, np.int32), brk=np.zeros(n_nodes), clock=np.zeros(2),
                counts=np.zeros(3, np.int64))


def burst_junctions(mat, net, n_steps, dt, capture_radius, max_break_time, stuck_disp, seed, state=None,
                    interactions=True):
    """n_steps DD steps with junctions and thermally activated breaking
    (Sec. 2.2, readings in junction_oracle.c).  `state` (from
    junction_state() or a previous call) is updated in place.  Returns
    dict(xyz, Lp_avg, rho_avg, S_t, state, status)."""
    lib = _load()
    st = junction_state(net.n_nodes) if state is None else state
    m, mp = _mat(mat)
    x, px = _d(net.xyz)
    off, poff = _i(net.loop_off)
    bv, pb = _d(net.burgers)
    nv, pn = _d(net.normal)
    pin, ppin = _u8(net.pinned)
    sg, ps = _d(net.sig_app)
    jp, pj = _d([capture_radius, max_break_time, stuck_disp])
    _I32 = ctypes.POINTER(ctypes.c_int32)
    for k, dt_ in (("seg", np.int32), ("last", np.int32), ("count", np.int32), ("brk", np.float64),
                   ("clock", np.float64), ("counts", np.int64)):
        st[k] = np.ascontiguousarray(st[k], dtype=dt_)
    xo = np.zeros((net.n_nodes, 3))
    Lp = np.zeros(9)
    rho, S_t = ctypes.c_double(0.0), ctypes.c_double(0.0)
    rc = lib.orc_burst_junctions(mp, net.n_nodes, px, net.n_loops, poff, pb, pn, ppin, float(net.volume), ps,
                                 int(bool(interactions)), int(n_steps), float(dt), pj, ctypes.c_uint64(seed),
                                 st["seg"].ctypes.data_as(_I32), st["last"].ctypes.data_as(_I32),
                                 st["count"].ctypes.data_as(_I32), st["brk"].ctypes.data_as(_D),
                                 st["clock"].ctypes.data_as(_D), st["counts"].ctypes.data_as(_I64),
                                 xo.ctypes.data_as(_D), Lp.ctypes.data_as(_D), ctypes.byref(rho), ctypes.byref(S_t))
    return dict(xyz=xo, Lp_avg=Lp.reshape(3, 3), rho_avg=rho.value, S_t=S_t.value, state=st, status=rc)


# ------------------------------------------------------------------ MLP
def _dims(dims):
    arr = (ctypes.c_int * len(dims))(*[int(d) for d in dims])
    return len(dims) - 1, arr


def gelu(z):
    return _load().orc_gelu(float(z))


def gelu_grad(z):
    return _load().orc_gelu_grad(float(z))


def mlp_param_count(dims):
    L, arr = _dims(dims)
    return int(_load().orc_mlp_param_count(L, arr))


def mlp_forward(dims, params, X):
    L, arr = _dims(dims)
    p, pp = _d(params)
    x, px = _d(np.asarray(X).reshape(-1, dims[0]))
    Y = np.zeros((x.shape[0], dims[-1]))
    _load().orc_mlp_forward(L, arr, pp, x.shape[0], px, Y.ctypes.data_as(_D))
    return Y


def mlp_loss_grad(dims, params, X, T):
    L, arr = _dims(dims)
    p, pp = _d(params)
    x, px = _d(np.asarray(X).reshape(-1, dims[0]))
    t, pt = _d(np.asarray(T).reshape(-1, dims[-1]))
    g = np.zeros_like(p)
    loss = _load().orc_mlp_loss_grad(L, arr, pp, x.shape[0], px, pt, g.ctypes.data_as(_D))
    return loss, g


def adam_step(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In place on float64 arrays p, m, v."""
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    gg, pg = _d(g)
    _load().orc_adam_step(p.size, p.ctypes.data_as(_D), pg, m.ctypes.data_as(_D), v.ctypes.data_as(_D),
                          int(t), float(lr), float(b1), float(b2), float(eps))
