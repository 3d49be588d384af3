"""Thin ctypes binding of libptadd.so (ptadd.h).

Argument marshalling only: every step of the burst runs in the library's CUDA
kernels.  If the library has not been built, or cannot be loaded, every call
raises -- there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

PTADD_FP64 = 0
PTADD_MIXED = 1

STATUS = {0: "PTADD_OK", 1: "PTADD_ERR_ARG", 2: "PTADD_ERR_CUDA", 3: "PTADD_ERR_NONFINITE",
          4: "PTADD_ERR_TIMEOUT", 5: "PTADD_ERR_STATE", 6: "PTADD_ERR_NOMEM"}

# Every symbol ptadd.h declares (the CPU test checks the library exports them).
EXPORTS = ["ptadd_version", "ptadd_create", "ptadd_destroy", "ptadd_last_error", "ptadd_set_precision",
           "ptadd_set_stream", "ptadd_set_network", "ptadd_set_applied_stress", "ptadd_get_info",
           "ptadd_advance", "ptadd_get_nodes", "ptadd_get_forces", "ptadd_get_forces_dev",
           "ptadd_get_state", "ptadd_set_state", "ptadd_fma_peak", "ptadd_set_nodes",
           "ptadd_profile_reset", "ptadd_profile_read", "ptadd_forces_noalloc",
           "ptadd_batch_set", "ptadd_batch_set_stress", "ptadd_batch_advance", "ptadd_batch_get_nodes",
           "ptadd_batch_set_nodes", "ptadd_batch_get_info", "ptadd_batch_autotune", "ptadd_batch_run",
           "ptadd_batch_configure", "ptadd_batch_get_forces", "ptadd_get_polar_velocity",
           "ptadd_batch_get_polar_velocity",
           "ptadd_gemm_bf16", "ptadd_gemm_timeout_selftest", "ptadd_mlp_param_count", "ptadd_mlp_init", "ptadd_mlp_set_params",
           "ptadd_mlp_get_params", "ptadd_mlp_loss_grad", "ptadd_mlp_train", "ptadd_mlp_forward",
           "ptadd_surrogate_fit", "ptadd_surrogate_predict", "ptadd_surrogate_predict_dev",
           "ptadd_closure_sweep", "ptadd_closure_realisation", "ptadd_dissipation_projection",
           "ptadd_dissipation_projection_dev",
           "ptadd_block_average", "ptadd_block_stress_pair", "ptadd_set_junctions", "ptadd_get_junctions", "ptadd_set_mobility",
           "ptadd_batch_set_junctions", "ptadd_batch_get_junctions", "ptadd_system_densities",
           "ptadd_surrogate_get_state", "ptadd_surrogate_set_state"]
NOALLOC_MAX_SEGMENTS = 16384


class PtaddError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class Material(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("nu", ctypes.c_double), ("b", ctypes.c_double),
                ("a", ctypes.c_double), ("B", ctypes.c_double)]


class Profile(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int64), ("pair_launches", ctypes.c_int64),
                ("pair_evals", ctypes.c_int64), ("pair_ms", ctypes.c_double),
                ("near_point_pairs", ctypes.c_int64)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("R", ctypes.c_int32), ("n_nodes", ctypes.c_int64), ("n_loops", ctypes.c_int64),
                ("n_targets", ctypes.c_int64), ("pairs_per_step", ctypes.c_int64), ("work_items", ctypes.c_int64),
                ("tile_targets", ctypes.c_int32), ("chunk_sources", ctypes.c_int32), ("tuned", ctypes.c_int32)]


class JunctionParams(ctypes.Structure):
    _fields_ = [("capture_radius", ctypes.c_double), ("max_break_time", ctypes.c_double),
                ("stuck_disp", ctypes.c_double), ("seed", ctypes.c_uint64)]


class JunctionInfo(ctypes.Structure):
    _fields_ = [("clock", ctypes.c_double), ("jumped", ctypes.c_double), ("held", ctypes.c_int64),
                ("formed", ctypes.c_int64), ("broken", ctypes.c_int64), ("jumps", ctypes.c_int64)]


class Info(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_loops", ctypes.c_int64), ("n_targets", ctypes.c_int64),
                ("pairs_per_step", ctypes.c_int64), ("precision", ctypes.c_int32), ("device", ctypes.c_int32)]


_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_VP = ctypes.c_void_p
_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libptadd.so (building it first if asked); raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libptadd.so is not built (%s); run __graft_entry__.build()" % _build.LIB)
    lib = ctypes.CDLL(_build.LIB)
    st = ctypes.c_int
    lib.ptadd_version.restype = ctypes.c_int
    lib.ptadd_last_error.restype = ctypes.c_char_p
    lib.ptadd_create.argtypes = [ctypes.POINTER(_VP), ctypes.POINTER(Material), ctypes.c_int, ctypes.c_int]
    lib.ptadd_create.restype = st
    lib.ptadd_destroy.argtypes = [_VP]
    lib.ptadd_destroy.restype = None
    lib.ptadd_set_precision.argtypes = [_VP, ctypes.c_int]
    lib.ptadd_set_precision.restype = st
    lib.ptadd_set_stream.argtypes = [_VP, _VP]
    lib.ptadd_set_stream.restype = st
    lib.ptadd_set_network.argtypes = [_VP, ctypes.c_int64, _D, ctypes.c_int64, _I64, _D, _D, _U8, ctypes.c_double]
    lib.ptadd_set_network.restype = st
    lib.ptadd_set_applied_stress.argtypes = [_VP, _D]
    lib.ptadd_set_applied_stress.restype = st
    lib.ptadd_get_info.argtypes = [_VP, ctypes.POINTER(Info)]
    lib.ptadd_get_info.restype = st
    lib.ptadd_advance.argtypes = [_VP, ctypes.c_int64, ctypes.c_double, _D, _D]
    lib.ptadd_advance.restype = st
    lib.ptadd_get_nodes.argtypes = [_VP, _D]
    lib.ptadd_get_nodes.restype = st
    lib.ptadd_get_forces.argtypes = [_VP, _D]
    lib.ptadd_get_forces.restype = st
    lib.ptadd_get_forces_dev.argtypes = [_VP, _VP]
    lib.ptadd_get_forces_dev.restype = st
    lib.ptadd_get_state.argtypes = [_VP, _VP, ctypes.POINTER(ctypes.c_size_t)]
    lib.ptadd_get_state.restype = st
    lib.ptadd_set_state.argtypes = [_VP, _VP, ctypes.c_size_t]
    lib.ptadd_set_state.restype = st
    lib.ptadd_set_nodes.argtypes = [_VP, _VP]
    lib.ptadd_set_nodes.restype = st
    lib.ptadd_profile_reset.argtypes = [_VP, ctypes.c_int]
    lib.ptadd_profile_reset.restype = st
    lib.ptadd_profile_read.argtypes = [_VP, ctypes.POINTER(Profile)]
    lib.ptadd_profile_read.restype = st
    lib.ptadd_forces_noalloc.argtypes = [ctypes.POINTER(Material), ctypes.c_int64, _VP, _VP, _VP, _VP, _D, _VP, _VP]
    lib.ptadd_forces_noalloc.restype = st
    lib.ptadd_batch_set.argtypes = [_VP, ctypes.c_int32, _I64, ctypes.c_int64, _I64, _D, _D, _D, _U8, _D, _D]
    lib.ptadd_batch_set.restype = st
    lib.ptadd_batch_set_stress.argtypes = [_VP, _D]
    lib.ptadd_batch_set_stress.restype = st
    lib.ptadd_batch_advance.argtypes = [_VP, ctypes.c_int64, ctypes.c_double, _D, _D]
    lib.ptadd_batch_advance.restype = st
    lib.ptadd_batch_get_nodes.argtypes = [_VP, _D]
    lib.ptadd_batch_get_nodes.restype = st
    lib.ptadd_batch_set_nodes.argtypes = [_VP, _D]
    lib.ptadd_batch_set_nodes.restype = st
    lib.ptadd_batch_get_info.argtypes = [_VP, ctypes.POINTER(BatchInfo)]
    lib.ptadd_batch_get_info.restype = st
    lib.ptadd_batch_autotune.argtypes = [_VP, ctypes.c_char_p, ctypes.c_int]
    lib.ptadd_batch_autotune.restype = st
    lib.ptadd_get_polar_velocity.argtypes = [_VP, ctypes.c_double, _D]
    lib.ptadd_get_polar_velocity.restype = st
    lib.ptadd_batch_get_polar_velocity.argtypes = [_VP, ctypes.c_double, _D]
    lib.ptadd_batch_get_polar_velocity.restype = st
    lib.ptadd_batch_configure.argtypes = [_VP, ctypes.c_int32, ctypes.c_int32]
    lib.ptadd_batch_configure.restype = st
    lib.ptadd_batch_get_forces.argtypes = [_VP, _D]
    lib.ptadd_batch_get_forces.restype = st
    lib.ptadd_batch_run.argtypes = [_VP, ctypes.c_int32, _I64, ctypes.c_int64, _I64, _D, _D, _D, _U8, _D, _D,
                                    ctypes.c_int64, ctypes.c_double, _D, _D]
    lib.ptadd_batch_run.restype = st
    lib.ptadd_gemm_bf16.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _VP, _VP, _VP]
    lib.ptadd_gemm_bf16.restype = st
    lib.ptadd_gemm_timeout_selftest.argtypes = [ctypes.c_int]
    lib.ptadd_gemm_timeout_selftest.restype = st
    _F = ctypes.POINTER(ctypes.c_float)
    lib.ptadd_mlp_param_count.restype = ctypes.c_int64
    lib.ptadd_mlp_init.argtypes = [_VP, ctypes.c_uint64]
    lib.ptadd_mlp_init.restype = st
    lib.ptadd_mlp_set_params.argtypes = [_VP, _F, ctypes.c_int64]
    lib.ptadd_mlp_set_params.restype = st
    lib.ptadd_mlp_get_params.argtypes = [_VP, _F, ctypes.c_int64]
    lib.ptadd_mlp_get_params.restype = st
    lib.ptadd_mlp_loss_grad.argtypes = [_VP, ctypes.c_int64, _F, _F, _F, _F]
    lib.ptadd_mlp_loss_grad.restype = st
    lib.ptadd_mlp_train.argtypes = [_VP, ctypes.c_int64, _F, _F, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                    ctypes.c_uint64, _F]
    lib.ptadd_mlp_train.restype = st
    lib.ptadd_mlp_forward.argtypes = [_VP, ctypes.c_int64, _F, _F]
    lib.ptadd_mlp_forward.restype = st
    lib.ptadd_surrogate_fit.argtypes = [_VP, ctypes.c_int64, _D, _D, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                        ctypes.c_uint64, _F]
    lib.ptadd_surrogate_fit.restype = st
    lib.ptadd_surrogate_predict.argtypes = [_VP, ctypes.c_int64, _D, _D, _U8]
    lib.ptadd_surrogate_predict.restype = st
    lib.ptadd_surrogate_predict_dev.argtypes = [_VP, ctypes.c_int64, _VP, _VP, _VP]
    lib.ptadd_surrogate_predict_dev.restype = st
    lib.ptadd_closure_sweep.argtypes = [_VP, ctypes.c_int64, _D, _D, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_double, ctypes.c_uint64, _D, _U8]
    lib.ptadd_closure_sweep.restype = st
    lib.ptadd_closure_realisation.argtypes = [ctypes.POINTER(Material), ctypes.c_uint64, _D, ctypes.c_int32, _D, _D,
                                              _D, _U8, _D]
    lib.ptadd_closure_realisation.restype = st
    lib.ptadd_dissipation_projection.argtypes = [_D, _D, _D, _D]
    lib.ptadd_dissipation_projection.restype = st
    lib.ptadd_dissipation_projection_dev.argtypes = [ctypes.c_int64, _VP, _VP, _VP, _VP, _VP, _VP]
    lib.ptadd_dissipation_projection_dev.restype = st
    _I32 = ctypes.POINTER(ctypes.c_int32)
    lib.ptadd_set_junctions.argtypes = [_VP, ctypes.POINTER(JunctionParams)]
    lib.ptadd_set_junctions.restype = st
    lib.ptadd_get_junctions.argtypes = [_VP, ctypes.POINTER(JunctionInfo), _I32, _I32, _I32, _D]
    lib.ptadd_get_junctions.restype = st
    lib.ptadd_set_mobility.argtypes = [_VP, ctypes.c_int32]
    lib.ptadd_set_mobility.restype = st
    lib.ptadd_batch_set_junctions.argtypes = [_VP, ctypes.POINTER(JunctionParams)]
    lib.ptadd_batch_set_junctions.restype = st
    lib.ptadd_batch_get_junctions.argtypes = [_VP, ctypes.POINTER(JunctionInfo), _I32, _I32, _I32, _D]
    lib.ptadd_batch_get_junctions.restype = st
    lib.ptadd_system_densities.argtypes = [ctypes.c_int64, _D, ctypes.c_int64, _I64, _D, _D, _U8, ctypes.c_double, _D]
    lib.ptadd_system_densities.restype = st
    lib.ptadd_block_average.argtypes = [ctypes.c_int64, _D, _D, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, _D]
    lib.ptadd_block_average.restype = st
    lib.ptadd_block_stress_pair.argtypes = [ctypes.c_int32, _D, _D, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, _D, _D, _D]
    lib.ptadd_block_stress_pair.restype = st
    lib.ptadd_surrogate_get_state.argtypes = [_VP, _VP, ctypes.POINTER(ctypes.c_size_t)]
    lib.ptadd_surrogate_get_state.restype = st
    lib.ptadd_surrogate_set_state.argtypes = [_VP, _VP, ctypes.c_size_t]
    lib.ptadd_surrogate_set_state.restype = st
    lib.ptadd_fma_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _D]
    lib.ptadd_fma_peak.restype = st
    _lib = lib
    return lib


def _check(status):
    if status != 0:
        raise PtaddError(status, _lib.ptadd_last_error().decode())


def _dptr(a):
    return a.ctypes.data_as(_D)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def version():
    return load().ptadd_version()


def fma_peak(device=0, fp64=True, seconds=1.0, packed=False):
    """Measured FMA throughput (FLOP/s) of every SM: FP64, FP32, or packed FP32 pairs."""
    lib = load()
    out = ctypes.c_double(0.0)
    mode = 2 if packed else (1 if fp64 else 0)
    _check(lib.ptadd_fma_peak(int(device), mode, float(seconds), ctypes.byref(out)))
    return out.value


def forces_noalloc(material, n_nodes, xyz_ptr, nxt_ptr, prv_ptr, burgers_ptr, sig_app, F_ptr, stream=None):
    """ptadd_forces_noalloc on caller-owned device buffers (raw device pointers).

    Allocates no device memory; see ptadd.h for the scratch-array contract
    (fixed maximum size, first call per device before any stream capture,
    overlapping calls race)."""
    lib = load()
    m = Material(*tuple(material))
    s = _c(sig_app, np.float64)
    _check(lib.ptadd_forces_noalloc(ctypes.byref(m), int(n_nodes), _VP(xyz_ptr), _VP(nxt_ptr), _VP(prv_ptr),
                                    _VP(burgers_ptr), _dptr(s), _VP(F_ptr), _VP(stream) if stream else None))


def mlp_param_count():
    return int(load().ptadd_mlp_param_count())


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def closure_realisation(material, seed, rho24, n_loops):
    """ptadd_closure_realisation: one stratified realisation for the 24
    densities (host only).  Returns (xyz [32 n_loops, 3], burgers [n_loops, 3],
    normal [n_loops, 3], pinned [32 n_loops], volume)."""
    lib = load()
    m = Material(*tuple(material))
    r = _c(rho24, np.float64)
    xyz = np.zeros((32 * n_loops, 3))
    b = np.zeros((n_loops, 3))
    nv = np.zeros((n_loops, 3))
    pin = np.zeros(32 * n_loops, np.uint8)
    vol = ctypes.c_double(0.0)
    _check(lib.ptadd_closure_realisation(ctypes.byref(m), ctypes.c_uint64(seed), _dptr(r), int(n_loops), _dptr(xyz),
                                         _dptr(b), _dptr(nv), pin.ctypes.data_as(_U8), ctypes.byref(vol)))
    return xyz, b, nv, pin, vol.value


def dissipation_projection(T6, Lp, V=None, alpha=None):
    """ptadd_dissipation_projection (host only): returns the corrected
    (Lp [3,3], V [3] or None)."""
    lib = load()
    t = _c(T6, np.float64)
    L = np.array(Lp, dtype=np.float64).reshape(9)
    v = None if V is None else np.array(V, dtype=np.float64).reshape(3)
    a = None if alpha is None else _c(np.asarray(alpha, np.float64).reshape(9), np.float64)
    _check(lib.ptadd_dissipation_projection(_dptr(t), _dptr(a) if a is not None else None, _dptr(L),
                                            _dptr(v) if v is not None else None))
    return L.reshape(3, 3), v


def dissipation_projection_dev(n_points, T6_ptr, Lp_ptr, alpha_ptr=None, V_ptr=None, n_bad_ptr=None, stream=None):
    """ptadd_dissipation_projection_dev on caller-owned device arrays (raw pointers)."""
    lib = load()
    _check(lib.ptadd_dissipation_projection_dev(int(n_points), _VP(T6_ptr), _VP(alpha_ptr) if alpha_ptr else None,
                                                _VP(Lp_ptr), _VP(V_ptr) if V_ptr else None,
                                                _VP(n_bad_ptr) if n_bad_ptr else None, _VP(stream) if stream else None))


def system_densities(net, xyz=None):
    """ptadd_system_densities (host only): [24] line densities (1/m^2),
    12 mobile then 12 sessile, of `net` (positions `xyz` if given)."""
    lib = load()
    x = _c(net.xyz if xyz is None else xyz, np.float64)
    off = _c(net.loop_off, np.int64)
    bv = _c(net.burgers, np.float64)
    nv = _c(net.normal, np.float64)
    pin = _c(net.pinned, np.uint8) if net.pinned is not None else None
    out = np.zeros(24)
    _check(lib.ptadd_system_densities(x.shape[0], _dptr(x), off.shape[0] - 1, off.ctypes.data_as(_I64), _dptr(bv),
                                      _dptr(nv), pin.ctypes.data_as(_U8) if pin is not None else None,
                                      float(net.volume), _dptr(out)))
    return out


def block_average(T6, w, block, n_blocks):
    """ptadd_block_average (host only): volume-weighted block averages of the
    Gauss-point stresses T6 [n, 6] with weights w [n] and block indices
    block [n]; returns [n_blocks, 6]."""
    lib = load()
    t = _c(T6, np.float64).reshape(-1, 6)
    ww = _c(w, np.float64).reshape(-1)
    bl = _c(block, np.int32).reshape(-1)
    if not (t.shape[0] == ww.shape[0] == bl.shape[0]):
        raise ValueError("T6, w and block must describe the same Gauss points")
    out = np.zeros((int(n_blocks), 6))
    _check(lib.ptadd_block_average(t.shape[0], _dptr(t), _dptr(ww), bl.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   int(n_blocks), _dptr(out)))
    return out


def block_stress_pair(T6_k, T6_km1, delta_star, dt_prev, gap_min):
    """ptadd_block_stress_pair (host only): returns (T_prev [R, 6],
    T_t [R, 6], mag [R]) for the block stresses T6_k [R, 6] and
    T6_km1 [R, 6] (or None)."""
    lib = load()
    tk = _c(T6_k, np.float64).reshape(-1, 6)
    tm = None if T6_km1 is None else _c(T6_km1, np.float64).reshape(-1, 6)
    if tm is not None and tm.shape != tk.shape:
        raise ValueError("T6_k and T6_km1 differ in shape")
    R = tk.shape[0]
    tp, tt, mag = np.zeros((R, 6)), np.zeros((R, 6)), np.zeros(R)
    _check(lib.ptadd_block_stress_pair(R, _dptr(tk), _dptr(tm) if tm is not None else None, float(delta_star),
                                       float(dt_prev), float(gap_min), _dptr(tp), _dptr(tt), _dptr(mag)))
    return tp, tt, mag


def gemm_bf16(A_bits, B_bits, device=0):
    """C = A B^T on the tensor cores; A [M,K], B [N,K] as uint16 BF16 bit patterns."""
    lib = load()
    A = np.ascontiguousarray(A_bits, dtype=np.uint16)
    B = np.ascontiguousarray(B_bits, dtype=np.uint16)
    M, K = A.shape
    N = B.shape[0]
    C = np.zeros((M, N), dtype=np.float32)
    _check(lib.ptadd_gemm_bf16(int(device), M, N, K, A.ctypes.data, B.ctypes.data, C.ctypes.data))
    return C


def gemm_timeout_selftest(device=0):
    """Status of ptadd_gemm_timeout_selftest (PTADD_ERR_TIMEOUT = 4 expected)."""
    return int(load().ptadd_gemm_timeout_selftest(int(device)))


def to_bf16_bits(x):
    """Round-to-nearest-even FP32 -> BF16 bit patterns (uint16)."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u >> 16) & 1) + 0x7FFF
    return ((u + r) >> 16).astype(np.uint16)


def from_bf16_bits(b):
    return (np.asarray(b, dtype=np.uint32) << 16).view(np.float32)


class Context:
    """One realisation on one GPU (wraps ptadd_ctx)."""

    def __init__(self, material, precision=PTADD_FP64, device=0):
        lib = load()
        self._lib = lib
        self._h = _VP()
        m = Material(*tuple(material))
        _check(lib.ptadd_create(ctypes.byref(self._h), ctypes.byref(m), int(precision), int(device)))
        self.n_nodes = 0

    def close(self):
        if self._h:
            self._lib.ptadd_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_precision(self, precision):
        _check(self._lib.ptadd_set_precision(self._h, int(precision)))

    def set_stream(self, stream_handle):
        """stream_handle: an int cudaStream_t (e.g. torch.cuda.current_stream().cuda_stream) or None."""
        _check(self._lib.ptadd_set_stream(self._h, _VP(stream_handle) if stream_handle else None))

    def set_network(self, net):
        """net: workloads.Network (SI).  Also loads its applied stress."""
        x = _c(net.xyz, np.float64)
        off = _c(net.loop_off, np.int64)
        bv = _c(net.burgers, np.float64)
        nv = _c(net.normal, np.float64)
        pin = _c(net.pinned, np.uint8) if net.pinned is not None else None
        _check(self._lib.ptadd_set_network(self._h, x.shape[0], _dptr(x), off.shape[0] - 1,
                                           off.ctypes.data_as(_I64), _dptr(bv), _dptr(nv),
                                           pin.ctypes.data_as(_U8) if pin is not None else None,
                                           float(net.volume)))
        self.n_nodes = x.shape[0]
        self.set_applied_stress(net.sig_app)

    def set_applied_stress(self, sig6):
        s = _c(sig6, np.float64)
        _check(self._lib.ptadd_set_applied_stress(self._h, _dptr(s)))

    def info(self):
        i = Info()
        _check(self._lib.ptadd_get_info(self._h, ctypes.byref(i)))
        return dict(n_nodes=i.n_nodes, n_loops=i.n_loops, n_targets=i.n_targets,
                    pairs_per_step=i.pairs_per_step, precision=i.precision, device=i.device)

    def advance(self, n_steps, dt):
        """Run a burst; returns (Lp_avg 3x3, rho_avg)."""
        Lp = np.zeros(9)
        rho = ctypes.c_double(0.0)
        _check(self._lib.ptadd_advance(self._h, int(n_steps), float(dt), _dptr(Lp), ctypes.byref(rho)))
        return Lp.reshape(3, 3), rho.value

    def get_polar_velocity(self, core_area):
        """R^V (m/s) of the last burst, Eq. 2.11 with one core area for every segment."""
        V = np.zeros(3)
        _check(self._lib.ptadd_get_polar_velocity(self._h, float(core_area), _dptr(V)))
        return V

    def get_nodes(self):
        out = np.zeros((self.n_nodes, 3))
        _check(self._lib.ptadd_get_nodes(self._h, _dptr(out)))
        return out

    def set_nodes(self, xyz):
        """xyz: [n,3] float64 host array (SI) or a raw host pointer (int)."""
        if isinstance(xyz, int):
            _check(self._lib.ptadd_set_nodes(self._h, _VP(xyz)))
            return
        x = _c(xyz, np.float64)
        _check(self._lib.ptadd_set_nodes(self._h, x.ctypes.data_as(_VP)))

    def get_nodes_into(self, ptr):
        """Positions into a caller-owned host buffer given as a raw pointer."""
        _check(self._lib.ptadd_get_nodes(self._h, ctypes.cast(_VP(ptr), _D)))

    def profile_reset(self, timing=False):
        _check(self._lib.ptadd_profile_reset(self._h, int(bool(timing))))

    def profile_read(self):
        p = Profile()
        _check(self._lib.ptadd_profile_read(self._h, ctypes.byref(p)))
        return dict(kernel_launches=p.kernel_launches, pair_launches=p.pair_launches,
                    pair_evals=p.pair_evals, pair_ms=p.pair_ms, near_point_pairs=p.near_point_pairs)

    def get_forces(self):
        out = np.zeros((self.n_nodes, 3))
        _check(self._lib.ptadd_get_forces(self._h, _dptr(out)))
        return out

    def get_forces_dev(self, ptr):
        _check(self._lib.ptadd_get_forces_dev(self._h, _VP(ptr)))

    def get_state(self):
        n = ctypes.c_size_t(0)
        _check(self._lib.ptadd_get_state(self._h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(self._lib.ptadd_get_state(self._h, ctypes.cast(buf, _VP), ctypes.byref(n)))
        return bytes(buf.raw[:n.value])

    def set_state(self, blob):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(self._lib.ptadd_set_state(self._h, ctypes.cast(buf, _VP), len(blob)))

    def set_mobility(self, consistent):
        """ptadd_set_mobility: True for the consistent (Galerkin) mass matrix of Eq. 2.1."""
        _check(self._lib.ptadd_set_mobility(self._h, int(bool(consistent))))

    # ---------------------------------------------------------- junctions
    def set_junctions(self, capture_radius=None, max_break_time=1e-3, stuck_disp=0.0, seed=0):
        """ptadd_set_junctions; capture_radius None switches junctions off."""
        if capture_radius is None:
            _check(self._lib.ptadd_set_junctions(self._h, None))
            return
        p = JunctionParams(float(capture_radius), float(max_break_time), float(stuck_disp), int(seed))
        _check(self._lib.ptadd_set_junctions(self._h, ctypes.byref(p)))

    def junctions(self):
        """ptadd_get_junctions: dict(clock, jumped, held, formed, broken,
        jumps, seg, last, count, break_time)."""
        n = self.info()["n_nodes"]
        info = JunctionInfo()
        seg, last, cnt = (np.zeros(n, np.int32) for _ in range(3))
        brk = np.zeros(n)
        i32 = ctypes.POINTER(ctypes.c_int32)
        _check(self._lib.ptadd_get_junctions(self._h, ctypes.byref(info), seg.ctypes.data_as(i32),
                                             last.ctypes.data_as(i32), cnt.ctypes.data_as(i32), _dptr(brk)))
        out = {k: getattr(info, k) for k, _ in JunctionInfo._fields_}
        out.update(seg=seg, last=last, count=cnt, break_time=brk)
        return out

    # ------------------------------------------------------------ batched
    def batch_set(self, batch):
        """batch: workloads.Batch (SI)."""
        b = batch
        self._batch_keep = [_c(b.node_off, np.int64), _c(b.loop_off, np.int64), _c(b.xyz, np.float64),
                            _c(b.burgers, np.float64), _c(b.normal, np.float64), _c(b.pinned, np.uint8),
                            _c(b.sig6, np.float64), _c(b.volume, np.float64)]
        no, lo, x, bv, nv, pin, sg, vol = self._batch_keep
        _check(self._lib.ptadd_batch_set(self._h, int(b.R), no.ctypes.data_as(_I64), lo.shape[0] - 1,
                                         lo.ctypes.data_as(_I64), _dptr(x), _dptr(bv), _dptr(nv),
                                         pin.ctypes.data_as(_U8), _dptr(sg), _dptr(vol)))
        self.batch_R = int(b.R)
        self.batch_n = int(x.shape[0])
        self._batch_keep = None

    def batch_set_stress(self, sig6):
        s = _c(sig6, np.float64).reshape(-1)
        _check(self._lib.ptadd_batch_set_stress(self._h, _dptr(s)))

    def batch_advance(self, n_steps, dt):
        """Returns (Lp_avg [R,3,3], rho_avg [R])."""
        Lp = np.zeros(9 * self.batch_R)
        rho = np.zeros(self.batch_R)
        _check(self._lib.ptadd_batch_advance(self._h, int(n_steps), float(dt), _dptr(Lp), _dptr(rho)))
        return Lp.reshape(-1, 3, 3), rho

    def batch_get_nodes(self):
        out = np.zeros((self.batch_n, 3))
        _check(self._lib.ptadd_batch_get_nodes(self._h, _dptr(out)))
        return out

    def batch_set_nodes(self, xyz):
        x = _c(xyz, np.float64)
        _check(self._lib.ptadd_batch_set_nodes(self._h, _dptr(x)))

    def batch_info(self):
        i = BatchInfo()
        _check(self._lib.ptadd_batch_get_info(self._h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in BatchInfo._fields_}

    def batch_get_polar_velocity(self, core_area):
        """R^V [R, 3] (m/s) of the last batch burst."""
        V = np.zeros(3 * self.batch_R)
        _check(self._lib.ptadd_batch_get_polar_velocity(self._h, float(core_area), _dptr(V)))
        return V.reshape(-1, 3)

    def batch_configure(self, tile_targets, chunk_sources):
        _check(self._lib.ptadd_batch_configure(self._h, int(tile_targets), int(chunk_sources)))

    def batch_get_forces(self):
        """Nodal forces [n_nodes, 3] (N) at the current positions; 0 at pinned nodes."""
        out = np.zeros((self.batch_n, 3))
        _check(self._lib.ptadd_batch_get_forces(self._h, _dptr(out)))
        return out

    def batch_set_junctions(self, capture_radius=None, max_break_time=1e-3, stuck_disp=0.0, seed=0):
        """ptadd_batch_set_junctions; capture_radius None switches them off."""
        if capture_radius is None:
            _check(self._lib.ptadd_batch_set_junctions(self._h, None))
            return
        p = JunctionParams(float(capture_radius), float(max_break_time), float(stuck_disp), int(seed))
        _check(self._lib.ptadd_batch_set_junctions(self._h, ctypes.byref(p)))

    def batch_junctions(self):
        """ptadd_batch_get_junctions: list of R dicts (clock, jumped, held,
        formed, broken, jumps) and the per-node arrays seg, last, count,
        break_time [n_nodes] in realisation-local numbers."""
        R, n = self.batch_R, self.batch_n
        info = (JunctionInfo * R)()
        seg, last, cnt = (np.zeros(n, np.int32) for _ in range(3))
        brk = np.zeros(n)
        i32 = ctypes.POINTER(ctypes.c_int32)
        _check(self._lib.ptadd_batch_get_junctions(self._h, info, seg.ctypes.data_as(i32), last.ctypes.data_as(i32),
                                                   cnt.ctypes.data_as(i32), _dptr(brk)))
        per = [{k: getattr(info[r], k) for k, _ in JunctionInfo._fields_} for r in range(R)]
        return per, dict(seg=seg, last=last, count=cnt, break_time=brk)

    def batch_autotune(self, cache_path=None, force=False):
        _check(self._lib.ptadd_batch_autotune(self._h, cache_path.encode() if cache_path else None,
                                              int(bool(force))))

    # ---------------------------------------------------------- surrogate
    def mlp_init(self, seed=0):
        _check(self._lib.ptadd_mlp_init(self._h, int(seed)))

    def mlp_set_params(self, params):
        p = _c(params, np.float32)
        _check(self._lib.ptadd_mlp_set_params(self._h, _fptr(p), p.size))

    def mlp_get_params(self):
        p = np.zeros(mlp_param_count(), np.float32)
        _check(self._lib.ptadd_mlp_get_params(self._h, _fptr(p), p.size))
        return p

    def mlp_loss_grad(self, xn, yn):
        x = _c(xn, np.float32)
        y = _c(yn, np.float32)
        g = np.zeros(mlp_param_count(), np.float32)
        loss = ctypes.c_float(0.0)
        _check(self._lib.ptadd_mlp_loss_grad(self._h, x.shape[0], _fptr(x), _fptr(y), _fptr(g), ctypes.byref(loss)))
        return loss.value, g

    def mlp_train(self, xn, yn, epochs, batch=512, lr=1e-3, seed=0):
        x = _c(xn, np.float32)
        y = _c(yn, np.float32)
        losses = np.zeros(max(1, epochs), np.float32)
        _check(self._lib.ptadd_mlp_train(self._h, x.shape[0], _fptr(x), _fptr(y), int(epochs), int(batch),
                                         float(lr), int(seed), _fptr(losses)))
        return losses[:epochs]

    def mlp_forward(self, xn):
        x = _c(xn, np.float32)
        y = np.zeros((x.shape[0], 6), np.float32)
        _check(self._lib.ptadd_mlp_forward(self._h, x.shape[0], _fptr(x), _fptr(y)))
        return y

    def surrogate_fit(self, feat, lp6, epochs, batch=512, lr=1e-3, seed=0):
        f = _c(feat, np.float64)
        y = _c(lp6, np.float64)
        losses = np.zeros(max(1, epochs), np.float32)
        _check(self._lib.ptadd_surrogate_fit(self._h, f.shape[0], _dptr(f), _dptr(y), int(epochs), int(batch),
                                             float(lr), int(seed), _fptr(losses)))
        return losses[:epochs]

    def surrogate_predict(self, feat):
        """Returns (lp6 [n,6], in_region [n] bool)."""
        f = _c(feat, np.float64)
        y = np.zeros((f.shape[0], 6))
        r = np.zeros(f.shape[0], np.uint8)
        _check(self._lib.ptadd_surrogate_predict(self._h, f.shape[0], _dptr(f), _dptr(y),
                                                 r.ctypes.data_as(_U8)))
        return y, r.astype(bool)

    def surrogate_predict_dev(self, n, feat_ptr, lp6_ptr, region_ptr=None):
        _check(self._lib.ptadd_surrogate_predict_dev(self._h, int(n), _VP(feat_ptr), _VP(lp6_ptr),
                                                     _VP(region_ptr) if region_ptr else None))

    def closure_sweep(self, sig6, rho24, ens, segments, steps, dt, seed):
        """ptadd_closure_sweep: (lp6 [n, 6], used_fallback [n] bool)."""
        s6 = _c(sig6, np.float64)
        r = _c(rho24, np.float64)
        n = s6.shape[0]
        out = np.zeros((n, 6))
        used = np.zeros(n, np.uint8)
        _check(self._lib.ptadd_closure_sweep(self._h, n, _dptr(s6), _dptr(r), int(ens), int(segments), int(steps),
                                             float(dt), ctypes.c_uint64(seed), _dptr(out), used.ctypes.data_as(_U8)))
        return out, used.astype(bool)

    def surrogate_get_state(self):
        n = ctypes.c_size_t(0)
        _check(self._lib.ptadd_surrogate_get_state(self._h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(self._lib.ptadd_surrogate_get_state(self._h, ctypes.cast(buf, _VP), ctypes.byref(n)))
        return bytes(buf.raw[:n.value])

    def surrogate_set_state(self, blob):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(self._lib.ptadd_surrogate_set_state(self._h, ctypes.cast(buf, _VP), len(blob)))
