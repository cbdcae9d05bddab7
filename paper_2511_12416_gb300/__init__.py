"""Python binding of libextraferm, the GB300 extended-matchgate probability
library (C ABI in ``include/extraferm.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library. The functions carry the C names; host-pointer calls take numpy
arrays, ``*_dev`` calls take device pointers (``int``) and a CUDA stream
handle (``int``, e.g. ``torch.cuda.current_stream().cuda_stream``).
There is no CPU fallback: ``load()`` raises if the library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from ._build import build, lib_path  # noqa: F401

EF_OK, EF_EINVAL, EF_ENOMEM, EF_ECUDA, EF_ETIMEOUT, EF_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
EF_GIVENS, EF_PHASE, EF_CPHASE = 0, 1, 2
EF_PREC_FP64, EF_PREC_FP32_MINOR, EF_PREC_AUTO = 0, 1, 2
EF_FLAG_TIME_KERNELS = 1

_STATUS = {0: "EF_OK", -1: "EF_EINVAL", -2: "EF_ENOMEM", -3: "EF_ECUDA", -4: "EF_ETIMEOUT", -5: "EF_EUNSUPPORTED"}


class EfGate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("p", ctypes.c_int32), ("q", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("theta", ctypes.c_double), ("phi", ctypes.c_double)]


class EfOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("flags", ctypes.c_int32), ("tol", ctypes.c_double),
                ("tile_override", ctypes.c_int32 * 4)]


class EfStats(ctypes.Structure):
    _fields_ = [("logical_branch_dets", ctypes.c_int64), ("executed_minor_lus", ctypes.c_int64),
                ("fp64_recomputed", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("sampled_flips", ctypes.c_int64), ("max_est_rel_err", ctypes.c_double),
                ("dominant_kernel_ms", ctypes.c_double), ("dominant_kernel_launches", ctypes.c_int64),
                ("dominant_kernel_flops", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


# name -> (restype, argtypes); the exported C ABI
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_DP = ctypes.POINTER(ctypes.c_double)
_U64P = ctypes.POINTER(ctypes.c_uint64)
SIGNATURES = {
    "ef_version": (ctypes.c_int, []),
    "ef_last_error": (ctypes.c_char_p, []),
    "ef_circuit_create": (ctypes.c_int, [ctypes.c_int32, _U64P, ctypes.POINTER(EfGate), _I64,
                                         ctypes.POINTER(EfOptions), ctypes.POINTER(_P)]),
    "ef_circuit_destroy": (ctypes.c_int, [_P]),
    "ef_circuit_num_angles": (ctypes.c_int, [_P, ctypes.POINTER(_I64)]),
    "ef_circuit_get_angles": (ctypes.c_int, [_P, _DP, _I64]),
    "ef_circuit_set_angles": (ctypes.c_int, [_P, _DP, _I64]),
    "ef_circuit_extent": (ctypes.c_int, [_P, _DP]),
    "ef_circuit_set_precision": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double]),
    "ef_prob_exact": (ctypes.c_int, [_P, _U64P, _I64, _DP, _DP]),
    "ef_prob_exact_dev": (ctypes.c_int, [_P, _P, _I64, _P, _P, _P]),
    "ef_prob_approx": (ctypes.c_int, [_P, _U64P, _I64, _I64, _U64, _U64, _DP, _DP, _DP]),
    "ef_prob_approx_dev": (ctypes.c_int, [_P, _P, _I64, _I64, _U64, _U64, _P, _P, _P, _P]),
    "ef_prob_estimate": (ctypes.c_int, [_P, _U64P, _I64, ctypes.c_double, ctypes.c_double, _U64, _U64, _DP, _DP,
                                        ctypes.POINTER(_I64)]),
    "ef_prob_grad": (ctypes.c_int, [_P, _U64P, _I64, _DP, _DP, _DP]),
    "ef_prob_grad_dev": (ctypes.c_int, [_P, _P, _I64, _P, _P, _P, _P]),
    "ef_circuit_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(EfStats)]),
    "ef_prob_exact_noalloc_dev": (ctypes.c_int, [_P, _P, _I64, _P, _P, _P]),
    "ef_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, ctypes.POINTER(_P)]),
    "ef_batch_destroy": (ctypes.c_int, [_P]),
    "ef_batch_prob_dev": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_I64), ctypes.POINTER(_P),
                                         ctypes.POINTER(_I64), _U64, _P]),
    "ef_batch_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(EfStats)]),
    "ef_measure_peak": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _DP]),
}

_lib = None


class ExtraFermError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


def load(path: str | None = None):
    """Load libextraferm (building it first if it is missing and nvcc is
    available). Raises if the CUDA library cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or lib_path()
    if not os.path.exists(path):
        build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int):
    if rc != EF_OK:
        raise ExtraFermError(rc, _lib.ef_last_error().decode())


def _dptr(a):
    return a.ctypes.data_as(_DP) if a is not None else None


def _bits_array(bits) -> np.ndarray:
    b = np.ascontiguousarray(np.asarray(bits, dtype=np.uint64).reshape(-1, 2))
    return b


# ------------------------------------------------------------------ functions with the C names


def ef_version() -> int:
    return load().ef_version()


def ef_last_error() -> str:
    return load().ef_last_error().decode()


def ef_circuit_create(n_modes: int, occupation, gates, precision: int = EF_PREC_AUTO, tol: float = 1e-5,
                      flags: int = 0, tile_override=(0, 0, 0, 0)):
    """gates: numpy structured array with fields kind, p, q, theta, phi (or
    any sequence of such records). Returns an opaque handle (c_void_p)."""
    lib = load()
    g = np.asarray(gates)
    arr = (EfGate * max(1, len(g)))()
    for i, rec in enumerate(g):
        arr[i].kind = int(rec["kind"])
        arr[i].p = int(rec["p"])
        arr[i].q = int(rec["q"])
        arr[i].reserved = 0
        arr[i].theta = float(rec["theta"])
        arr[i].phi = float(rec["phi"])
    occ = np.ascontiguousarray(np.asarray(occupation, dtype=np.uint64).reshape(2))
    opt = EfOptions(precision, flags, tol, (ctypes.c_int32 * 4)(*tile_override))
    h = _P()
    _check(lib.ef_circuit_create(int(n_modes), occ.ctypes.data_as(_U64P), arr, len(g), ctypes.byref(opt),
                                 ctypes.byref(h)))
    return h


def ef_circuit_destroy(c):
    if c:
        _check(load().ef_circuit_destroy(c))


def ef_circuit_num_angles(c) -> int:
    n = _I64()
    _check(load().ef_circuit_num_angles(c, ctypes.byref(n)))
    return n.value


def ef_circuit_get_angles(c) -> np.ndarray:
    n = ef_circuit_num_angles(c)
    a = np.zeros(n)
    _check(load().ef_circuit_get_angles(c, _dptr(a), n))
    return a


def ef_circuit_set_angles(c, angles):
    a = np.ascontiguousarray(np.asarray(angles, dtype=np.float64))
    _check(load().ef_circuit_set_angles(c, _dptr(a), len(a)))


def ef_circuit_extent(c) -> float:
    x = ctypes.c_double()
    _check(load().ef_circuit_extent(c, ctypes.byref(x)))
    return x.value


def ef_circuit_set_precision(c, precision: int, tol: float = 0.0):
    _check(load().ef_circuit_set_precision(c, precision, tol))


def ef_prob_exact(c, bits, want_err: bool = False):
    b = _bits_array(bits)
    nb = b.shape[0]
    out = np.zeros(nb)
    err = np.zeros(nb) if want_err else None
    _check(load().ef_prob_exact(c, b.ctypes.data_as(_U64P), nb, _dptr(out), _dptr(err)))
    return (out, err) if want_err else out


def ef_prob_exact_dev(c, d_bits: int, nb: int, d_out: int, d_err: int = 0, stream: int = 0):
    _check(load().ef_prob_exact_dev(c, d_bits, nb, d_out, d_err or None, stream or None))


def ef_prob_exact_noalloc_dev(c, d_bits: int, nb: int, d_out: int, d_err: int = 0, stream: int = 0):
    """Exact probabilities without any device allocation by the library: all
    scratch comes from the library's fixed 64 MiB per-GPU array (see
    extraferm.h for who needs this, the size limit and the ordering rule)."""
    _check(load().ef_prob_exact_noalloc_dev(c, d_bits, nb, d_out, d_err or None, stream or None))


def ef_prob_approx(c, bits, n_traj: int, seed: int = 0, index_base: int = 0, want_stderr: bool = True,
                   want_err: bool = False):
    """Returns p_hat, then stderr (want_stderr) and the estimated relative
    error of p_hat (want_err) as further arrays."""
    b = _bits_array(bits)
    nb = b.shape[0]
    out = np.zeros(nb)
    se = np.zeros(nb) if want_stderr else None
    err = np.zeros(nb) if want_err else None
    _check(load().ef_prob_approx(c, b.ctypes.data_as(_U64P), nb, int(n_traj), int(seed), int(index_base),
                                 _dptr(out), _dptr(se), _dptr(err)))
    res = (out,) + ((se,) if want_stderr else ()) + ((err,) if want_err else ())
    return res if len(res) > 1 else out


def ef_prob_approx_dev(c, d_bits: int, nb: int, n_traj: int, seed: int, index_base: int, d_out: int,
                       d_stderr: int = 0, stream: int = 0, d_err: int = 0):
    _check(load().ef_prob_approx_dev(c, d_bits, nb, int(n_traj), int(seed), int(index_base), d_out,
                                     d_stderr or None, d_err or None, stream or None))


def ef_prob_estimate(c, bits, eps: float, delta: float, seed: int = 0, index_base: int = 0):
    """Estimate (eps, delta): returns (p_hat, stderr, trajectories per bitstring)."""
    b = _bits_array(bits)
    nb = b.shape[0]
    out = np.zeros(nb)
    se = np.zeros(nb)
    traj = np.zeros(nb, dtype=np.int64)
    _check(load().ef_prob_estimate(c, b.ctypes.data_as(_U64P), nb, float(eps), float(delta), int(seed),
                                   int(index_base), _dptr(out), _dptr(se), traj.ctypes.data_as(ctypes.POINTER(_I64))))
    return out, se, traj


def ef_prob_grad(c, bits, grad_p):
    b = _bits_array(bits)
    nb = b.shape[0]
    g = np.ascontiguousarray(np.asarray(grad_p, dtype=np.float64))
    out_p = np.zeros(nb)
    grad = np.zeros(ef_circuit_num_angles(c))
    _check(load().ef_prob_grad(c, b.ctypes.data_as(_U64P), nb, _dptr(g), _dptr(out_p), _dptr(grad)))
    return out_p, grad


def ef_prob_grad_dev(c, d_bits: int, nb: int, d_grad_p: int, d_out_p: int, d_grad: int, stream: int = 0):
    _check(load().ef_prob_grad_dev(c, d_bits, nb, d_grad_p, d_out_p or None, d_grad, stream or None))


def ef_circuit_get_stats(c) -> dict:
    st = EfStats()
    _check(load().ef_circuit_get_stats(c, ctypes.byref(st)))
    return st.as_dict()


def ef_batch_create(circuits):
    """Batch over circuit handles (the batch does not own them)."""
    arr = (_P * len(circuits))(*[c.value if isinstance(c, _P) else c for c in circuits])
    h = _P()
    _check(load().ef_batch_create(arr, len(circuits), ctypes.byref(h)))
    return h


def ef_batch_destroy(b):
    if b:
        _check(load().ef_batch_destroy(b))


def ef_batch_prob_dev(b, d_bits, nb, d_out, n_traj, seed: int = 0, stream: int = 0):
    """d_bits, d_out: sequences of device pointers; nb, n_traj: sequences of
    ints (n_traj 0 = Exact, > 0 = Raw Estimate with that many trajectories)."""
    n = len(nb)
    _check(load().ef_batch_prob_dev(b, (_P * n)(*d_bits), (_I64 * n)(*nb), (_P * n)(*d_out), (_I64 * n)(*n_traj),
                                    int(seed), stream or None))


def ef_batch_get_stats(b) -> dict:
    st = EfStats()
    _check(load().ef_batch_get_stats(b, ctypes.byref(st)))
    return st.as_dict()


class Circuit:
    """Owning handle: ``with Circuit(n, occupation, gates) as c: ...``."""

    def __init__(self, n_modes, occupation, gates, **kw):
        self.handle = ef_circuit_create(n_modes, occupation, gates, **kw)

    def close(self):
        if self.handle:
            ef_circuit_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PEAK_FP32, PEAK_FP32X2, PEAK_FP64, PEAK_PHILOX = 0, 1, 2, 3


def ef_measure_peak(kind: int, reps: int = 5) -> float:
    """Measured rate of the current GPU: flops/s (FP32 scalar, FP32 packed,
    FP64) or Philox4x32-10 blocks/s."""
    r = ctypes.c_double()
    _check(load().ef_measure_peak(int(kind), int(reps), ctypes.byref(r)))
    return r.value
