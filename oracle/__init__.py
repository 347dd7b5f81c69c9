"""FP64 CPU oracle for the d-dimensional DFT and the cyclic four-step method.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only users.  Nothing in the CUDA library imports,
links or calls anything here, and nothing here uses the CUDA library.

* ``fftn`` / ``fft_axis`` / ``dft_bruteforce`` / ``dft_points`` wrap the plain C
  code in ``fftu_oracle.c`` (eq. dftd of Sec. 1, row-column as in Sec. 1.2).
* ``cyclic_model`` restates Algorithm 2.3 (Sec. 2.2) superstep by superstep on
  explicit virtual processors, for stage-level checks.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fftu_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math, no -march)."""
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64p = ctypes.POINTER(ctypes.c_int64)
            dp = ctypes.c_void_p
            lib.oracle_fft_axis.argtypes = [ctypes.c_int, i64p, ctypes.c_int, dp, ctypes.c_int]
            lib.oracle_fftn.argtypes = [ctypes.c_int, i64p, dp, dp, ctypes.c_int]
            lib.oracle_dft_bruteforce.argtypes = [ctypes.c_int, i64p, dp, dp, ctypes.c_int]
            lib.oracle_dft_points.argtypes = [ctypes.c_int, i64p, dp, ctypes.c_int64, i64p, dp,
                                              ctypes.c_int]
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_max_threads.restype = ctypes.c_int
            for f in (lib.oracle_fft_axis, lib.oracle_fftn, lib.oracle_dft_bruteforce,
                      lib.oracle_dft_points):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _shape_arg(shape):
    arr = (ctypes.c_int64 * len(shape))(*[int(s) for s in shape])
    return arr


def _as_c128(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x), dtype=np.complex128)


def set_threads(n: int) -> None:
    """Number of OpenMP threads the oracle uses (0 = all available)."""
    _load().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def fft_axis(x, axis: int, sign: int = -1) -> np.ndarray:
    """Unscaled 1D DFT along one axis; sign -1 uses w = exp(-2 pi i/n), +1 its conjugate."""
    y = _as_c128(x).copy()
    rc = _load().oracle_fft_axis(y.ndim, _shape_arg(y.shape), int(axis) % y.ndim,
                                 y.ctypes.data, int(sign))
    if rc != 0:
        raise RuntimeError("oracle_fft_axis failed")
    return y


def fftn(x, inverse: bool = False) -> np.ndarray:
    """d-dim DFT (eq. dftd); inverse: conjugated weights and 1/N (Sec. 1.3)."""
    x = _as_c128(x)
    y = np.empty_like(x)
    rc = _load().oracle_fftn(x.ndim, _shape_arg(x.shape), x.ctypes.data, y.ctypes.data,
                             int(bool(inverse)))
    if rc != 0:
        raise RuntimeError("oracle_fftn failed")
    return y


def dft_bruteforce(x, inverse: bool = False) -> np.ndarray:
    """eq. dftd summed directly, O(N^2); for small arrays only."""
    x = _as_c128(x)
    y = np.empty_like(x)
    rc = _load().oracle_dft_bruteforce(x.ndim, _shape_arg(x.shape), x.ctypes.data,
                                       y.ctypes.data, int(bool(inverse)))
    if rc != 0:
        raise RuntimeError("oracle_dft_bruteforce failed")
    return y


def dft_points(x, ks, inverse: bool = False) -> np.ndarray:
    """eq. dftd at chosen output indices ks (npts x d), O(N) per point."""
    x = _as_c128(x)
    ks = np.ascontiguousarray(np.asarray(ks, dtype=np.int64).reshape(-1, x.ndim))
    y = np.empty(ks.shape[0], dtype=np.complex128)
    rc = _load().oracle_dft_points(x.ndim, _shape_arg(x.shape), x.ctypes.data,
                                   ks.shape[0], ks.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                   y.ctypes.data, int(bool(inverse)))
    if rc != 0:
        raise RuntimeError("oracle_dft_points failed")
    return y


def max_abs_rel(y, y_ref) -> float:
    """max |y - y_ref| / max |y_ref| over the whole array, in FP64."""
    y = np.asarray(y, dtype=np.complex128).ravel()
    r = np.asarray(y_ref, dtype=np.complex128).ravel()
    den = float(np.abs(r).max()) if r.size else 0.0
    num = float(np.abs(y - r).max()) if r.size else 0.0
    return num / den if den > 0 else num


def rel_l2(y, y_ref) -> float:
    """||y - y_ref||_2 / ||y_ref||_2 over the whole array, in FP64."""
    y = np.asarray(y, dtype=np.complex128).ravel()
    r = np.asarray(y_ref, dtype=np.complex128).ravel()
    den = np.linalg.norm(r)
    num = np.linalg.norm(y - r)
    return float(num / den) if den > 0 else float(num)


from . import cyclic_model  # noqa: E402,F401
