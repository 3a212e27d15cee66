"""Kernel functions of the oracle, FP64 (test infrastructure only).

Sec. 1 ("Problem statement") defines a kernel as K(x, y) = <phi(x), phi(y)>
for some feature map phi. Sec. 6 gives the Gaussian kernel exp(-||x-y||^2/kappa).
Sec. 1 names the Laplacian kernel as a normalised kernel (gamma = 1) but prints
no formula. The oracle reads it as exp(-||x-y||_2 / sigma). The linear and
degree-p polynomial kernels are the textbook ones. The pins use them because
they have explicit feature maps.

The pairwise values come from ``gram.c``. It is compiled here with gcc on first
use and loaded through ctypes. The values follow the definitions directly:
squared distances are sums of squared coordinate differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

GAUSSIAN, LAPLACIAN, LINEAR, POLY = 0, 1, 2, 3
_NORMALISED = (GAUSSIAN, LAPLACIAN)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gram.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle_gram.so")
_lock = threading.Lock()
_lib = None


@dataclass(frozen=True)
class Kernel:
    """A kernel K(x, y).

    ``param`` is kappa for the Gaussian kernel and sigma for the Laplacian kernel.
    ``coef0`` and ``degree`` apply only to the polynomial kernel.
    """

    kind: int
    param: float = 1.0
    coef0: float = 0.0
    degree: int = 2

    @property
    def normalised(self) -> bool:
        """True for kernels with K(x, x) = 1 for every x (gamma = 1, Sec. 1)."""
        return self.kind in _NORMALISED


def build(force: bool = False) -> str:
    """Compile gram.c into a shared object, with OpenMP when gcc supports it."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_kernel_matrix.argtypes = [dp, ctypes.c_int64, dp, ctypes.c_int64,
                                                 ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_int, dp]
            lib.oracle_kernel_wsum.argtypes = [dp, ctypes.c_int64, dp, ctypes.c_int64, dp,
                                               ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_int, dp]
            lib.oracle_num_threads.restype = ctypes.c_int
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def num_threads() -> int:
    """Threads the C helper uses (OpenMP's maximum, or 1 without OpenMP)."""
    return int(_load().oracle_num_threads())


def set_threads(n: int) -> None:
    """Threads later calls of the C helper use (timing only; results do not depend on it)."""
    _load().oracle_set_threads(int(n))


def _rows(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.ndim == 1:
        a = a[None, :]
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def kernel_matrix(A, B, kern: Kernel) -> np.ndarray:
    """K(a_i, b_j) for every pair of rows, shape (len(A), len(B)), FP64."""
    A, B = _rows(A), _rows(B)
    if A.shape[1] != B.shape[1]:
        raise ValueError("row dimensions differ")
    out = np.empty((A.shape[0], B.shape[0]), dtype=np.float64)
    if out.size == 0:
        return out
    rc = _load().oracle_kernel_matrix(_ptr(A), A.shape[0], _ptr(B), B.shape[0], A.shape[1],
                                      kern.kind, kern.param, kern.coef0, kern.degree,
                                      _ptr(out))
    if rc != 0:
        raise ValueError("bad kernel arguments")
    return out


def kernel_wsum(A, B, w, kern: Kernel) -> np.ndarray:
    """sum_j w_j K(a_i, b_j) for every row a_i, FP64."""
    A, B = _rows(A), _rows(B)
    w = np.ascontiguousarray(w, dtype=np.float64)
    if w.shape != (B.shape[0],):
        raise ValueError("one weight per row of B expected")
    out = np.zeros(A.shape[0], dtype=np.float64)
    if A.shape[0] == 0 or B.shape[0] == 0:
        return out
    rc = _load().oracle_kernel_wsum(_ptr(A), A.shape[0], _ptr(B), B.shape[0], _ptr(w),
                                    A.shape[1], kern.kind, kern.param, kern.coef0,
                                    kern.degree, _ptr(out))
    if rc != 0:
        raise ValueError("bad kernel arguments")
    return out


def kernel_diag(A, kern: Kernel) -> np.ndarray:
    """K(a, a) for every row. Equals 1 exactly for the normalised kernels."""
    A = _rows(A)
    if kern.normalised:
        return np.ones(A.shape[0], dtype=np.float64)
    return np.array([kernel_matrix(a, a, kern)[0, 0] for a in A], dtype=np.float64)
