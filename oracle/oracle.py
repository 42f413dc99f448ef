"""ctypes front end of the binary128 CPU oracle (tor_oracle.c) -- TEST INFRASTRUCTURE ONLY.

Eq. (tor) of the paper (Sec. 1):
    Tor(O) = sum_{Z subset [n]} (-1)^{n-|Z|} / sqrt(|det(I - O_Z)|)

``tor_brute`` is that definition written out (one LU determinant per subset,
mask-order Neumaier sum, all in binary128).  ``tor_recursive`` is the paper's
Algorithm 2 (Sec. 2) in binary128.  Neither shares code with the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tor_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = None


def library_path() -> str:
    return os.path.join(_BUILD, f"libtororacle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile tor_oracle.c with gcc (plain C, pthreads; libquadmath on x86_64)."""
    out = library_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-o", out + ".tmp", _SRC]
    if platform.machine() in ("x86_64", "AMD64"):
        cmd.append("-lquadmath")
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.tor_oracle_brute.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                         ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, dp]
        lib.tor_oracle_recursive.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp]
        lib.tor_oracle_recursive_split.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_int, dp]
        lib.tor_oracle_det.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, dp]
        lib.tor_oracle_quad_bits.argtypes = []
        _LIB = lib
    return _LIB


@dataclass
class OracleResult:
    hi: float          # Tor as double-double: hi + lo
    lo: float
    abs_sum: float     # sum over the summed subsets of |term|
    im_ratio: float    # max |Im det| / |det| over those subsets
    count: int

    @property
    def tor(self) -> float:
        return self.hi + self.lo


def _as_input(O: np.ndarray):
    O = np.ascontiguousarray(np.asarray(O, dtype=np.complex128))
    m = O.shape[0]
    if O.ndim != 2 or O.shape[1] != m or m % 2:
        raise ValueError("O must be a square 2n x 2n complex matrix")
    return O, m // 2


def _threads(threads):
    return int(threads) if threads else max(1, os.cpu_count() or 1)


def tor_brute(O: np.ndarray, layout: int = 0, threads: int | None = None, base: int = 0,
              stride: int = 1, count: int | None = None, mutate: int = 0) -> OracleResult:
    """Brute-force Eq. (tor) over the masks base + k*stride, k < count (default: all 2^n)."""
    O, n = _as_input(O)
    if count is None:
        count = 1 << n
    out = (ctypes.c_double * 5)()
    ptr = O.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if n else None
    rc = _lib().tor_oracle_brute(n, ptr, max(2 * n, 1), layout, base, stride, count,
                                 _threads(threads), mutate, out)
    if rc:
        raise ValueError(f"tor_oracle_brute failed ({rc})")
    return OracleResult(out[0], out[1], out[2], out[3], int(out[4]))


def tor_unit(O: np.ndarray, p: int, u: int, layout: int = 0, threads: int | None = None) -> OracleResult:
    """Sum of the terms whose decisions on modes 0..p-1 are the bits of u
    (mask & (2^p - 1) == u): one prefix unit of the subset tree."""
    O, n = _as_input(O)
    return tor_brute(O, layout, threads, base=u, stride=1 << p, count=1 << (n - p))


def tor_recursive(O: np.ndarray, layout: int = 0, split: int = 0, threads: int | None = 1) -> OracleResult:
    """The paper's Algorithm 2 (remove-mode recursion reusing L11/L21) in binary128.

    split = d > 0 cuts the recursion into the 2^d tasks given by the removals
    among modes 0..d-1 (the paper spreads the first loop of Algorithm 2 over
    workers, Sec. 4); each task sums its addends, and the task sums are added in
    task order, so the value depends on d but not on the thread count."""
    O, n = _as_input(O)
    out = (ctypes.c_double * 3)()
    ptr = O.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if n else None
    split = max(0, min(int(split), n))
    rc = _lib().tor_oracle_recursive_split(n, ptr, max(2 * n, 1), layout, split, _threads(threads), out)
    if rc == -2:
        raise ValueError("I - O is not positive definite")
    if rc:
        raise ValueError(f"tor_oracle_recursive failed ({rc})")
    return OracleResult(out[0], out[1], out[2], 0.0, 1 << n)


def det_quad(O: np.ndarray, mask: int, layout: int = 0) -> complex:
    """det(I - O_Z) for one mask, LU in binary128, rounded to complex128."""
    O, n = _as_input(O)
    out = (ctypes.c_double * 2)()
    ptr = O.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if n else None
    _lib().tor_oracle_det(n, ptr, max(2 * n, 1), layout, mask, out)
    return complex(out[0], out[1])


def quad_bits() -> int:
    return int(_lib().tor_oracle_quad_bits())
