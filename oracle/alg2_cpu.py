"""ctypes front end of the FP64 multithreaded Algorithm 2 (tor_alg2_cpu.c) --
CPU BASELINE; TEST AND BENCHMARK INFRASTRUCTURE ONLY.

The paper's recursive Torontonian (Sec. 2, Algorithm 2) in FP64 complex
arithmetic on all host cores: the CPU implementation of the method itself,
timed beside the GPU path.  It is not the oracle (``oracle.tor_brute`` in
binary128 is) and shares no code with the CUDA path or the oracle.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tor_alg2_cpu.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = None


def library_path() -> str:
    return os.path.join(_BUILD, f"libtoralg2_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile tor_alg2_cpu.c with gcc (plain C, pthreads)."""
    out = library_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-o", out + ".tmp", _SRC, "-lm"], check=True)
    os.replace(out + ".tmp", out)
    return out


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.tor_alg2_fp64.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_longlong, dp]
        lib.tor_alg2_fp64.restype = ctypes.c_int
        _LIB = lib
    return _LIB


@dataclass
class Alg2Result:
    tor: float       # the (partial) sum of the evaluated terms
    abs_sum: float   # their sum of |term|
    terms: int       # number of terms evaluated (2^n for the full sum)


def tor_alg2(O: np.ndarray, threads: int | None = None, max_tasks: int = -1, layout: int = 0) -> Alg2Result:
    """Algorithm 2 in FP64 on `threads` host threads (default: all cores).
    max_tasks >= 0 evaluates only the nodes above the task level and the first
    max_tasks tasks (largest subtrees first): a bounded sample for timing."""
    a = np.ascontiguousarray(O, dtype=np.complex128)
    n = a.shape[0] // 2
    out = (ctypes.c_double * 3)()
    thr = int(threads) if threads else (os.cpu_count() or 1)
    rc = _lib().tor_alg2_fp64(n, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), a.shape[1], layout, thr,
                              int(max_tasks), out)
    if rc == -2:
        raise ValueError("I - O is not positive definite")
    if rc != 0:
        raise RuntimeError(f"tor_alg2_fp64 failed ({rc})")
    return Alg2Result(out[0], out[1], int(out[2]))
