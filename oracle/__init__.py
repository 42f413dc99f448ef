"""CPU oracle for the Torontonian -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  The library's product path never loads
it, and it shares no code with the CUDA path.
"""
from .oracle import (OracleResult, build, tor_brute, tor_unit, tor_recursive, det_quad,
                     quad_bits, library_path)

__all__ = ["OracleResult", "build", "tor_brute", "tor_unit", "tor_recursive", "det_quad",
           "quad_bits", "library_path"]
