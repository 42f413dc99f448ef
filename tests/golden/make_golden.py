"""Writes the golden fixtures in this folder.  Calls only the oracle (and the
seeded input generator that produces the matrices, which it stores verbatim so
that every machine reads the same complex128 entries).

Usage: python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2109_04528_gb300 import inputs  # noqa: E402


def write(name, inst, note):
    r = oracle.tor_brute(inst.O)
    rec = {
        "citation": "Eq. (tor), Sec. 1 (definition); values from the binary128 brute-force oracle",
        "note": note,
        "n": inst.n, "layout": "block", "kind": inst.kind, "seed": inst.seed,
        "O_re": np.real(inst.O).tolist(), "O_im": np.imag(inst.O).tolist(),
        "tor_hi": r.hi, "tor_lo": r.lo, "abs_sum": r.abs_sum,
    }
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(rec, f, indent=0)
        f.write("\n")


if __name__ == "__main__":
    write("lossy_n8.json", inputs.config_n8(),
          "n=8 squeezed vacua r~U[0.3,0.8], Haar U, eta=0.5 (256 subsets)")
    write("lossy_n4_hi.json", inputs.lossy_squeezed(4, 99, (1.0, 1.5), 0.7),
          "n=4, higher squeezing r~U[1.0,1.5], eta=0.7")
