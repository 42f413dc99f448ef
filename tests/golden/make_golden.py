"""Writes the golden fixtures in this folder.  Calls only the oracle (and the
seeded input generator that produces the matrices, which it stores verbatim so
that every machine reads the same complex128 entries).

Up to n = 22 the full sum is the brute force of Eq. (tor); beyond that it is
the oracle's binary128 Algorithm 2 (Sec. 2), split into 2^10 tasks over the
host cores (the brute force would take hours to days), with prefix units from
the brute force stored beside it.

Usage: python tests/golden/make_golden.py [fixture names]  (default: all)
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2109_04528_gb300 import inputs  # noqa: E402


def write(name, inst, note, units=(), method="brute"):
    if method == "brute":
        r = oracle.tor_brute(inst.O)
        cite = "Eq. (tor), Sec. 1 (definition); values from the binary128 brute-force oracle"
    else:
        r = oracle.tor_recursive(inst.O, split=10, threads=None)
        cite = ("Eq. (tor), Sec. 1; full sum from the oracle's binary128 Algorithm 2 (Sec. 2) split into "
                "2^10 tasks, prefix units from the binary128 brute force")
    rec = {
        "citation": cite,
        "method": "brute force" if method == "brute" else "Algorithm 2, binary128, split 10",
        "note": note,
        "n": inst.n, "layout": "block", "kind": inst.kind, "seed": inst.seed,
        "O_re": np.real(inst.O).tolist(), "O_im": np.imag(inst.O).tolist(),
        "tor_hi": r.hi, "tor_lo": r.lo, "abs_sum": r.abs_sum,
    }
    if units:
        # prefix units (bit j of u = mode j in Z, j < p): each sums the terms whose first p decisions are u
        p = units[0]
        rec["unit_p"] = p
        rec["units"] = []
        for u in units[1]:
            q = oracle.tor_unit(inst.O, p, u)
            rec["units"].append({"u": u, "hi": q.hi, "lo": q.lo, "abs_sum": q.abs_sum})
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(rec, f, indent=0)
        f.write("\n")


FIXTURES = {
    "lossy_n8.json": (inputs.config_n8, "n=8 squeezed vacua r~U[0.3,0.8], Haar U, eta=0.5 (256 subsets)", ()),
    "lossy_n4_hi.json": (lambda: inputs.lossy_squeezed(4, 99, (1.0, 1.5), 0.7),
                         "n=4, higher squeezing r~U[1.0,1.5], eta=0.7", ()),
    "lossy_n20.json": (lambda: inputs.config_single(20),
                       "n=20 lossy squeezed state of the benchmark's kind (r~U[0.3,0.8], eta_j~U[0.3,0.7]); "
                       "full brute force over 2^20 subsets", (8, [0, 37, 255])),
    "lossy_n22.json": (lambda: inputs.config_single(22),
                       "n=22 lossy squeezed state of the benchmark's kind (r~U[0.3,0.8], eta_j~U[0.3,0.7]); "
                       "full brute force over 2^22 subsets", (8, [0, 37, 255])),
    "lossy_n24.json": (lambda: inputs.config_single(24),
                       "n=24 lossy squeezed state of the single-matrix benchmark (r~U[0.3,0.8], eta_j~U[0.3,0.7]); "
                       "full sum by Algorithm 2 in binary128", (12, [0, 1365, 4095]), "alg2"),
    "lossy_n30.json": (lambda: inputs.config_single(30),
                       "n=30 lossy squeezed state of the large single-matrix benchmark (r~U[0.3,0.8], "
                       "eta_j~U[0.3,0.7]); full sum by Algorithm 2 in binary128", (18, [0, 87381, 262143]), "alg2"),
}


if __name__ == "__main__":
    # python tests/golden/make_golden.py [NAME ...]   (default: every fixture)
    for name in sys.argv[1:] or FIXTURES:
        make, note, units, *method = FIXTURES[name]
        write(name, make(), note, units, *method)
