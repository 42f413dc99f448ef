"""Pins for the CPU oracle (-m "not gpu").

The oracle is pinned to facts that do not come from its own code:
closed forms of Eq. (tor) (paper Sec. 1) for states whose click statistics
are known, identities of the definition, and numpy's independent LU
determinant.  The last test plants mistakes in the oracle and checks that
the pins catch every one of them.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2109_04528_gb300 import inputs

RNG = np.random.default_rng(12345)


def closed_product(inst):
    """Product state: Tor = prod_j (x_j - 1), sum|term| = prod_j (x_j + 1),
    x_j = sqrt(det Sigma_j) for the single lossy squeezed mode j
    (N = eta sinh^2 r, M = eta sinh r cosh r)."""
    sh, ch = np.sinh(inst.r), np.cosh(inst.r)
    N = inst.eta * sh * sh
    M = inst.eta * sh * ch
    x = np.sqrt((1 + N) ** 2 - M ** 2)
    return float(np.prod(x - 1)), float(np.prod(x + 1))


def check_pins(oracle, mutate=0):
    """Run the pin checks against one oracle variant; return the names that failed."""
    failed = []
    tb = lambda O, layout=0: oracle.tor_brute(O, layout=layout, threads=2, mutate=mutate)

    # n = 1 closed form with numpy's determinant
    for seed in range(3):
        inst = inputs.random_hermitian_contraction(1, 100 + seed)
        want = 1 / math.sqrt(np.linalg.det(np.eye(2) - inst.O).real) - 1
        got = tb(inst.O).tor
        if abs(got - want) > 1e-13 * (abs(want) + 2):
            failed.append("n1"); break
    # single-mode squeezed vacuum: cosh r - 1
    for r in (0.3, 1.1):
        inst = inputs.lossy_squeezed(1, 7, (r, r), 1.0)
        if abs(tb(inst.O).tor - (math.cosh(r) - 1)) > 1e-13:
            failed.append("squeezed1"); break
    # product states (odd and even n, both layouts)
    for n, layout in ((5, 0), (6, 1), (7, 0)):
        inst = inputs.product_state(n, 40 + n)
        O = inst.O if layout == 0 else inputs.to_pairs(inst.O)
        tor, absum = closed_product(inst)
        res = tb(O, layout)
        if abs(res.tor - tor) > 1e-12 * absum or abs(res.abs_sum - absum) > 1e-12 * absum:
            failed.append(f"product{n}"); break
    # vacuum: terms are +-1, Tor = 0 exactly
    res = tb(inputs.vacuum(5).O)
    if res.tor != 0.0 or res.abs_sum != 32.0:
        failed.append("vacuum")
    # two-mode squeezed vacuum: Tor = sinh^2 r, single-mode patterns give 0
    inst = inputs.two_mode_squeezed_vacuum(0.7)
    if abs(tb(inst.O).tor - math.sinh(0.7) ** 2) > 1e-13:
        failed.append("tmsv")
    for j in range(2):
        if abs(tb(inputs.submatrix(inst.O, [j])).tor) > 1e-13:
            failed.append("tmsv_single"); break
    # normalisation: sum_S Tor(O_S) = sqrt(det Sigma) (numpy det of Sigma)
    inst = inputs.lossy_squeezed(5, 77, (0.4, 0.9), 0.6)
    total = 0.0
    for k in range(6):
        for S in itertools.combinations(range(5), k):
            t = tb(inputs.submatrix(inst.O, S)).tor if S else tb(np.zeros((0, 0))).tor
            total += t
    want = math.sqrt(np.linalg.det(inst.sigma).real)
    if abs(total - want) > 1e-11 * want:
        failed.append("normalisation")
    return failed


def test_quad_is_binary128(oracle_mod):
    assert oracle_mod.quad_bits() == 113


def test_empty_matrix_is_one(oracle_mod):
    r = oracle_mod.tor_brute(np.zeros((0, 0)))
    assert r.tor == 1.0 and r.abs_sum == 1.0


def test_all_pins_pass(oracle_mod):
    assert check_pins(oracle_mod) == []


@pytest.mark.parametrize("mutate", [1, 2, 3, 4, 5])
def test_planted_mistakes_are_caught(oracle_mod, mutate):
    # 1 sign (-1)^{|Z|}; 2 wrong row pairing; 3 empty-set term dropped;
    # 4 identity dropped (det(-O_Z)); 5 off-diagonal block transposed.
    assert check_pins(oracle_mod, mutate) != []


def test_det_matches_numpy(oracle_mod):
    inst = inputs.lossy_squeezed(6, 5, (0.3, 1.0), 0.5)
    for mask in (1, 5, 22, 63, 40):
        S = [j for j in range(6) if mask >> j & 1]
        want = np.linalg.det(np.eye(2 * len(S)) - inputs.submatrix(inst.O, S))
        got = oracle_mod.det_quad(inst.O, mask)
        assert abs(got - want) <= 1e-13 * abs(want)
        assert abs(got.imag) <= 1e-13 * abs(got)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 9, 10, 11, 12])
def test_brute_equals_algorithm2(oracle_mod, n):
    # the paper's Algorithm 2 (plain recursion, and split into 2^d tasks as in Sec. 4)
    # against the definition written out, on physical and on general Hermitian inputs
    for inst in (inputs.lossy_squeezed(n, 300 + n, (0.3, 0.8), 0.5),
                 inputs.random_hermitian_contraction(n, 400 + n, 0.8)):
        a = oracle_mod.tor_brute(inst.O)
        for split in (0, min(n, 3), n):
            b = oracle_mod.tor_recursive(inst.O, split=split, threads=4)
            assert abs((a.hi - b.hi) + (a.lo - b.lo)) <= 1e-28 * a.abs_sum, split
            assert abs(a.abs_sum - b.abs_sum) <= 1e-14 * a.abs_sum


def test_algorithm2_split_is_independent_of_threads(oracle_mod):
    inst = inputs.lossy_squeezed(11, 17, (0.3, 0.8), (0.3, 0.7))
    got = {(r.hi, r.lo, r.abs_sum) for r in (oracle_mod.tor_recursive(inst.O, split=6, threads=t)
                                             for t in (1, 3, 8))}
    assert len(got) == 1


def test_algorithm2_reproduces_the_n20_brute_force(oracle_mod):
    # the stored n = 20 fixture is the full brute force; the split Algorithm 2 (the
    # method the n >= 24 fixtures use) must reach it to binary128 rounding
    g, O = load_golden("lossy_n20.json")
    r = oracle_mod.tor_recursive(O, split=8, threads=None)
    assert abs((r.hi - g["tor_hi"]) + (r.lo - g["tor_lo"])) <= 1e-30 * g["abs_sum"]
    assert abs(r.abs_sum - g["abs_sum"]) <= 1e-14 * g["abs_sum"]


def test_algorithm2_rejects_non_pd(oracle_mod):
    O = 2.0 * np.eye(6, dtype=np.complex128)  # I - O = -I
    with pytest.raises(ValueError):
        oracle_mod.tor_recursive(O, split=2, threads=2)


def test_invariances(oracle_mod):
    inst = inputs.lossy_squeezed(6, 9, (0.3, 0.8), 0.5)
    base = oracle_mod.tor_brute(inst.O)
    perm = RNG.permutation(6)
    theta = RNG.uniform(0, 2 * np.pi, 6)
    for O, layout in ((inputs.permute_modes(inst.O, perm), 0),
                      (inputs.to_pairs(inst.O), 1),
                      (inputs.local_phase(inst.O, theta), 0)):
        r = oracle_mod.tor_brute(O, layout=layout)
        assert abs(r.tor - base.tor) <= 1e-14 * base.abs_sum


def test_physical_patterns_non_negative(oracle_mod):
    inst = inputs.lossy_squeezed(6, 21, (0.5, 1.2), 0.4)
    for S in itertools.combinations(range(6), 3):
        r = oracle_mod.tor_brute(inputs.submatrix(inst.O, S))
        assert r.tor >= -1e-14 * r.abs_sum


def test_units_partition_the_sum(oracle_mod):
    inst = inputs.lossy_squeezed(7, 31, (0.3, 0.8), 0.5)
    full = oracle_mod.tor_brute(inst.O)
    p = 3
    parts = [oracle_mod.tor_unit(inst.O, p, u) for u in range(1 << p)]
    assert sum(x.count for x in parts) == 128
    s = sum(x.hi for x in parts) + sum(x.lo for x in parts)
    assert abs(s - full.tor) <= 1e-20 * full.abs_sum
    assert abs(sum(x.abs_sum for x in parts) - full.abs_sum) <= 1e-13 * full.abs_sum


def load_golden(name):
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        g = json.load(f)
    O = np.array(g["O_re"]) + 1j * np.array(g["O_im"])
    return g, O


@pytest.mark.parametrize("name", ["lossy_n8.json", "lossy_n4_hi.json"])
def test_golden_fixture_reproduces(oracle_mod, name):
    g, O = load_golden(name)
    r = oracle_mod.tor_brute(O)
    assert r.hi == g["tor_hi"] and abs(r.lo - g["tor_lo"]) <= 1e-30 * g["abs_sum"]


@pytest.mark.parametrize("name", ["lossy_n20.json", "lossy_n22.json", "lossy_n24.json", "lossy_n30.json"])
def test_large_golden_units_reproduce(oracle_mod, name):
    # the full sums over 2^20 .. 2^24 subsets take minutes; the stored prefix units
    # (2^12 .. 2^14 subsets each, brute force) are recomputed here
    g, O = load_golden(name)
    assert O.shape == (2 * g["n"], 2 * g["n"]) and g["abs_sum"] > 0
    for unit in g["units"]:
        r = oracle_mod.tor_unit(O, g["unit_p"], unit["u"])
        assert r.hi == unit["hi"] and abs(r.lo - unit["lo"]) <= 1e-30 * unit["abs_sum"]
        assert abs(r.abs_sum - unit["abs_sum"]) <= 1e-15 * unit["abs_sum"]
        assert unit["abs_sum"] < g["abs_sum"]
