"""The FLO-count experiment of Sec. 3 (Eq. linear_fit), on CPU.

The combinatorial counts in paper_2109_04528_gb300.flops are checked against
explicit enumeration, and against an instrumented implementation of
Algorithms 1 and 2 that counts every operation as it executes it and computes
Tor, which is compared with the binary128 oracle.
"""
import itertools
import math

import numpy as np

from paper_2109_04528_gb300 import flops, inputs


class Counter:
    def __init__(self):
        self.f = 0


def chol_counted(A, c, L=None, start=0):
    """Algorithm 1 (rows start.. of a Hermitian A), counting operations."""
    m = A.shape[0]
    L = np.zeros((m, m), dtype=complex) if L is None else L
    for i in range(start, m):
        for j in range(start, i):
            s = A[i, j]
            for k in range(j):
                s -= L[i, k] * np.conj(L[j, k])
                c.f += 8
            L[i, j] = s / L[j, j].real
            c.f += 2
        d = A[i, i].real
        for k in range(i):
            d -= abs(L[i, k]) ** 2
            c.f += 4
        c.f += 1
        L[i, i] = math.sqrt(d)
        c.f += 1
    return L


def det_term_counted(L, c):
    det = 1.0
    for i in range(L.shape[0]):
        det *= L[i, i].real ** 2
        c.f += 1
    c.f += 3  # 1/sqrt, sign, accumulation
    return 1.0 / math.sqrt(det)


def algorithm2_counted(O):
    """The paper's Algorithm 2 in pairs order, instrumented."""
    n = O.shape[0] // 2
    perm = [j + cc * n for j in range(n) for cc in (0, 1)]
    A = np.eye(2 * n) - O[np.ix_(perm, perm)]
    c = Counter()
    L = chol_counted(A, c)
    tor = det_term_counted(L, c)

    def rec(kept, L, removed, start):
        nonlocal tor
        for i in range(start, n):
            q = kept.index(i)
            kept2 = [k for k in kept if k != i]
            rows = [2 * k + cc for k in kept2 for cc in (0, 1)]
            M = A[np.ix_(rows, rows)]
            m2 = len(rows)
            L2 = np.zeros((m2, m2), dtype=complex)
            r0 = 2 * q
            for a in range(m2):
                for b in range(min(r0, a + 1)):
                    L2[a, b] = L[a if a < r0 else a + 2, b]
            L2 = chol_counted(M, c, L2, r0)
            t = det_term_counted(L2, c)
            tor += (-1) ** (removed + 1) * t
            rec(kept2, L2, removed + 1, i + 1)

    rec(list(range(n)), L, 0, 0)
    return tor, c.f


def test_standard_count_is_the_sum_over_subsets():
    for n in range(0, 9):
        direct = sum(flops.cholesky_flops(2 * len(Z)) + flops.det_term_flops(2 * len(Z))
                     for k in range(n + 1) for Z in itertools.combinations(range(n), k))
        assert flops.standard_flops(n) == direct


def test_algorithm2_count_matches_instrumented_run(oracle_mod):
    for n in (1, 2, 3, 4, 5):
        inst = inputs.lossy_squeezed(n, 80 + n, (0.3, 0.8), 0.5)
        tor, counted = algorithm2_counted(inst.O)
        assert counted == flops.algorithm2_flops(n), n
        ref = oracle_mod.tor_brute(inst.O)
        assert abs(tor - ref.tor) <= 1e-12 * ref.abs_sum


def test_rank2_count_is_the_sum_over_nodes():
    for n in range(1, 12):
        # 2^j internal nodes at depth j include mode j into m = n-1-j trailing modes
        direct = sum(2 ** j * (32 * (n - 1 - j) ** 2 + 40 * (n - 1 - j) + 10) for j in range(n)) + 10 * 2 ** n
        assert flops.rank2_flops(n) == direct
    assert abs(flops.rank2_flops(30) / 2 ** 30 - 156.0) < 1e-3


def test_omega_fit_reproduces_the_paper_qualitatively():
    out = flops.experiment(26, 60)
    # paper (Sec. 3): omega_std = 2.7355, omega_rec = 1.0695; 18x fewer FLOs at N = 50, 57x at N = 100
    assert 2.6 < out["standard"] < 3.0
    assert 1.0 < out["algorithm2"] < 1.25
    assert abs(out["rank2"]) < 0.05  # O(1) flops per subset, amortised
    assert 15 < out["ratio_std_alg2_N50"] < 25
    assert 45 < out["ratio_std_alg2_N100"] < 90
