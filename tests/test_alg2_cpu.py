"""The FP64 multithreaded Algorithm 2 (oracle/tor_alg2_cpu.c), the CPU baseline
of the paper's own method (Sec. 2, Algorithm 2), checked on the CPU against
the binary128 oracle and against what its task split fixes.
"""
import numpy as np
import pytest

from paper_2109_04528_gb300 import inputs

alg2_cpu = pytest.importorskip("oracle.alg2_cpu")


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 9, 12])
def test_reaches_the_oracle(oracle_mod, n):
    # FP64 Cholesky factors along the remove-mode recursion: every term to a few
    # ulps, the sum within 1e-12 of sum|term| (the GPU's FP64 bar is 1e-10)
    inst = inputs.lossy_squeezed(n, 900 + n, (0.3, 0.8), (0.3, 0.7))
    r = alg2_cpu.tor_alg2(inst.O, threads=3)
    o = oracle_mod.tor_brute(inst.O)
    assert r.terms == 2 ** n
    assert abs(r.tor - o.tor) <= 1e-12 * o.abs_sum
    assert abs(r.abs_sum - o.abs_sum) <= 1e-12 * o.abs_sum


def test_general_hermitian_and_pairs_layout(oracle_mod):
    inst = inputs.random_hermitian_contraction(8, 17, 0.85)
    o = oracle_mod.tor_brute(inst.O)
    r = alg2_cpu.tor_alg2(inst.O, threads=2)
    assert abs(r.tor - o.tor) <= 1e-12 * o.abs_sum
    # the same matrix in pairs order (mode j owns rows 2j, 2j+1)
    n = 8
    perm = [j + c * n for j in range(n) for c in (0, 1)]
    Op = inst.O[np.ix_(perm, perm)]
    rp = alg2_cpu.tor_alg2(Op, threads=2, layout=1)
    assert (rp.tor, rp.abs_sum) == (r.tor, r.abs_sum)


def test_product_state_closed_form(oracle_mod):
    # Tor of a product state is the product of the one-mode Torontonians (Eq. tor factorises)
    n = 10
    inst = inputs.product_state(n, 31)
    want, absum = 1.0, 1.0
    for j in range(n):
        f = oracle_mod.tor_brute(inputs.submatrix(inst.O, [j]))
        want *= f.tor
        absum *= f.abs_sum
    r = alg2_cpu.tor_alg2(inst.O, threads=4)
    assert abs(r.tor - want) <= 1e-12 * absum


def test_thread_count_does_not_change_the_result():
    inst = inputs.config_single(13)
    a = alg2_cpu.tor_alg2(inst.O, threads=1)
    b = alg2_cpu.tor_alg2(inst.O, threads=7)
    assert (a.tor, a.abs_sum, a.terms) == (b.tor, b.abs_sum, b.terms)


def _split(n, threads):
    # the baseline's task split, restated: a node whose largest removed mode is r
    # heads 2^(n-1-r) nodes; nodes above 2^n / (32 threads) are split, the rest are
    # tasks, largest subtree first
    T = max(1.0, 2.0 ** n / (32 * threads))
    top, tasks = [], []

    def gen(R):
        size = 2.0 ** n if not R else 2.0 ** (n - 1 - R[-1])
        if R and size <= T:
            tasks.append(tuple(R))
            return
        top.append(tuple(R))
        for i in range(R[-1] + 1 if R else 0, n):
            gen(R + [i])

    gen([])
    tasks.sort(key=lambda R: R[-1])
    return top, tasks


@pytest.mark.parametrize("n,threads", [(11, 2), (14, 16)])
def test_sample_counts_its_terms(n, threads):
    # max_tasks = 0: only the split nodes; each task adds the nodes of its subtree
    inst = inputs.config_single(n)
    top, tasks = _split(n, threads)
    assert len(top) + sum(2 ** (n - 1 - R[-1]) for R in tasks) == 2 ** n
    assert max(2 ** (n - 1 - R[-1]) for R in tasks) <= max(1, 2 ** n // (32 * threads))  # balanced
    assert alg2_cpu.tor_alg2(inst.O, threads=threads, max_tasks=0).terms == len(top)
    first = len(top) + 2 ** (n - 1 - tasks[0][-1])
    assert alg2_cpu.tor_alg2(inst.O, threads=threads, max_tasks=1).terms == first
    assert alg2_cpu.tor_alg2(inst.O, threads=threads, max_tasks=10 ** 9).terms == 2 ** n


def test_not_positive_definite():
    with pytest.raises(ValueError):
        alg2_cpu.tor_alg2(2 * np.eye(6, dtype=np.complex128), threads=2)
