"""CPU model of the FP64 subset-tree walk, counting its FP64 instructions.

A plain-Python restatement of the GPU's FP64 arithmetic: the include step of
the subset tree (Sec. 2, Fig. 2, in the add-a-mode direction: the 2x2 pivot,
its reciprocal and reciprocal square root -- hardware estimate plus one cubic
series step -- the pivot columns and the rank-2 update), the leaf pairs and the
signed sums of Eq. (tor), with the lane's double-double accumulator.  Python
floats are IEEE doubles rounded to nearest; an FMA is rounded once, through
exact rationals.  Every FP64-pipe instruction is counted (add, mul and FMA one
each; the reciprocal estimates are not FP64-pipe instructions).  Checks:
  * the count equals paper_2109_04528_gb300.flops.path_ops for the real (x, p)
    and the complex walk -- the figure the benchmark's instruction fraction
    divides by;
  * the model's Tor reaches the binary128 oracle within the FP64 tolerance,
    1e-10 sum|term|, as the GPU tests require.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2109_04528_gb300 import flops, inputs


class Ops:
    def __init__(self):
        self.n = 0

    def add(self, a, b):
        self.n += 1
        return a + b

    def mul(self, a, b):
        self.n += 1
        return a * b

    def fma(self, a, b, c):
        self.n += 1
        return float(Fraction(a) * Fraction(b) + Fraction(c))

    def rcp(self, x):
        y = float(np.float32(1.0 / x))  # a coarse estimate (the hardware's is ~2^-20; not an FP64-pipe op)
        e = self.fma(-x, y, 1.0)
        s = self.fma(e, e, e)
        return self.fma(y, s, y)

    def rsqrt(self, x):
        y = float(np.float32(1.0 / math.sqrt(x)))
        t = self.mul(x, y)
        e = self.fma(-t, y, 1.0)
        p = self.fma(0.375, e, 0.5)
        q = self.mul(y, e)
        return self.fma(q, p, y)

    def two_sum(self, a, b):
        s = self.add(a, b)
        bb = self.add(s, -a)
        return s, self.add(self.add(a, -self.add(s, -bb)), self.add(b, -bb))


class RealArith:
    def __init__(self, o):
        self.o = o

    def re(self, v):
        return v

    def diag(self, d):
        return d

    def det2(self, a, b, e):
        return self.o.fma(a, e, -self.o.mul(b, b))

    def cl(self, b, ia):
        return self.o.mul(b, ia)

    def reduce_col(self, x, y, c):
        return self.o.fma(-x, c, y)

    def scale(self, v, s):
        return self.o.mul(v, s)

    def rank2(self, s, xt, xk, yt, yk):
        return self.o.fma(-yt, yk, self.o.fma(-xt, xk, s))

    rank2_diag = rank2


class CplxArith:
    def __init__(self, o):
        self.o = o

    def re(self, v):
        return v[0]

    def diag(self, d):
        return (d, 0.0)

    def det2(self, a, b, e):
        abs2 = self.o.fma(b[0], b[0], self.o.mul(b[1], b[1]))
        return self.o.fma(a, e, -abs2)

    def cl(self, b, ia):
        return (self.o.mul(b[0], ia), -self.o.mul(b[1], ia))

    def reduce_col(self, x, y, c):  # y - x c
        f = self.o.fma
        return (f(x[1], c[1], f(-x[0], c[0], y[0])), f(-x[1], c[0], f(-x[0], c[1], y[1])))

    def scale(self, v, s):
        return (self.o.mul(v[0], s), self.o.mul(v[1], s))

    def rank2(self, s, xt, xk, yt, yk):  # s - xt conj(xk) - yt conj(yk)
        f = self.o.fma
        r = f(-yt[1], yk[1], f(-yt[0], yk[0], f(-xt[1], xk[1], f(-xt[0], xk[0], s[0]))))
        i = f(yt[0], yk[1], f(-yt[1], yk[0], f(xt[0], xk[1], f(-xt[1], xk[0], s[1]))))
        return (r, i)

    def rank2_diag(self, d, xt, x, yt, y):
        f = self.o.fma
        return f(-yt[1], y[1], f(-yt[0], y[0], f(-xt[1], x[1], f(-xt[0], x[0], d))))


def include(A, S, o):
    R = max(i for i, _ in S) + 1
    a, b, e = A.re(S[(0, 0)]), S[(1, 0)], A.re(S[(1, 1)])
    det2 = A.det2(a, b, e)
    assert a > 0 and det2 > 0
    rho = o.rsqrt(det2)
    ia = o.rcp(a)
    cl = A.cl(b, ia)
    id2 = o.mul(a, o.mul(rho, rho))
    x = [S[(r + 2, 0)] for r in range(R - 2)]
    yp = [A.reduce_col(x[r], S[(r + 2, 1)], cl) for r in range(R - 2)]
    C = {}
    for i in range(R - 2):
        xt, yt = A.scale(x[i], ia), A.scale(yp[i], id2)
        for k in range(i):
            C[(i, k)] = A.rank2(S[(i + 2, k + 2)], xt, x[k], yt, yp[k])
        C[(i, i)] = A.diag(A.rank2_diag(A.re(S[(i + 2, i + 2)]), xt, x[i], yt, yp[i]))
    return C, rho


def trail(S):
    return {(i - 2, k - 2): v for (i, k), v in S.items() if i >= 2 and k >= 2}


def subtree(A, S, m, phi, o):
    """(signed sum, sum of magnitudes) below a register-resident node of m modes."""
    if m == 1:
        det2 = A.det2(A.re(S[(0, 0)]), S[(1, 0)], A.re(S[(1, 1)]))
        r = o.rsqrt(det2)
        return o.fma(phi, r, -phi), o.fma(phi, r, phi)  # the pair's signed and magnitude sums
    v1, a1 = subtree(A, trail(S), m - 1, phi, o)
    C, rho = include(A, S, o)
    v2, a2 = subtree(A, C, m - 1, o.mul(phi, rho), o)
    return o.add(v2, -v1), o.add(a1, a2)


def walk(A, S, m, phi, excl, acc, o, regs):
    if m <= regs:
        v, a = subtree(A, S, m, phi, o)
        v = -v if excl % 2 else v  # a sign, no arithmetic
        acc[0], e = o.two_sum(acc[0], v)  # double-double accumulator (Sum2)
        acc[1] = o.add(acc[1], e)
        acc[2] = o.add(acc[2], a)
        return
    walk(A, trail(S), m - 1, phi, excl + 1, acc, o, regs)
    C, rho = include(A, S, o)
    walk(A, C, m - 1, o.mul(phi, rho), excl, acc, o, regs)


def b_entries(O, real):
    """B = I - O in pairs order, or its real form V = U^H B U (one rounding each)."""
    n = O.shape[0] // 2
    idx = [j + c * n for j in range(n) for c in (0, 1)]
    S = {}
    for r in range(2 * n):
        for s in range(r + 1):
            if not real:
                v = O[idx[r], idx[s]]
                S[(r, s)] = (1.0 - v.real, 0.0) if r == s else (-v.real, -v.imag)
            else:
                j, k = r // 2, s // 2
                Are, Aim = (1.0 if j == k else 0.0) - O[j, k].real, -O[j, k].imag
                Cre, Cim = -O[j, k + n].real, -O[j, k + n].imag
                if r % 2 == 0:
                    S[(r, s)] = Are + Cre if s % 2 == 0 else Cim - Aim
                else:
                    S[(r, s)] = Aim + Cim if s % 2 == 0 else Are - Cre
    return S


def model_tor(O, real):
    o = Ops()
    A = RealArith(o) if real else CplxArith(o)
    acc = [0.0, 0.0, 0.0]
    # subtrees of 4 modes stay in registers on the real path, 3 on the complex one
    walk(A, b_entries(O, real), O.shape[0] // 2, 1.0, 0, acc, o, 4 if real else 3)
    return acc[0] + acc[1], acc[2], o.n


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("real", [True, False])
def test_count_equals_path_ops(n, real):
    O = inputs.lossy_squeezed(n, 41 + n, (0.3, 0.8), 0.5).O
    _, _, count = model_tor(O, real)
    assert count == flops.path_ops(n, 1 if real else 0)


@pytest.mark.parametrize("real", [True, False])
def test_model_reaches_the_oracle(oracle_mod, real):
    for n, seed in ((5, 3), (7, 9)):
        O = inputs.lossy_squeezed(n, seed, (0.3, 0.8), 0.5).O
        tor, absum, _ = model_tor(O, real)
        ref = oracle_mod.tor_brute(O)
        assert abs(tor - ref.tor) <= 1e-10 * ref.abs_sum
        assert abs(absum - ref.abs_sum) <= 1e-12 * ref.abs_sum
