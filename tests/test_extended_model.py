"""CPU model of the double-double (extended-precision) subset-tree walk.

A plain-Python restatement of the arithmetic of TOR_EXTENDED: double-word
values (h, l) built from the error-free transformations (two_sum, fast_two_sum,
two_prod via a correctly rounded FMA), products accumulated into sums, the
Newton-refined reciprocal and reciprocal square root, the rank-2 include step
of the subset tree (Sec. 2, Fig. 2, run in the add-a-mode direction) and the
signed leaf sums of Eq. (tor).  Every FP64 operation is counted (add / mul 1,
FMA 2).  Two checks:
  * the count equals paper_2109_04528_gb300.flops.path_flops (the figure the
    benchmark divides by), for the real (x, p) and the complex walk;
  * the model reaches the binary128 oracle to 1e-26 sum|term|, i.e. the
    double-word algorithms themselves carry the accuracy the GPU tests ask for.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2109_04528_gb300 import flops, inputs


class Ops:
    def __init__(self):
        self.f = 0    # flops (FMA 2, a reciprocal estimate 1)
        self.fmas = 0
        self.ests = 0

    @property
    def ops(self):  # FP64-pipe instructions (FMA 1; the estimates are not FP64-pipe instructions)
        return self.f - self.fmas - self.ests

    def add(self, a, b):
        self.f += 1
        return a + b

    def sub(self, a, b):
        self.f += 1
        return a - b

    def mul(self, a, b):
        self.f += 1
        return a * b

    def fma(self, a, b, c):
        self.f += 2
        self.fmas += 1
        return float(Fraction(a) * Fraction(b) + Fraction(c))

    # error-free transformations
    def two_sum(self, a, b):
        s = self.add(a, b)
        bb = self.sub(s, a)
        return s, self.add(self.sub(a, self.sub(s, bb)), self.sub(b, bb))

    def fast_two_sum(self, a, b):
        s = self.add(a, b)
        return s, self.sub(b, self.sub(s, a))

    def two_prod(self, a, b):
        p = self.mul(a, b)
        return p, self.fma(a, b, -p)

    # double-word operations
    def dd_add(self, a, b):
        s, e = self.two_sum(a[0], b[0])
        t, f = self.two_sum(a[1], b[1])
        s, e = self.fast_two_sum(s, self.add(e, t))
        return self.fast_two_sum(s, self.add(e, f))

    def dd_sum(self, a, b):  # the sloppy double-word sum, for sums of terms
        s, e = self.two_sum(a[0], b[0])
        e = self.add(e, self.add(a[1], b[1]))
        return self.fast_two_sum(s, e)

    def dd_sub(self, a, b):
        return self.dd_sum(a, (-b[0], -b[1]))

    def dd_mul(self, a, b):  # not renormalised: |e| <= ~2.5 u |p|
        p, e = self.two_prod(a[0], b[0])
        e = self.fma(a[0], b[1], e)
        e = self.fma(a[1], b[0], e)
        return (p, e)

    def acc_start(self, b, c):  # a sum that starts from the product b c
        h, t = self.two_prod(b[0], c[0])
        t = self.fma(b[0], c[1], t)
        return [h, self.fma(b[1], c[0], t)]

    def acc_add(self, acc, b, c, sign):  # acc += sign b c
        p, e = self.two_prod(sign * b[0], c[0])
        e = self.fma(sign * b[0], c[1], e)
        e = self.fma(sign * b[1], c[0], e)
        s, r = self.two_sum(acc[0], p)
        acc[0] = s
        acc[1] = self.add(acc[1], self.add(r, e))

    def acc_out(self, acc):
        return self.fast_two_sum(acc[0], acc[1])

    def rcp(self, a):
        x = a[0]
        y = float(np.float32(1.0 / x))  # a coarse estimate (the hardware's is ~2^-20)
        self.f += 1
        self.ests += 1
        e = self.fma(-x, y, 1.0)
        s = self.fma(e, e, e)
        y = self.fma(y, s, y)
        p, q = self.two_prod(x, y)
        e = self.fma(-a[1], y, self.sub(self.sub(1.0, p), q))
        return self.fast_two_sum(y, self.mul(y, e))

    def rsqrt(self, a):
        x = a[0]
        y = float(np.float32(1.0 / math.sqrt(x)))
        self.f += 1
        self.ests += 1
        t = self.mul(x, y)
        e = self.fma(-t, y, 1.0)
        p = self.fma(0.375, e, 0.5)
        q = self.mul(y, e)
        y = self.fma(q, p, y)
        s, t = self.two_prod(y, y)
        p, q = self.two_prod(x, s)
        e = self.sub(self.sub(1.0, p), q)
        e = self.fma(-x, t, e)
        e = self.fma(-a[1], s, e)
        return self.fast_two_sum(y, self.mul(self.mul(0.5, y), e))


# Real entries are double words (h, l); complex entries pairs of them.
Z = (0.0, 0.0)


class RealArith:
    def __init__(self, ops):
        self.o = ops

    def det2(self, a, b, e):
        acc = self.o.acc_start(a, e)
        self.o.acc_add(acc, b, b, -1.0)
        return self.o.acc_out(acc)

    def cl(self, b, ia):
        return self.o.dd_mul(b, ia)

    def reduce_col(self, x, y, c):
        acc = list(y)
        self.o.acc_add(acc, x, c, -1.0)
        return self.o.acc_out(acc)

    def scale(self, v, s):
        return self.o.dd_mul(v, s)

    def rank2(self, s, xt, xk, yt, yk):
        acc = list(s)
        self.o.acc_add(acc, xt, xk, -1.0)
        self.o.acc_add(acc, yt, yk, -1.0)
        return self.o.acc_out(acc)

    rank2_diag = rank2

    def re(self, v):
        return v

    def diag(self, d):
        return d


class CplxArith:
    def __init__(self, ops):
        self.o = ops

    def det2(self, a, b, e):
        acc = self.o.acc_start(a, e)
        self.o.acc_add(acc, b[0], b[0], -1.0)
        self.o.acc_add(acc, b[1], b[1], -1.0)
        return self.o.acc_out(acc)

    def cl(self, b, ia):
        im = self.o.dd_mul(b[1], ia)
        return (self.o.dd_mul(b[0], ia), (-im[0], -im[1]))

    def reduce_col(self, x, y, c):
        r, i = list(y[0]), list(y[1])
        self.o.acc_add(r, x[0], c[0], -1.0)
        self.o.acc_add(r, x[1], c[1], 1.0)
        self.o.acc_add(i, x[0], c[1], -1.0)
        self.o.acc_add(i, x[1], c[0], -1.0)
        return (self.o.acc_out(r), self.o.acc_out(i))

    def scale(self, v, s):
        return (self.o.dd_mul(v[0], s), self.o.dd_mul(v[1], s))

    def rank2(self, s, xt, xk, yt, yk):  # s - xt conj(xk) - yt conj(yk)
        r, i = list(s[0]), list(s[1])
        for (u, w) in ((xt, xk), (yt, yk)):
            self.o.acc_add(r, u[0], w[0], -1.0)
            self.o.acc_add(r, u[1], w[1], -1.0)
        for (u, w) in ((xt, xk), (yt, yk)):
            self.o.acc_add(i, u[1], w[0], -1.0)
            self.o.acc_add(i, u[0], w[1], 1.0)
        return (self.o.acc_out(r), self.o.acc_out(i))

    def rank2_diag(self, d, xt, x, yt, y):
        r = list(d)
        for (u, w) in ((xt, x), (yt, y)):
            self.o.acc_add(r, u[0], w[0], -1.0)
            self.o.acc_add(r, u[1], w[1], -1.0)
        return self.o.acc_out(r)

    def re(self, v):
        return v[0]

    def diag(self, d):
        return (d, Z)


def include(A, S, o):
    """Include the first mode of S (dict (i, k) -> entry, i >= k, rows 0..R-1):
    returns the Schur complement over the other rows and rho = det(pivot)^-1/2."""
    R = max(i for i, _ in S) + 1
    a, b, e = A.re(S[(0, 0)]), S[(1, 0)], A.re(S[(1, 1)])
    det2 = A.det2(a, b, e)
    rho = o.rsqrt(det2)
    ia = o.rcp(a)
    cl = A.cl(b, ia)
    id2 = o.dd_mul(a, o.dd_mul(rho, rho))
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
    R = max(i for i, _ in S) + 1
    return {(i - 2, k - 2): v for (i, k), v in S.items() if i >= 2 and k >= 2 and i < R}


def leaf_pair(A, S, phi, o):
    det2 = A.det2(A.re(S[(0, 0)]), S[(1, 0)], A.re(S[(1, 1)]))
    pr = o.dd_mul(phi, o.rsqrt(det2))
    v = o.dd_sub(pr, phi)
    o.f += 1  # sum of magnitudes
    return v


def subtree(A, S, m, phi, o):
    """Signed sum below a node with m <= 2 modes (register subtree)."""
    if m == 1:
        return leaf_pair(A, S, phi, o)
    v1 = subtree(A, trail(S), m - 1, phi, o)
    C, rho = include(A, S, o)
    v2 = subtree(A, C, m - 1, o.dd_mul(phi, rho), o)
    o.f += 1  # sum of magnitudes
    return o.dd_sub(v2, v1)


def walk(A, S, m, phi, excl, acc, o):
    if m <= 2:
        v = subtree(A, S, m, phi, o)  # signs of the exclusions below this node included
        sign = -1.0 if excl % 2 else 1.0  # (-1)^(modes excluded above)
        acc[0] = o.dd_sum(acc[0], (sign * v[0], sign * v[1]))
        o.f += 1
        return
    walk(A, trail(S), m - 1, phi, excl + 1, acc, o)
    C, rho = include(A, S, o)
    walk(A, C, m - 1, o.dd_mul(phi, rho), excl, acc, o)


def b_entries(O, real):
    """B = I - O in pairs order (or V = U^H B U for the real walk), as double words."""
    n = O.shape[0] // 2
    idx = [j + c * n for j in range(n) for c in (0, 1)]
    S = {}
    for r in range(2 * n):
        for s in range(r + 1):
            if not real:
                hr = Fraction(int(r == s)) - Fraction(O[idx[r], idx[s]].real)
                S[(r, s)] = (split(hr), split(-Fraction(O[idx[r], idx[s]].imag))) if r != s else (split(hr), Z)
            else:
                j, k = r // 2, s // 2
                Are = Fraction(int(j == k)) - Fraction(O[j, k].real)
                Aim = -Fraction(O[j, k].imag)
                Cre = -Fraction(O[j, k + n].real)
                Cim = -Fraction(O[j, k + n].imag)
                if r % 2 == 0:
                    v = Are + Cre if s % 2 == 0 else Cim - Aim
                else:
                    v = Aim + Cim if s % 2 == 0 else Are - Cre
                S[(r, s)] = split(v)
    return S


def split(q: Fraction):
    h = float(q)
    return (h, float(q - Fraction(h)))


def model_tor(O, real):
    o = Ops()
    A = RealArith(o) if real else CplxArith(o)
    n = O.shape[0] // 2
    S = b_entries(O, real)
    acc = [(0.0, 0.0)]
    walk(A, S, n, (1.0, 0.0), 0, acc, o)
    h, l = acc[0]
    model_tor.ops = o.ops
    return Fraction(h) + Fraction(l), o.f


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("real", [True, False])
def test_count_equals_path_flops(n, real):
    O = inputs.lossy_squeezed(n, 31 + n, (0.3, 0.8), 0.5).O
    _, f = model_tor(O, real)
    assert f == flops.path_flops(n, 2 | (1 if real else 0))
    assert model_tor.ops == flops.path_ops(n, 2 | (1 if real else 0))


@pytest.mark.parametrize("real", [True, False])
def test_model_reaches_the_oracle(oracle_mod, real):
    for n, seed, rr, eta in ((5, 3, (0.3, 0.8), 0.5), (6, 4256, (0.1, 0.2), 1.0)):
        O = inputs.lossy_squeezed(n, seed, rr, eta).O
        tor, _ = model_tor(O, real)
        ref = oracle_mod.tor_brute(O)
        assert abs(tor - (Fraction(ref.hi) + Fraction(ref.lo))) <= Fraction(1e-26) * Fraction(ref.abs_sum)
