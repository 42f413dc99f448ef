"""Floating-point operation counts of three ways to evaluate Eq. (tor), and
the fit of the polynomial exponent omega of Sec. 3 (Eq. linear_fit):

    omega ln N = ln(FLOs) - (N/2) ln 2 - C,      N = 2n (matrix size).

The counts are exact sums over the subset trees, done combinatorially (no
enumeration of the 2^n subsets), with one convention throughout: a complex
multiply-add = 8 flops, a complex |x|^2 = 4, a complex-by-real division = 2,
a real multiply or add = 1, sqrt / 1/sqrt = 1.

  standard   every determinant by its own Cholesky decomposition (Algorithm 1),
             Sec. 1 / Sec. 3 ("each determinant evaluated independently").
  algorithm2 the paper's recursion (Algorithm 2): remove one mode per step,
             reuse L11 and L21 of the parent factor, recompute L22 (Fig. 2).
  rank2      this library's walk: include/exclude one mode per level, extend
             the factor by the mode's two rows with a rank-2 Schur update of
             the trailing block (right-looking), so the polynomial factor per
             subset is O(1) amortised.
"""
from __future__ import annotations

import math


def cholesky_flops(rows: int, start: int = 0) -> int:
    """Algorithm 1 on an m x m Hermitian matrix, computing rows start..m-1 only
    (rows < start, and their columns in later rows, already known).

    Entry (i, j), j < i: j complex MACs and one division; diagonal (i, i):
    i |.|^2 updates, a subtraction and a sqrt.  Columns < start of rows
    >= start are also reused (the L21 block)."""
    f = 0
    for i in range(start, rows):
        for j in range(start, i):
            f += 8 * j + 2
        f += 4 * i + 1 + 1
    return f


def det_term_flops(rows: int) -> int:
    """det = prod |L_ii|^2 (rows multiplies), 1/sqrt, sign and accumulation."""
    return rows + 1 + 2


def standard_flops(n: int) -> int:
    """Sum over all subsets of an independent Cholesky of I - O_Z (2|Z| rows)."""
    return sum(math.comb(n, k) * (cholesky_flops(2 * k) + det_term_flops(2 * k)) for k in range(n + 1))


def algorithm2_flops(n: int) -> int:
    """The remove-mode recursion of Algorithm 2.

    Removing mode i from a node whose removed set R has r modes (all < i, the
    recursion keeps removed indices increasing) leaves q_b = i - r kept modes
    before i and q_a = n - 1 - i after it; the child's factor keeps its first
    2 q_b rows and the L21 columns and recomputes the 2 q_a rows of L22.  The
    number of such nodes is C(i, r)."""
    f = cholesky_flops(2 * n) + det_term_flops(2 * n)  # root: L = chol(I - A)
    for i in range(n):
        for r in range(i + 1):
            qb, qa = i - r, n - 1 - i
            rows = 2 * (qb + qa)
            f += math.comb(i, r) * (cholesky_flops(rows, 2 * qb) + det_term_flops(rows))
    return f


def rank2_flops(n: int) -> int:
    """The add-direction rank-2 walk: at depth j the 2^j nodes include mode j
    into a trailing block of m = n-1-j modes: pivot 10, pivot columns 40 m,
    rank-2 update of the 2m x 2m lower triangle 32 m^2; every leaf 10."""
    f = 10 * 2 ** n
    for j in range(n):
        m = n - 1 - j
        f += 2 ** j * (32 * m * m + 40 * m + 10)
    return f


def path_flops(n: int, path: int = 0) -> float:
    """FP64 flops of the GPU walk over all 2^n subsets in the arithmetic it
    took (tor_result.path: bit 0 real (x, p) basis, bit 1 double-double).

    FP64 factor: the fixed figure of the hot-path contract, per include at m
    trailing modes plus 10 per leaf,
      complex  32 m^2 + 40 m + 10   (= rank2_flops; complex MAC 8 flops,
               complex x real 2, sqrt / rsqrt / div 1)
      real      8 m^2 + 12 m + 10   (real FMA 2: update of the 2m x 2m lower
               triangle 8 m^2 + 4 m, pivot columns 8 m, pivot 10)
    Double-double factor: every FP64 operation of the double-word algorithms
    (add / mul 1, FMA 2; two_sum 6, fast_two_sum 3, two_prod 3; a product
    accumulated into a sum 15, a sum started from a product 7, its final
    normalisation 3; dd_mul 7, the sloppy double-word sum of terms 11,
    reciprocal 18 and reciprocal square root 26 with their Newton steps).
    Includes at m >= 1 trailing modes; the last level (m = 0) is a leaf pair,
    which needs only the determinant factor and the signed pair sum; every
    leaf carries 6 of subtree and accumulator sums:
      real     66 m^2 + 97 m + 97 per include, 70 per leaf pair
               (an update entry: two accumulated products + normalisation 33;
               a pivot-column row 32; pivot 90 and the phi product 7)
      complex 252 m^2 + 188 m + 119 per include, 85 per leaf pair
               (off-diagonal entry 8 products 126, diagonal 63; pivot-column
               row 94; pivot 112 + 7)"""
    real, ext = bool(path & 1), bool(path & 2)
    if not ext:
        a, b, c = (8, 12, 10) if real else (32, 40, 10)
        f = 10.0 * 2.0 ** n
        for j in range(n):
            m = n - 1 - j
            f += 2.0 ** j * (a * m * m + b * m + c)
        return f
    a, b, c, pair = (66, 97, 97, 70.0) if real else (252, 188, 119, 85.0)
    f = 6.0 * 2.0 ** n + pair * 2.0 ** (n - 1)
    for j in range(n - 1):
        m = n - 1 - j
        f += 2.0 ** j * (a * m * m + b * m + c)
    return f


def _leaf_sums(n: int, combine: float, acc: float, regs: int) -> float:
    """Sums above the leaf pairs: every node with 2..regs undecided modes (the
    register-resident subtree) adds its two children's signed sums and
    magnitudes (`combine`), and every register-subtree root -- the nodes with
    min(n, regs) undecided modes -- adds its sum to the lane's accumulator (`acc`)."""
    top = min(n, regs)
    return sum(2.0 ** (n - k) * combine for k in range(2, top + 1)) + 2.0 ** (n - top) * acc


def path_ops(n: int, path: int) -> float:
    """Algorithmic FP64-pipe instructions (add, mul and FMA one each) of the GPU
    walk over all 2^n subsets in the arithmetic `path` (tor_result.path).  The
    FP64 pipe issues one of these per slot whatever its kind, so ops / (the
    measured issue rate) is the pipe's busy fraction in algorithmic work.  The
    hardware rcp / rsqrt estimates that start each reciprocal are not FP64-pipe
    instructions and are not counted.  Per include at m >= 1 trailing modes /
    per leaf pair, and the sums above the leaves:
      FP64 real      4 m^2 + 8 m + 14 / 9    (2 FMA per entry; a pivot-column
                     row 3; pivot: det 2, rsqrt 5, rcp 3, l 1, 1/d2 2, phi 1;
                     a leaf pair: det 2, rsqrt 5, its signed and magnitude
                     sums one FMA each); a subtree sum 2, the lane's
                     double-double sum 8; subtrees of 4 modes in registers
      FP64 complex  16 m^2 + 16 m + 16 / 10  (8 FMA per off-diagonal entry, 4
                     per diagonal one; a row 8; pivot 15 + phi 1); 3 modes
      double-double real     54 m^2 + 73 m + 65 / 53
      double-double complex 204 m^2 + 140 m + 81 / 65
                     (two_sum 6, fast_two_sum 3, two_prod 2, an accumulated
                     product 12, a sum started from a product 4, its
                     normalisation 3, dd_mul 4, the sloppy double-word sum of
                     terms 11, reciprocal 12, reciprocal square root 18); a
                     subtree sum and the lane's sum 12 each; 2 modes."""
    real, ext = bool(path & 1), bool(path & 2)
    a, b, c, pair, combine, acc, regs = {
        (True, False): (4, 8, 14, 9.0, 2.0, 8.0, 4), (False, False): (16, 16, 16, 10.0, 2.0, 8.0, 3),
        (True, True): (54, 73, 65, 53.0, 12.0, 12.0, 2), (False, True): (204, 140, 81, 65.0, 12.0, 12.0, 2)}[(real, ext)]
    f = pair * 2.0 ** (n - 1) + _leaf_sums(n, combine, acc, regs)
    for j in range(n - 1):
        m = n - 1 - j
        f += 2.0 ** j * (a * m * m + b * m + c)
    return f


def fit_omega(counts: dict[int, int]) -> tuple[float, float]:
    """Least-squares fit of Eq. (linear_fit): ln F - (N/2) ln 2 = omega ln N + C
    over the given {N: FLOs}.  Returns (omega, C)."""
    xs = [math.log(N) for N in counts]
    ys = [math.log(F) - (N / 2) * math.log(2.0) for N, F in counts.items()]
    k = len(xs)
    mx, my = sum(xs) / k, sum(ys) / k
    sxx = sum((x - mx) ** 2 for x in xs)
    sxy = sum((x - mx) * (y - my) for x, y in zip(xs, ys))
    omega = sxy / sxx
    return omega, my - omega * mx


def experiment(N_lo: int = 26, N_hi: int = 60):
    """The Sec. 3 experiment on even N in [N_lo, N_hi]: omega of each method and
    the standard / recursive ratios at N = 50 and N = 100."""
    Ns = list(range(N_lo, N_hi + 1, 2))
    out = {}
    for name, fn in (("standard", standard_flops), ("algorithm2", algorithm2_flops), ("rank2", rank2_flops)):
        out[name] = fit_omega({N: fn(N // 2) for N in Ns})[0]
    out["ratio_std_alg2_N50"] = standard_flops(25) / algorithm2_flops(25)
    out["ratio_std_alg2_N100"] = standard_flops(50) / algorithm2_flops(50)
    out["ratio_alg2_rank2_N50"] = algorithm2_flops(25) / rank2_flops(25)
    return out


if __name__ == "__main__":
    import json
    print(json.dumps(experiment(), indent=1))
