"""GPU parity of the extended-precision factor (TOR_EXTENDED; Sec. 5, "X =
extended": the Cholesky / Schur arithmetic in more than double precision)
against the binary128 oracle, through the C ABI.

Pass criterion (element by element, same seeded inputs):
    |Tor_gpu - Tor_oracle| <= 1e-26 * sum_Z |term_Z|.
Derivation: a term passes through at most n include steps, each a few
double-double operations per entry with relative error <= ~10 u^2
(u^2 = 2^-106 ~ 1.2e-32), amplified by the conditioning of the pivot blocks
(below ~100 for these inputs), so a term is off by < ~1e-28 of itself and the
sum by < ~1e-28 sum|term|; 1e-26 leaves a factor of 100.  The oracle's own
error (binary128, u = 2^-113) is below 1e-31 sum|term|.  One FP64 operation
left anywhere on the path (a lost low word) misses the bound by ~10 orders.
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_2109_04528_gb300 import binding, inputs, shard

pytestmark = pytest.mark.gpu
TOL_X = 1e-26
_REF = {}


@pytest.fixture(scope="module", params=["auto", "complex"])
def xctx(request):
    # "auto": structured inputs take the real (x, p) basis (RealX), others CplxX
    from paper_2109_04528_gb300 import build
    build.build()
    flags = binding.TOR_EXTENDED | (binding.TOR_COMPLEX_PATH if request.param == "complex" else 0)
    c = binding.Context(device=0, flags=flags)
    c.kind = request.param
    yield c
    c.close()


def ref(oracle_mod, key, O):
    if key not in _REF:
        _REF[key] = oracle_mod.tor_brute(O)
    return _REF[key]


def err(got, r):
    return abs((got.hi - r.hi) + (got.lo - r.lo))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 9, 12, 14, 16])
def test_lossy_vs_oracle(xctx, oracle_mod, n):
    inst = inputs.lossy_squeezed(n, 500 + n, (0.3, 0.8), (0.3, 0.7))
    r = binding.tor_eval(xctx, inst.O)
    o = ref(oracle_mod, ("lossy", n), inst.O)
    assert r.status == 0
    assert r.path == (2 if xctx.kind == "complex" else 3)
    assert err(r, o) <= TOL_X * o.abs_sum, (r, o, err(r, o) / o.abs_sum)
    assert abs(r.abs_sum - o.abs_sum) <= 1e-12 * o.abs_sum


@pytest.mark.parametrize("n", [3, 8, 11])
def test_general_hermitian_vs_oracle(xctx, oracle_mod, n):
    inst = inputs.random_hermitian_contraction(n, 600 + n, 0.85)
    r = binding.tor_eval(xctx, inst.O)
    o = ref(oracle_mod, ("herm", n), inst.O)
    assert r.path == 2  # no (x, p) structure: complex double-double
    assert err(r, o) <= TOL_X * o.abs_sum


def test_every_prefix_depth(xctx, oracle_mod):
    # p < 5 (lane-built roots) and p >= 5 (warp-built task node + fan-out)
    n = 11
    inst = inputs.lossy_squeezed(n, 77, (0.5, 1.2), 0.4)
    o = ref(oracle_mod, ("depth", n), inst.O)
    old = xctx.plan_prefix_depth(n)
    try:
        for p in range(0, n):
            xctx.set_prefix_depth(n, p)
            r = binding.tor_eval(xctx, inst.O)
            assert r.status == 0
            assert err(r, o) <= TOL_X * o.abs_sum, p
    finally:
        xctx.set_prefix_depth(n, old)


def test_product_state_exact_product(xctx, oracle_mod):
    # Tor of a product state is prod_j Tor(O_j) exactly (Eq. tor factorises);
    # the one-mode factors from the oracle, multiplied exactly in rationals.
    n = 20
    inst = inputs.product_state(n, 720)
    mask = np.zeros((2 * n, 2 * n), dtype=bool)
    for j in range(n):
        idx = [j, j + n]
        mask[np.ix_(idx, idx)] = True
    assert np.all(inst.O[~mask] == 0)
    want, absum = Fraction(1), Fraction(1)
    for j in range(n):
        f = oracle_mod.tor_brute(inputs.submatrix(inst.O, [j]))
        want *= Fraction(f.hi) + Fraction(f.lo)
        absum *= Fraction(f.abs_sum)
    r = binding.tor_eval(xctx, inst.O)
    assert r.status == 0
    assert abs(Fraction(r.hi) + Fraction(r.lo) - want) <= Fraction(TOL_X) * absum


def test_low_squeezing_relative_accuracy(xctx, oracle_mod):
    # Sec. 5: weak squeezing, terms near +-1 cancelling to Tor ~ 1e-15
    # (kappa = sum|term| / |Tor| ~ 1e19).  Double-double keeps ~10 digits of
    # Tor; the FP64 factor keeps none.
    inst = inputs.lossy_squeezed(14, 4256, (0.1, 0.2), 1.0)
    o = ref(oracle_mod, ("weak", 14), inst.O)
    assert o.abs_sum / abs(o.tor) > 1e18
    r = binding.tor_eval(xctx, inst.O)
    ex = err(r, o)
    assert ex <= 1e-6 * abs(o.tor), ex / abs(o.tor)
    flags = binding.TOR_COMPLEX_PATH if xctx.kind == "complex" else 0
    with binding.Context(device=0, flags=flags) as c:
        d = binding.tor_eval(c, inst.O)
    assert err(d, o) > 100 * ex


def test_batch_bitwise_equals_single(xctx):
    rng = np.random.default_rng(12)
    mats = [inputs.lossy_squeezed(int(k), 950 + i, (0.5, 1.2), 0.4).O
            for i, k in enumerate(rng.integers(1, 17, size=24))]
    mats.append(inputs.random_hermitian_contraction(7, 3, 0.8).O)
    batch = binding.tor_eval_batch(xctx, mats)
    for O, b in zip(mats, batch):
        s = binding.tor_eval(xctx, O)
        assert (s.hi, s.lo, s.abs_sum, s.status, s.path) == (b.hi, b.lo, b.abs_sum, b.status, b.path)


def test_deterministic_and_errors(xctx):
    inst = inputs.config_single(18)
    a = binding.tor_eval(xctx, inst.O)
    b = binding.tor_eval(xctx, inst.O)
    assert (a.hi, a.lo, a.abs_sum) == (b.hi, b.lo, b.abs_sum)
    r = binding.tor_eval(xctx, np.zeros((0, 0), dtype=np.complex128))
    assert r.tor == 1.0 and r.status == 0
    with pytest.raises(binding.TorError) as e:
        binding.tor_eval(xctx, 2 * np.eye(4, dtype=np.complex128))
    assert e.value.status == binding.TOR_ENOTPD
    v = binding.tor_eval(xctx, inputs.vacuum(9).O)
    assert v.tor == 0.0 and v.abs_sum == 512.0


def test_units_at_n24_sampled(xctx, oracle_mod):
    inst = inputs.config_single(24)
    res, p, parts = binding.tor_eval_units(xctx, inst.O)
    assert res.status == 0 and p >= 5
    rng = np.random.default_rng(3)
    for u in [0, (1 << p) - 1] + list(rng.integers(0, 1 << p, size=3)):
        o = oracle_mod.tor_unit(inst.O, p, int(u))
        got_hi, got_lo, got_abs = parts[int(u)]
        assert abs((got_hi - o.hi) + (got_lo - o.lo)) <= TOL_X * o.abs_sum, u


def test_ranges_merge_bitwise(xctx):
    inst = inputs.config_single(20)
    full = binding.tor_eval(xctx, inst.O)
    L = binding.tor_plan_leaves(xctx, inst.n)
    for world in (2, 4):
        parts = []
        for rank in range(world):
            lo, count = shard.shard_range(L, world, rank)
            r = binding.tor_eval_range(xctx, inst.O, lo, count)
            parts.append((r.hi, r.lo, r.abs_sum))
        assert shard.tree_merge(parts) == (full.hi, full.lo, full.abs_sum), world


def test_inexact_structure_takes_complex_path(xctx, oracle_mod):
    # structured only to ~1e-16 (as a numerically inverted O would be): the
    # double-double path must not take the real (x, p) form, which reads one
    # half of the blocks only
    inst = inputs.lossy_squeezed(9, 66, (0.3, 0.8), 0.5)
    O = inst.O.copy()
    n = 9
    O[n + 1, n + 2] += 1e-16
    O[n + 2, n + 1] += 1e-16
    r = binding.tor_eval(xctx, O)
    o = oracle_mod.tor_brute(O)
    assert r.path == 2
    assert err(r, o) <= TOL_X * o.abs_sum


def test_graph_replay_and_served_equal_plain(xctx):
    # the same matrices through a CUDA-graph context and through the serving loop:
    # bitwise the plain extended result
    rng = np.random.default_rng(21)
    mats = [inputs.lossy_squeezed(int(k), 1500 + i, (0.5, 1.2), 0.4).O for i, k in enumerate(rng.integers(4, 15, 8))]
    plain = binding.tor_eval_batch(xctx, mats)
    flags = binding.TOR_EXTENDED | binding.TOR_GRAPHS | (binding.TOR_COMPLEX_PATH if xctx.kind == "complex" else 0)
    with binding.Context(device=0, flags=flags) as g:
        for _ in range(2):  # capture, then replay
            got = binding.tor_eval_batch(g, mats)
            assert [(r.hi, r.lo, r.abs_sum, r.path) for r in got] == [(r.hi, r.lo, r.abs_sum, r.path) for r in plain]
    tickets = [binding.tor_submit(xctx, O) for O in mats]
    for t, p in zip(tickets, plain):
        st, r = binding.tor_poll(xctx, t, 60.0)
        assert st == 0 and (r.hi, r.lo, r.abs_sum) == (p.hi, p.lo, p.abs_sum)


@pytest.mark.parametrize("name", ["lossy_n20.json", "lossy_n22.json", "lossy_n24.json", "lossy_n30.json"])
def test_golden_full_sum(xctx, name):
    # n = 20, 22 (full brute force), 24 and 30 (binary128 Algorithm 2) against the
    # oracle's stored sums, at the double-double bound
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)) as f:
        g = json.load(f)
    O = np.array(g["O_re"]) + 1j * np.array(g["O_im"])
    r = binding.tor_eval(xctx, O)
    assert r.status == 0
    assert abs((r.hi - g["tor_hi"]) + (r.lo - g["tor_lo"])) <= TOL_X * g["abs_sum"]
