"""GPU side of sharding: the leaves of one matrix split into 1, 2, 4, 8 aligned
ranges (as 1..8 GPUs would take them), each evaluated with tor_eval_range,
merged on the host, reproduce tor_eval bitwise."""
import numpy as np
import pytest

from paper_2109_04528_gb300 import binding, inputs, shard

pytestmark = pytest.mark.gpu


def test_ranges_merge_to_tor_eval_bitwise():
    inst = inputs.config_single(22)
    with binding.Context(device=0) as c:
        full = binding.tor_eval(c, inst.O)
        L = binding.tor_plan_leaves(c, inst.n)
        assert L >= 8
        for world in (1, 2, 4, 8):
            parts = []
            for rank in range(world):
                lo, count = shard.shard_range(L, world, rank)
                r = binding.tor_eval_range(c, inst.O, lo, count)
                assert r.status == 0
                parts.append((r.hi, r.lo, r.abs_sum))
            merged = shard.tree_merge(parts)
            assert merged == (full.hi, full.lo, full.abs_sum), world
        with pytest.raises(binding.TorError):
            binding.tor_eval_range(c, inst.O, 1, 2)  # not aligned


def test_batch_partition_merges_to_tor_eval_batch_bitwise():
    # each rank's share of a batch, evaluated as its own batch, gives the same
    # bits as the whole batch in one call
    rng = np.random.default_rng(4)
    ns = [int(k) for k in rng.integers(3, 21, size=30)]
    mats = [inputs.lossy_squeezed(n, 3100 + i, (0.5, 1.2), 0.4).O for i, n in enumerate(ns)]
    with binding.Context(device=0) as c:
        whole = binding.tor_eval_batch(c, mats)
        for world in (2, 4):
            for part in shard.partition_batch(ns, world):
                got = binding.tor_eval_batch(c, [mats[i] for i in part]) if part else []
                for i, r in zip(part, got):
                    assert (r.hi, r.lo, r.abs_sum) == (whole[i].hi, whole[i].lo, whole[i].abs_sum)


def test_deep_prefix_two_stage_reduction():
    # p = 23 at n = 24: 2^18 task partials, so the first reduction stage sums
    # chunks of 1024 leaves (4 per thread) and ranges of 2^17 and 2^16 leaves take
    # 2 and 1 per thread; the result agrees with the built-in plan within the
    # FP64 bar, and the ranges merge to it bitwise
    inst = inputs.config_single(24)
    with binding.Context(device=0) as c:
        ref = binding.tor_eval(c, inst.O)
        c.set_prefix_depth(24, 23)
        full = binding.tor_eval(c, inst.O)
        assert full.status == 0
        assert abs((full.hi - ref.hi) + (full.lo - ref.lo)) <= 1e-10 * ref.abs_sum
        assert abs(full.abs_sum - ref.abs_sum) <= 1e-12 * ref.abs_sum
        L = binding.tor_plan_leaves(c, 24)
        assert L == 1 << 18
        for world in (2, 4):
            parts = []
            for rank in range(world):
                lo, count = shard.shard_range(L, world, rank)
                r = binding.tor_eval_range(c, inst.O, lo, count)
                assert r.status == 0
                parts.append((r.hi, r.lo, r.abs_sum))
            assert shard.tree_merge(parts) == (full.hi, full.lo, full.abs_sum), world


def test_range_batch_equals_single_ranges_bitwise():
    # every rank's share of three matrices in one launch (tor_eval_range_batch) gives
    # the bits of its ranges evaluated one by one, whole-matrix entries those of
    # tor_eval, and the ranks' merge those of tor_eval
    mats = [inputs.config_single(22).O, inputs.lossy_squeezed(18, 31, (0.5, 1.2), 0.4).O,
            inputs.lossy_squeezed(8, 32, (0.5, 1.2), 0.4).O]
    with binding.Context(device=0) as c:
        whole = [binding.tor_eval(c, O) for O in mats]
        Ls = [binding.tor_plan_leaves(c, O.shape[0] // 2) for O in mats[:2]]
        assert min(Ls) >= 4
        for world in (2, 4):
            parts = [[], []]
            for rank in range(world):
                ranges = [shard.shard_range(L, world, rank) for L in Ls] + [None]
                got = binding.tor_eval_range_batch(c, mats, ranges)
                for i, (O, rg) in enumerate(zip(mats[:2], ranges)):
                    one = binding.tor_eval_range(c, O, *rg)
                    assert (got[i].hi, got[i].lo, got[i].abs_sum) == (one.hi, one.lo, one.abs_sum)
                    parts[i].append((got[i].hi, got[i].lo, got[i].abs_sum))
                assert (got[2].hi, got[2].lo, got[2].abs_sum) == (whole[2].hi, whole[2].lo, whole[2].abs_sum)
            for i in range(2):
                assert shard.tree_merge(parts[i]) == (whole[i].hi, whole[i].lo, whole[i].abs_sum), (world, i)
        # invalid ranges fail their own entry only
        bad = binding.tor_eval_range_batch(c, mats * 2, [(1, 2), (0, 0), (0, 1), (0, Ls[0]), (Ls[1], 1), None],
                                           check=False)
        assert [r.status for r in bad] == [binding.TOR_EINVAL] * 3 + [0, binding.TOR_EINVAL, 0]
        assert (bad[3].hi, bad[3].lo, bad[3].abs_sum) == (whole[0].hi, whole[0].lo, whole[0].abs_sum)
        assert (bad[5].hi, bad[5].lo, bad[5].abs_sum) == (whole[2].hi, whole[2].lo, whole[2].abs_sum)


def _product_range(inst, p, lo, cnt):
    # closed form of the leaves [lo, lo + cnt) of a product state: leaf t fixes the
    # decisions of modes 0..p-6 (bit j of t set <=> mode j included), its 32 lanes
    # modes p-5..p-1, the walk the rest; each term is prod_{j in Z} x_j times -1 per
    # excluded mode, so free modes give (x_j - 1) (magnitudes x_j + 1) and fixed
    # ones x_j or -1 (magnitudes x_j or 1)
    sh, ch = np.sinh(inst.r), np.cosh(inst.r)
    N, M = inst.eta * sh * sh, inst.eta * sh * ch
    x = np.sqrt((1 + N) ** 2 - M ** 2)
    c = cnt.bit_length() - 1
    tor, absum = 1.0, 1.0
    for j in range(inst.n):
        if c <= j < p - 5:
            inc = (lo >> j) & 1
            tor *= x[j] if inc else -1.0
            absum *= x[j] if inc else 1.0
        else:
            tor *= x[j] - 1.0
            absum *= x[j] + 1.0
    return tor, absum


def test_deep_prefix_shards_beyond_40_modes_against_the_closed_form():
    # n = 42 at p = 26 (2^21 leaves of 2^21 subsets): ranges of one leaf at both ends
    # and inside, and of 1024 leaves, against the product-state closed form
    inst = inputs.product_state(42, 4242, (1.5, 2.5), (0.8, 1.0))
    p = 26
    with binding.Context(device=0) as c:
        c.set_prefix_depth(42, p)
        L = binding.tor_plan_leaves(c, 42)
        assert L == 1 << 21
        ranges = [(0, 1), (L - 1, 1), (0x0A5F3C, 1), (1 << 20, 1024)]
        got = binding.tor_eval_range_batch(c, [inst.O] * len(ranges), ranges)
        for (lo, cnt), r in zip(ranges, got):
            want, absum = _product_range(inst, p, lo, cnt)
            assert r.status == 0
            assert abs(r.abs_sum - absum) <= 1e-12 * absum, (lo, cnt)
            assert abs(r.tor - want) <= max(r.err_est, 1e-13 * absum), (lo, cnt, r.tor, want)
        one = binding.tor_eval_range(c, inst.O, *ranges[2])
        assert (one.hi, one.lo, one.abs_sum) == (got[2].hi, got[2].lo, got[2].abs_sum)


@pytest.mark.parametrize("flags", [0, binding.TOR_COMPLEX_PATH])
def test_deep_prefix_leaf_at_40_modes_against_the_oracle(oracle_mod, flags):
    # n = 40 (the oracle's largest) at p = 28: one leaf is 32 units of 2^12 subsets;
    # its sum against the oracle's units merged by the lane tree (leaves with few
    # prefix modes included, so the oracle's determinants stay small)
    inst = inputs.lossy_squeezed(40, 4040, (0.3, 0.8), 0.5)
    p = 28
    with binding.Context(device=0, flags=flags) as c:
        c.set_prefix_depth(40, p)
        for t in (0, (1 << 3) | (1 << 11) | (1 << 20)):
            r = binding.tor_eval_range(c, inst.O, t, 1)
            units = []
            for lane in range(32):
                u = oracle_mod.tor_unit(inst.O, p, t | (lane << (p - 5)))
                units.append((u.hi, u.lo, u.abs_sum))
            ref = shard.tree_merge(units)
            assert abs((r.hi - ref[0]) + (r.lo - ref[1])) <= 1e-10 * ref[2], t
            assert abs(r.abs_sum - ref[2]) <= 1e-12 * ref[2], t


def test_built_in_plan_bounds_the_units():
    # units of at most 20 modes up to n = 50 (then p = 30, the deepest), and the plan
    # below 41 modes as before: p <= n - 1, leaves = 2^(p-5)
    with binding.Context(device=0) as c:
        for n in range(1, 65):
            p = c.plan_prefix_depth(n)
            assert 0 <= p <= min(n - 1, 30), n
            assert n - p <= max(20, n - 30), n
            if p >= 5:
                assert binding.tor_plan_leaves(c, n) == 1 << (p - 5)
        assert c.plan_prefix_depth(38) == c.plan_prefix_depth(34) == 20
        assert c.plan_prefix_depth(44) == 24 and c.plan_prefix_depth(64) == 30
