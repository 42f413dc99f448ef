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
