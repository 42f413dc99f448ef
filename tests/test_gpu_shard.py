"""GPU side of sharding: the leaves of one matrix split into 1, 2, 4, 8 aligned
ranges (as 1..8 GPUs would take them), each evaluated with tor_eval_range,
merged on the host, reproduce tor_eval bitwise."""
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
