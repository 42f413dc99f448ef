"""Host-side helpers of bench.py, on the CPU: the kernel count behind the
`gpu_launches` claim, the spread sample of the oracle baseline, and the
Algorithm 2 baseline leg on a small matrix."""
import pytest

import bench
from paper_2109_04528_gb300 import inputs


class PlanStub:
    """Stands in for a context: prefix depth per n."""

    def __init__(self, plan):
        self.plan = plan

    def plan_prefix_depth(self, n):
        return self.plan[n]


def test_launches_per_step_counts_the_first_reduction_stage():
    # k_intake, k_units and k_reduce always; k_reduce_chunks once a matrix has more
    # than 256 reduction leaves (2^(p-5) for p >= 5, 2^p below)
    assert bench.launches_per_step(PlanStub({16: 12}), [16]) == 3        # 2^7 task partials
    assert bench.launches_per_step(PlanStub({16: 12, 20: 16}), [16, 20]) == 4  # 2^11 for n = 20
    assert bench.launches_per_step(PlanStub({8: 4}), [8]) == 3        # 2^4 unit partials
    assert bench.launches_per_step(PlanStub({14: 13}), [14]) == 3     # 2^8: one stage
    assert bench.launches_per_step(PlanStub({15: 14}), [15]) == 4     # 2^9: two stages
    assert bench.launches_per_step(PlanStub({30: 19, 8: 4}), [8, 30]) == 4


@pytest.mark.parametrize("n,count", [(10, 1), (10, 7), (12, 100), (20, 1000), (8, 1 << 8)])
def test_spread_sample_covers_the_range(n, count):
    stride, k = bench.spread_sample(n, count)
    assert k == min(count, 1 << n)
    assert stride % 2 == 1 or k >= (1 << n) or k == 1
    assert (k - 1) * stride < (1 << n)  # every mask of the sample exists


def test_cpu_alg2_leg_runs_the_whole_small_sum():
    pytest.importorskip("oracle.alg2_cpu")
    out = bench.cpu_alg2([inputs.config_single(10).O, inputs.config_single(12).O], 2.0)
    assert out["unit"] == "subset terms/s" and out["value"] > 0
    assert out["sample"].startswith("all of the 2^12 terms")
    assert out["cores"] >= 1 and "Algorithm 2" in out["kind"]
