"""Host-side helpers of bench.py, on the CPU: the kernel count behind the
`gpu_launches` claim, the spread sample of the oracle baseline, the
Algorithm 2 baseline leg on a small matrix, and the strong-scaling step of
several ranks (leaf ranges, gather, fixed-tree merge) on two gloo ranks."""
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


def test_sharded_depths_keep_the_tasks_per_rank():
    # two ranks keep the plan; 4 and 8 ranks deepen it by 1 and 2 levels, within p <= min(30, n - 1)
    plan = PlanStub({30: 19, 34: 20, 12: 11})
    assert bench.sharded_depths(plan, [30, 34], 2) == {30: 19, 34: 20}
    assert bench.sharded_depths(plan, [34, 30, 34], 4) == {30: 20, 34: 21}
    assert bench.sharded_depths(plan, [30, 34, 12], 8) == {12: 11, 30: 21, 34: 22}
    assert bench.sharded_depths(PlanStub({40: 29}), [40], 16) == {40: 30}


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


class LeafStub:
    """Stands in for the binding and a context on the CPU: a matrix with n modes has
    2^(n-10) reduction leaves with fixed partial sums, and tor_eval_range_batch
    returns the binary-tree sum of each range's leaves, as the device does."""

    class Res:
        def __init__(self, t):
            self.hi, self.lo, self.abs_sum = t

    def __init__(self):
        self.calls = []

    def leaves(self, n):
        return [(1.0 + k / 7.0, (k % 5) * 2.0 ** -60, 1.0 + k) for k in range(1 << (n - 10))]

    def tor_plan_leaves(self, ctx, n):
        return 1 << (n - 10)

    def tor_eval_range_batch(self, ctx, mats, ranges):
        from paper_2109_04528_gb300 import shard
        self.calls.append(list(zip(mats, ranges)))
        return [self.Res(shard.tree_merge(self.leaves(O)[lo:lo + cnt])) for O, (lo, cnt) in zip(mats, ranges)]

    def last_times(self):
        return {"units_ms": 1.0}


def _sharded_rank_main(rank, world, port, out_dir):
    import os

    import numpy as np
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    stub = LeafStub()
    ns = [14, 16]
    res, units = bench.sharded_step(stub, stub, ns, ns, world, rank)  # "matrices" are their n here
    np.save(os.path.join(out_dir, f"s{rank}.npy"),
            np.array([[r.hi, r.lo, r.abs_sum] for r in res] + [[units, len(stub.calls), stub.calls[0][1][1][0]]]))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_step_two_ranks_equals_one_gpu(tmp_path):
    # the bench's strong-scaling step on two gloo ranks: each rank evaluates half the leaves
    # of every matrix, and the merged results equal the single-range tree sum bitwise
    import socket

    import numpy as np
    import torch.multiprocessing as mp

    from paper_2109_04528_gb300 import shard
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mp.start_processes(_sharded_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    stub = LeafStub()
    want = [shard.tree_merge(stub.leaves(n)) for n in (14, 16)]
    for rank in range(2):
        got = np.load(tmp_path / f"s{rank}.npy")
        assert [tuple(row) for row in got[:2]] == want
        assert tuple(got[2]) == (1.0, 1, rank * (1 << 5))  # one launch; n = 16's half starts at leaf 32


def test_product_closed_form_matches_the_oracle(oracle_mod):
    # the bench's reference for its n = 38 product state, checked against the binary128
    # brute force of Eq. (tor) on a small product state of the same recipe
    inst = inputs.product_state(6, 4242)
    tor, absum = bench.product_closed_form(inst)
    r = oracle_mod.tor_brute(inst.O)
    assert abs(r.tor - tor) <= 1e-13 * abs(tor)
    assert abs(r.abs_sum - absum) <= 1e-13 * absum


def test_result_record_states_errors_against_the_reference():
    class R:
        def __init__(self, hi, lo, abs_sum, err_est):
            self.hi, self.lo, self.abs_sum, self.err_est, self.path = hi, lo, abs_sum, err_est, 1

        @property
        def tor(self):
            return self.hi + self.lo
    r64 = R(1.0e-10, 0.0, 1.0e6, 1.0e-8)
    rx = R(2.0e-12, 1.0e-29, 1.0e6, 1.0e-20)
    rec = bench.result_record("m", 20, r64, rx, {"hi": 2.0e-12, "lo": 0.0, "name": "binary128 oracle"})
    assert rec["kappa"] == 1.0e6 / 2.0e-12
    assert abs(rec["fp64"]["abs_err"] - (1.0e-10 - 2.0e-12)) <= 1e-25
    assert rec["fp64"]["within_err_est"] and rec["extended"]["within_err_est"]
    assert rec["extended"]["abs_err"] == 1.0e-29
    # against the double-double GPU path, only the FP64 result gets an error (the reference is itself)
    rec2 = bench.result_record("m", 20, r64, rx, {"hi": rx.hi, "lo": rx.lo, "name": "double-double GPU path",
                                                  "bound": rx.err_est})
    assert "abs_err" in rec2["fp64"] and "abs_err" not in rec2["extended"] and rec2["ref_err_bound"] == 1.0e-20
    assert bench.result_record("m", 20, r64)["ref"] is None


def test_accuracy_row_states_both_paths_against_the_reference():
    class R:
        def __init__(self, hi, lo=0.0, abs_sum=1.0e6, err_est=1.0e-9):
            self.hi, self.lo, self.abs_sum, self.err_est = hi, lo, abs_sum, err_est
    r64, rx, ref = R(1.1e-3), R(1.0e-3, 2.0e-20, err_est=1e-21), R(1.0e-3, 1.0e-20)
    row = bench.accuracy_row(12, 0.2, r64, rx, oracle_ref=ref)
    assert row["ref"] == "binary128 oracle" and abs(row["kappa"] - 1.0e9) <= 1e-3
    assert abs(row["fp64_rel_err"] - 0.1) <= 1e-12 and abs(row["ext_rel_err"] - 1e-17) <= 1e-22
    assert abs(row["fp64_rel_bound"] - 1e-6) <= 1e-18
    row = bench.accuracy_row(24, 0.2, r64, rx, rx_rev=R(1.0e-3, 5.0e-20))
    assert row["ref"] == "double-double GPU path" and "ext_rel_err" not in row
    assert abs(row["ext_rel_diff_reversed"] - 3e-17) <= 1e-22


def test_sample_work_counts_each_distinct_marginal_once():
    import numpy as np
    pat = np.array([[1, 0, 1], [1, 0, 0], [0, 1, 1]], dtype=np.uint8)
    terms, evals = bench.sample_work(pat)
    # step 0: S = {} for all; step 1: {0}, {}; step 2: {0}, {0}, {1} -> {0}, {1}
    assert evals == 2 * (1 + 2 + 2)
    assert terms == 3.0 * (1 + (2 + 1) + (2 + 2))
