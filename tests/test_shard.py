"""Sharding of one Torontonian across ranks (host logic, gloo, world_size 2, CPU).

Each rank computes its leaves' partial sums -- on CPU the leaves are warp
tasks of 32 prefix units whose sums come from the oracle -- and the ranks
merge them through torch.distributed.  The merged result must equal the
single-process tree bitwise and the full oracle sum to binary128 accuracy.
"""
import os

import numpy as np
import pytest

from paper_2109_04528_gb300 import binding, inputs, shard

N, P = 9, 6  # 2^(P-5) = 2 leaves (warp tasks), each 32 units of 2^(N-P) subsets


def task_partial(oracle_mod, O, t, p=P):
    # lane l of task t takes unit u = t | (l << (p-5)); lanes merge by a binary tree over lane index
    # (the shape of the device's lane tree, which leaves low parts unnormalised between levels)
    units = []
    for lane in range(32):
        r = oracle_mod.tor_unit(O, p, t | (lane << (p - 5)), threads=1)
        units.append((r.hi, r.lo, r.abs_sum))
    return shard.tree_merge(units)


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    O = inputs.lossy_squeezed(N, 1234, (0.5, 1.2), 0.4).O
    lo, count = shard.shard_range(1 << (P - 5), world, rank)
    mine = shard.tree_merge([task_partial(oracle, O, t) for t in range(lo, lo + count)])
    merged = shard.gather_merge(mine)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), np.array(merged))
    dist.barrier()
    dist.destroy_process_group()


def test_tree_merge_is_binary_and_ordered():
    parts = [(float(i), 0.0, 1.0) for i in range(8)]
    assert shard.tree_merge(parts) == (28.0, 0.0, 8.0)
    with pytest.raises(ValueError):
        shard.tree_merge(parts[:3])
    assert shard.shard_range(16, 4, 3) == (12, 4)
    with pytest.raises(ValueError):
        shard.shard_range(4, 3, 0)


def test_dd_add_is_accurate_on_cancelling_terms():
    # relative error <= 3 u^2 of the exact sum (u = 2^-53), also when the highs cancel
    from fractions import Fraction
    rng = np.random.default_rng(5)
    cases = [((1.0, 1e-17, 1.0), (-1.0, 2e-17, 1.0))]
    for _ in range(2000):
        ah = rng.uniform(-1, 1)
        al = ah * rng.uniform(-1, 1) * 2.0 ** -53
        bh = -ah * (1 + rng.uniform(-1, 1) * 2.0 ** -rng.integers(1, 60))
        bl = bh * rng.uniform(-1, 1) * 2.0 ** -53
        cases.append(((ah, al, 1.0), (bh, bl, 1.0)))
    for a, b in cases:
        h, lo, ab = shard.dd_add(a, b)
        exact = sum(Fraction(v) for v in (a[0], a[1], b[0], b[1]))
        assert abs(Fraction(h) + Fraction(lo) - exact) <= 3 * Fraction(2) ** -106 * abs(exact)
        assert abs(lo) <= abs(h) * 2.0 ** -53 and ab == 2.0


def test_two_ranks_gloo_match_single_process(oracle_mod, tmp_path):
    import socket

    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0 = tuple(np.load(tmp_path / "r0.npy"))
    r1 = tuple(np.load(tmp_path / "r1.npy"))
    assert r0 == r1
    O = inputs.lossy_squeezed(N, 1234, (0.5, 1.2), 0.4).O
    single = shard.tree_merge([task_partial(oracle_mod, O, t) for t in range(1 << (P - 5))])
    assert r0 == tuple(single)
    full = oracle_mod.tor_brute(O)
    assert abs((r0[0] - full.hi) + (r0[1] - full.lo)) <= 1e-25 * full.abs_sum


def test_partition_batch_balances_cost():
    ns = [20, 3, 18, 18, 12, 20, 5, 19]
    parts = shard.partition_batch(ns, 3)
    assert sorted(i for p in parts for i in p) == list(range(len(ns)))
    loads = [sum(1 << ns[i] for i in p) for p in parts]
    assert max(loads) <= 2 ** 20 + 2 ** 19  # LPT: the two n=20 on different ranks
    assert shard.partition_batch(ns, 3) == parts  # deterministic
    assert shard.partition_batch(ns, 1) == [list(range(len(ns)))]


def _batch_rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mats = [inputs.lossy_squeezed(n, 300 + i, (0.5, 1.2), 0.4).O for i, n in enumerate(BATCH_NS)]

    def evaluate(idx):
        return [(r.hi, r.lo, r.abs_sum) for r in (oracle.tor_brute(mats[i], threads=1) for i in idx)]
    out = shard.distributed_batch(evaluate, BATCH_NS)
    np.save(os.path.join(out_dir, f"b{rank}.npy"), np.array(out))
    dist.barrier()
    dist.destroy_process_group()


BATCH_NS = [6, 2, 7, 4, 7, 1, 5]


def test_batch_two_ranks_gloo_match_single_process(oracle_mod, tmp_path):
    import socket

    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mp.start_processes(_batch_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    b0, b1 = np.load(tmp_path / "b0.npy"), np.load(tmp_path / "b1.npy")
    assert np.array_equal(b0, b1)
    for i, n in enumerate(BATCH_NS):
        r = oracle_mod.tor_brute(inputs.lossy_squeezed(n, 300 + i, (0.5, 1.2), 0.4).O, threads=1)
        assert tuple(b0[i]) == (r.hi, r.lo, r.abs_sum)


def _bench_rank_main(rank, world, port, out_dir):
    import sys

    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    class Args:
        impl = "reference"  # the reference arm's rendezvous uses gloo
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    w, r, local = bench.dist_setup(Args())
    bench.barrier(w)
    got = bench.max_over_ranks(w, 10.0 + r, "cpu")  # each rank's time; the job's is the slowest
    np.save(os.path.join(out_dir, f"m{rank}.npy"), np.array([w, r, local, got]))
    bench.barrier(w)
    dist.destroy_process_group()


def test_bench_rank_helpers_gloo(tmp_path):
    # the bench's multi-rank plumbing (rendezvous, barrier, max over ranks) on two CPU ranks
    import socket

    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mp.start_processes(_bench_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for rank in range(2):
        w, r, local, got = np.load(tmp_path / f"m{rank}.npy")
        assert (w, r, local, got) == (2, rank, rank, 11.0)


def _failing_rank_main(rank, world, port, out_dir):
    import datetime

    import torch.distributed as dist

    from paper_2109_04528_gb300 import binding
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    seen = []

    def evaluate_batch(idx):  # rank 1's evaluation fails on the host, before the collective
        if rank == 1:
            raise binding.TorError(binding.TOR_ETIMEOUT, "planted")
        return [(1.0, 0.0, 1.0) for _ in idx]

    def evaluate_partial():
        if rank == 0:
            raise binding.TorError(binding.TOR_ENOTPD, "planted")
        return (1.0, 0.0, 1.0)
    for call in (lambda: shard.distributed_batch(evaluate_batch, [3, 4, 5, 6]),
                 lambda: shard.distributed_partial(evaluate_partial)):
        try:
            call()
            seen.append(0)
        except binding.TorError as e:
            seen.append(e.status)
    # the ranks are still in step: a plain merge afterwards works on both
    merged = shard.gather_merge((float(rank), 0.0, 1.0))
    np.save(os.path.join(out_dir, f"f{rank}.npy"), np.array(seen + list(merged)))
    dist.barrier()
    dist.destroy_process_group()


def test_failure_on_one_rank_raises_on_every_rank(tmp_path):
    # a rank whose evaluation fails still joins the gather, and then every rank raises
    # the failure (no rank is left waiting in the collective)
    import socket

    import torch.multiprocessing as mp

    from paper_2109_04528_gb300 import binding
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mp.start_processes(_failing_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for rank in range(2):
        got = np.load(tmp_path / f"f{rank}.npy")
        assert tuple(got[:2]) == (binding.TOR_ETIMEOUT, binding.TOR_ENOTPD)
        assert tuple(got[2:]) == (1.0, 0.0, 2.0)


MANY = [(9, 6, 1234), (10, 7, 77)]  # (n, p, seed): 2 and 4 reduction leaves


class _Res:
    def __init__(self, t, status=0):
        (self.hi, self.lo, self.abs_sum), self.status = t, status


def _many_rank_main(rank, world, port, out_dir, fail_rank):
    import torch.distributed as dist

    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    depth = {n: p for n, p, _ in MANY}
    calls = []

    def eval_range_batch(ctx, mats, ranges, check=True):  # the device's leaf sums, from the oracle
        calls.append(list(ranges))
        out = []
        for O, (lo, cnt) in zip(mats, ranges):
            p = depth[O.shape[0] // 2]
            out.append(_Res(shard.tree_merge([task_partial(oracle, O, t, p) for t in range(lo, lo + cnt)]),
                            binding.TOR_ENOTPD if rank == fail_rank else 0))
        return out
    binding.tor_plan_leaves = lambda ctx, n: 1 << (depth[n] - 5)
    binding.tor_eval_range_batch = eval_range_batch
    mats = [inputs.lossy_squeezed(n, seed, (0.5, 1.2), 0.4).O for n, _, seed in MANY]
    try:
        got = shard.distributed_tor_many(None, mats)
        status = 0
    except binding.TorError as e:
        got, status = [(0.0, 0.0, 0.0)] * len(mats), e.status
    np.save(os.path.join(out_dir, f"many{rank}.npy"),
            np.array([list(g) for g in got] + [[status, len(calls), calls[0][1][0]]]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("fail_rank", [-1, 1])
def test_many_matrices_sharded_in_one_launch_per_rank(oracle_mod, tmp_path, fail_rank):
    # distributed_tor_many on two gloo ranks: one range call per rank covering every
    # matrix; the merged results equal the single-process tree of all leaves bitwise
    # and the oracle's full sum; a failed result on one rank raises on both
    import socket

    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mp.start_processes(_many_rank_main, args=(2, port, str(tmp_path), fail_rank), nprocs=2, join=True,
                       start_method="spawn")
    rows = [np.load(tmp_path / f"many{r}.npy") for r in range(2)]
    for rank, got in enumerate(rows):
        status, ncalls, lo1 = got[-1]
        assert ncalls == 1 and lo1 == rank * 2  # the n = 10 matrix's 4 leaves: 2 per rank
        if fail_rank >= 0:
            assert status == binding.TOR_ENOTPD
            continue
        assert status == 0
        for (n, p, seed), g in zip(MANY, got[:-1]):
            O = inputs.lossy_squeezed(n, seed, (0.5, 1.2), 0.4).O
            single = shard.tree_merge([task_partial(oracle_mod, O, t, p) for t in range(1 << (p - 5))])
            assert tuple(g) == tuple(single)
            full = oracle_mod.tor_brute(O)
            assert abs((g[0] - full.hi) + (g[1] - full.lo)) <= 1e-25 * full.abs_sum
