"""Sharding across processes (one per GPU): one Torontonian by leaf ranges,
or a batch of Torontonians by matrices.

The final reduction of tor_eval is a fixed binary tree over the matrix's
reduction leaves (its warp tasks).  A shard evaluates an aligned power-of-two
range of leaves with tor_eval_range; merging the shards' partial sums with the
same tree and the same double-double addition reproduces the single-GPU
result bitwise.  The exchange is one gather of three doubles per rank.
"""
from __future__ import annotations


def shard_range(n_leaves: int, world: int, rank: int):
    """(leaf_lo, leaf_count) of `rank` among `world` ranks (world a power of two <= n_leaves)."""
    if world < 1 or world & (world - 1) or world > n_leaves or not 0 <= rank < world:
        raise ValueError("world must be a power of two no larger than the number of leaves")
    count = n_leaves // world
    return rank * count, count


def two_sum(a: float, b: float):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def fast_two_sum(a: float, b: float):
    s = a + b
    return s, b - (s - a)


def dd_add(x, y):
    """(hi, lo, abs) + (hi, lo, abs).  The double-double sum is the accurate
    double-word addition (Joldes, Muller, Popescu, ACM TOMS 44 (2017),
    AccurateDWPlusDW), the same operations in the same order as the device."""
    s, e = two_sum(x[0], y[0])
    t, f = two_sum(x[1], y[1])
    s, e = fast_two_sum(s, e + t)
    h, lo = fast_two_sum(s, e + f)
    return (h, lo, x[2] + y[2])


def tree_merge(parts):
    """Binary-tree sum of a power-of-two list of (hi, lo, abs), left operand first."""
    parts = list(parts)
    if not parts or len(parts) & (len(parts) - 1):
        raise ValueError("need a power-of-two number of parts")
    while len(parts) > 1:
        parts = [dd_add(parts[i], parts[i + 1]) for i in range(0, len(parts), 2)]
    return parts[0]


def partition_batch(ns, world: int):
    """Splits a batch of matrices with n_i modes over `world` ranks by cost
    2^n_i: largest first, each to the rank with the least work so far (lowest
    rank on ties).  Returns one list of batch indices per rank, each in
    ascending order.  Deterministic, so every rank computes the same split."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(ns)), key=lambda i: (-ns[i], i)):
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += 1 << ns[i]
    return [sorted(p) for p in parts]


def _gather_checked(work, group=None):
    """Runs work() on this rank and all-gathers (status, message, value) from every
    rank.  A rank whose work fails (a TorError such as ETIMEOUT or ENOTPD, or any
    other exception) still joins the collective, so no rank is left blocked in it;
    afterwards every rank raises the first failure, by rank order.  Returns the
    gathered values in rank order."""
    import torch.distributed as dist

    from .binding import TorError
    world = dist.get_world_size(group)
    try:
        item = (0, "", work())
    except TorError as e:
        item = (int(e.status), str(e), None)
    except Exception as e:  # reported to every rank below, then raised there
        item = (-1, f"{type(e).__name__}: {e}", None)
    got = [None] * world
    dist.all_gather_object(got, item, group=group)
    for r, (status, msg, _) in enumerate(got):
        if status:
            raise TorError(status if status > 0 else 1, f"rank {r} failed: {msg}")
    return [v for _, _, v in got]


def distributed_batch(evaluate, ns, group=None):
    """Evaluates a batch split by partition_batch: `evaluate(indices)` returns
    this rank's (hi, lo, abs) per index; one all-gather returns every rank the
    whole batch's results in batch order.  A matrix's result does not depend
    on the batch it is evaluated in, so this equals one rank's tor_eval_batch.
    If any rank's evaluation fails, every rank raises after the gather."""
    import torch.distributed as dist
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    mine = partition_batch(ns, world)[rank]

    def work():
        got = evaluate(mine)
        return [(i, tuple(float(v) for v in r)) for i, r in zip(mine, got)]
    out = [None] * len(ns)
    for rows_r in _gather_checked(work, group):
        for i, r in rows_r:
            out[i] = r
    return out


def gather_merge(partial, group=None):
    """All-gather each rank's (hi, lo, abs) (torch.distributed) and merge in rank order."""
    return distributed_partial(lambda: partial, group)


def distributed_partial(evaluate, group=None):
    """`evaluate()` gives this rank's (hi, lo, abs); all-gathers them and merges in
    rank order.  If any rank's evaluation fails, every rank raises after the gather."""
    got = _gather_checked(lambda: tuple(float(v) for v in evaluate()), group)
    return tree_merge(got)


def distributed_tor_batch(ctx, mats, group=None):
    """tor_eval_batch of `mats` with the matrices split over the ranks of `group`."""
    from . import binding
    ns = [m.shape[0] // 2 for m in mats]

    def evaluate(idx):
        res = binding.tor_eval_batch(ctx, [mats[i] for i in idx]) if idx else []
        for r in res:
            if r.status != binding.TOR_OK:
                raise binding.TorError(r.status, "tor_eval_batch")
        return [(r.hi, r.lo, r.abs_sum) for r in res]
    return distributed_batch(evaluate, ns, group)


def distributed_tor_many(ctx, mats, group=None):
    """Tor of each of several matrices with every matrix's leaves split over the
    ranks of `group` (strong scaling, paper Sec. 4): each rank evaluates its
    aligned leaf range of every matrix in one launch (tor_eval_range_batch), so
    one matrix's tail shares the GPU with the others' tasks; one gather of three
    doubles per matrix and rank, then the fixed tree.  Every rank gets the merged
    (hi, lo, abs) per matrix, equal bitwise to tor_eval of each matrix alone.
    If any rank's evaluation fails, every rank raises after the gather."""
    import torch.distributed as dist

    from . import binding
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    ranges = [shard_range(binding.tor_plan_leaves(ctx, m.shape[0] // 2), world, rank) for m in mats]

    def evaluate():
        res = binding.tor_eval_range_batch(ctx, mats, ranges, check=False)
        for r in res:
            if r.status != binding.TOR_OK:
                raise binding.TorError(r.status, "tor_eval_range_batch")
        return [(r.hi, r.lo, r.abs_sum) for r in res]
    got = _gather_checked(evaluate, group)
    return [tree_merge([g[i] for g in got]) for i in range(len(mats))]


def distributed_tor(ctx, O, group=None):
    """Tor of one matrix with its leaves split over the ranks of `group`; every rank
    gets the merged (hi, lo, abs)."""
    import torch.distributed as dist

    from . import binding
    n = O.shape[0] // 2
    lo, count = shard_range(binding.tor_plan_leaves(ctx, n), dist.get_world_size(group), dist.get_rank(group))

    def evaluate():
        r = binding.tor_eval_range(ctx, O, lo, count)
        if r.status != binding.TOR_OK:
            raise binding.TorError(r.status, "tor_eval_range")
        return (r.hi, r.lo, r.abs_sum)
    return distributed_partial(evaluate, group)
