"""Property tests of the host-side sharding arithmetic (CPU; hypothesis).

The batch partition must place every matrix exactly once and stay within the
longest-processing-time bound; the host merge of shard partials must be the
same binary tree and double-word addition whatever the values, accurate to
double-double rounding of the exact sum; the leaf ranges of 2^s ranks must
tile the leaves."""
from fractions import Fraction

import pytest

from paper_2109_04528_gb300 import shard

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings = hyp.given, hyp.settings


@settings(max_examples=200, deadline=None)
@given(st.lists(st.integers(1, 30), min_size=0, max_size=60), st.integers(1, 9))
def test_partition_places_every_matrix_once_within_the_lpt_bound(ns, world):
    parts = shard.partition_batch(ns, world)
    assert len(parts) == world
    assert sorted(i for p in parts for i in p) == list(range(len(ns)))
    assert all(p == sorted(p) for p in parts)
    assert shard.partition_batch(ns, world) == parts
    loads = [sum(1 << ns[i] for i in p) for p in parts]
    if ns:
        # greedy largest-first: no rank exceeds the average load by more than the largest matrix
        assert max(loads) <= sum(loads) / world + max(1 << n for n in ns)


@settings(max_examples=200, deadline=None)
@given(st.integers(0, 6), st.data())
def test_tree_merge_is_accurate_and_ordered(log_parts, data):
    k = 1 << log_parts
    vals = data.draw(st.lists(st.floats(-1e6, 1e6, allow_nan=False, width=64), min_size=k, max_size=k))
    parts = [(v, 0.0, abs(v)) for v in vals]
    h, lo, ab = shard.tree_merge(parts)
    exact = sum(Fraction(v) for v in vals)
    scale = sum(Fraction(abs(v)) for v in vals)
    # each double-word addition errs by <= 3 u^2 of its result; log2(k) levels
    assert abs(Fraction(h) + Fraction(lo) - exact) <= (log_parts + 1) * 3 * Fraction(2) ** -106 * scale
    assert abs(lo) <= abs(h) * 2.0 ** -53 or h == 0.0
    assert shard.tree_merge(parts) == (h, lo, ab)  # the same operations every time


@settings(max_examples=100, deadline=None)
@given(st.integers(0, 12), st.integers(0, 12))
def test_leaf_ranges_tile_the_leaves(log_leaves, log_world):
    leaves, world = 1 << log_leaves, 1 << log_world
    if world > leaves:
        with pytest.raises(ValueError):
            shard.shard_range(leaves, world, 0)
        return
    got = [shard.shard_range(leaves, world, r) for r in range(world)]
    assert got[0][0] == 0 and all(c == leaves // world for _, c in got)
    assert all(got[r][0] + got[r][1] == got[r + 1][0] for r in range(world - 1))
    assert got[-1][0] + got[-1][1] == leaves
