"""Host logic of the batching module (no GPU): scene sizes and grouping."""
import math

from paper_2605_04509_gb300 import batching


def test_scene_sizes_are_seeded_and_log_uniform_in_range():
    a = batching.scene_sizes(16)
    assert a == batching.scene_sizes(16)
    assert all(200_000 <= m <= 3_000_000 for m in a)
    small = batching.scene_sizes(16, 20_000, 100_000)
    assert all(20_000 <= m <= 100_000 for m in small)
    # the same seeds give the same position in the log range
    for m, n in zip(a, small):
        u1 = (math.log(m) - math.log(200_000)) / (math.log(3_000_000) - math.log(200_000))
        u2 = (math.log(n) - math.log(20_000)) / (math.log(100_000) - math.log(20_000))
        assert abs(u1 - u2) < 1e-4


def test_groups_respect_pair_and_scene_limits():
    assert batching.group_scenes([5, 5, 5], max_pairs=10) == [[0, 1], [2]]
    assert batching.group_scenes([10, 1], max_pairs=10) == [[0], [1]]
    assert batching.group_scenes([20, 1], max_pairs=10) == [[0], [1]]  # alone above the limit
    assert batching.group_scenes([1] * 20, max_pairs=100, max_scenes=16) == [list(range(16)),
                                                                              list(range(16, 20))]
    assert batching.group_scenes([]) == []
    groups = batching.group_scenes([3] * 7, max_pairs=7)
    assert [s for g in groups for s in g] == list(range(7))
    assert all(sum(3 for _ in g) <= 7 for g in groups)
