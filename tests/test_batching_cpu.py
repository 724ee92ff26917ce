"""Host logic of the grouped batched form: chunks packed into union levels of bounded size."""
import numpy as np

from paper_2107_14790_b300.batching import GROUP_VOXELS, group_chunks


def test_groups_cover_every_chunk_in_order_within_the_budget():
    rng = np.random.default_rng(3)
    sizes = [int(x) for x in np.exp(rng.uniform(np.log(32 ** 3), np.log(192 ** 3), 200))]
    groups = group_chunks(sizes, 12 << 20)
    assert [k for g in groups for k in g] == list(range(len(sizes)))
    for g in groups:
        tot = sum(sizes[k] for k in g)
        assert tot <= 12 << 20 or len(g) == 1
    # greedy: the next group's first chunk did not fit into the previous group
    for g, h in zip(groups, groups[1:]):
        assert sum(sizes[k] for k in g) + sizes[h[0]] > 12 << 20


def test_oversized_chunk_alone_and_no_budget_means_one_group():
    assert group_chunks([5, 5, 5, 20, 1, 1], 10) == [[0, 1], [2], [3], [4, 5]]
    assert group_chunks([3, 4, 5], 0) == [[0, 1, 2]]
    assert group_chunks([], 10) == []
    assert GROUP_VOXELS > 0
