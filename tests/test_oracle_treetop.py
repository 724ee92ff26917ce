"""Pins of the oracle's treetop (Sec. 4.3): the smallest rooted subtree whose leaf nodes
hold fewer than N leaf cubes each, with the first and last Z-ordered cube of each.

Hand cases: one dense brick (its Z-order is the Morton order of the voxels, so part
boundaries fall at multiples of 8^k); two levels with a refined octant, whose parts are
derived by hand.  Brute force on random nested levels: the parts tile the Z-ordered
cubes, each holds fewer than N, and each part's parent node holds at least N (the
treetop is minimal).
"""
import numpy as np
import pytest

import synth
from oracle.composite import Composite, leaf_keys, morton_code, treetop


def one_brick():
    return Composite([np.array([[0, 0, 0]])], 8)


def test_morton_code_by_hand():
    assert morton_code([1], [0], [0], 3)[0] == 1
    assert morton_code([0], [1], [0], 3)[0] == 2
    assert morton_code([0], [0], [1], 3)[0] == 4
    assert morton_code([2], [0], [0], 3)[0] == 8
    assert morton_code([7], [7], [7], 3)[0] == 511
    # x = 011, y = 101, z = 110: bit triples (z y x) 011, 101, 110 from the lowest
    assert morton_code([3], [5], [6], 3)[0] == 3 + (5 << 3) + (6 << 6)


@pytest.mark.parametrize("N,depth,size", [(513, 0, 512), (512, 1, 64), (64, 2, 8), (9, 2, 8), (8, 3, 1), (2, 3, 1)])
def test_one_dense_brick(N, depth, size):
    C = one_brick()
    d, c, f, l, p = treetop(C.keys, 1, 3, N)
    k = 512 // size
    assert len(d) == k and np.all(d == depth)
    np.testing.assert_array_equal(c, np.arange(k))
    np.testing.assert_array_equal(f, size * np.arange(k))
    np.testing.assert_array_equal(l, size * np.arange(k) + size - 1)
    # leaf order is local voxel order x + 8 y + 64 z; the voxel (3, 5, 6) has Morton code 427
    i = 3 + 8 * 5 + 64 * 6
    assert p[i] == 427 // size


def test_two_levels_by_hand():
    """Level 0: brick (0,0,0) (edge 2 in finest units); level 1: brick (0,0,0), which
    refines the level-0 octant [0,4)^3.  Root [0,16)^3 (root_bits 4); 448 + 512 cubes."""
    C = Composite([np.array([[0, 0, 0]]), np.array([[0, 0, 0]])], 8)
    assert C.n == 960
    # N = 600: the root splits; octant 0 holds the 512 fine cubes, octants 1..7 64 coarse each
    d, c, f, l, p = treetop(C.keys, 2, 4, 600)
    np.testing.assert_array_equal(d, [1] * 8)
    np.testing.assert_array_equal(c, np.arange(8))
    np.testing.assert_array_equal(f, [0] + [512 + 64 * j for j in range(7)])
    np.testing.assert_array_equal(l, [511] + [575 + 64 * j for j in range(7)])
    # N = 100: octant 0 splits once more into 8 nodes of 64 fine cubes
    d, c, f, l, p = treetop(C.keys, 2, 4, 100)
    np.testing.assert_array_equal(d, [2] * 8 + [1] * 7)
    np.testing.assert_array_equal(c, list(range(8)) + list(range(1, 8)))
    np.testing.assert_array_equal(f, 64 * np.arange(15))
    assert p[C.keys.index((0, 4, 0, 0))] == 8     # corner (8, 0, 0): octant 1
    assert p[C.keys.index((0, 0, 4, 4))] == 13    # corner (0, 8, 8): octant 6
    assert p[C.keys.index((1, 0, 0, 0))] == 0
    assert p[C.keys.index((1, 7, 7, 7))] == 7     # corner (7, 7, 7): octant 0, its octant 7
    assert p[C.keys.index((1, 4, 0, 0))] == 1
    # N above the total: the root is the one part
    d, c, f, l, p = treetop(C.keys, 2, 4, 961)
    assert list(d) == [0] and list(f) == [0] and list(l) == [959] and np.all(p == 0)


def nested_levels(seed, nbox=3):
    rng = np.random.default_rng(seed)
    box = synth.dense_bricks(nbox)
    l0 = box[rng.random(len(box)) > 0.3]
    kids = (2 * l0[:, None, :] + synth.dense_bricks(2)[None]).reshape(-1, 3)
    l1 = kids[rng.random(len(kids)) > 0.75]
    kids = (2 * l1[:, None, :] + synth.dense_bricks(2)[None]).reshape(-1, 3)
    l2 = kids[rng.random(len(kids)) > 0.8]
    return [l0, l1, l2]


def node_count(corner, depth, code, root_bits):
    """Cubes whose lower corner lies in the node (depth, code), by brute force."""
    lo = np.zeros(3, np.int64)
    for k in range(depth):
        ch = (int(code) >> (3 * (depth - 1 - k))) & 7
        half = 1 << (root_bits - k - 1)
        lo += half * np.array([ch & 1, (ch >> 1) & 1, ch >> 2])
    edge = 1 << (root_bits - depth)
    return int(np.sum(np.all((corner >= lo) & (corner < lo + edge), axis=1)))


@pytest.mark.parametrize("seed,N,nbox", [(1, 2, 1), (1, 50, 2), (2, 700, 3), (3, 4000, 3), (4, 10 ** 6, 3)])
def test_random_nested_levels_brute_force(seed, N, nbox):
    keys = leaf_keys(nested_levels(seed, nbox))
    n = len(keys)
    root_bits = 5 + 2  # level-0 bricks in [0, 3): voxels < 24 < 32; finest = 4x
    d, c, f, l, p = treetop(keys, 3, root_bits, N)
    k = np.array(keys, np.int64)
    corner = k[:, 1:] << (2 - k[:, 0])[:, None]
    z = morton_code(corner[:, 0], corner[:, 1], corner[:, 2], root_bits)
    order = np.argsort(z)
    # the parts tile the Z-ordered cubes, in order
    assert f[0] == 0 and l[-1] == n - 1
    np.testing.assert_array_equal(f[1:], l[:-1] + 1)
    rng = np.random.default_rng(seed)
    sample = range(len(d)) if len(d) <= 150 else rng.choice(len(d), 150, replace=False)
    assert np.all(l - f + 1 < N)
    for j in sample:
        cnt = l[j] - f[j] + 1
        assert cnt < N
        assert node_count(corner, d[j], c[j], root_bits) == cnt
        assert np.all(p[order[f[j]:l[j] + 1]] == j)
        if d[j] > 0:
            assert node_count(corner, d[j] - 1, int(c[j]) >> 3, root_bits) >= N
        # every cube of the part carries the part's code in its top bits
        top = z[order[f[j]:l[j] + 1]] >> np.uint64(3 * (root_bits - d[j]))
        assert np.all(top == c[j])
    assert np.all(p >= 0)


def test_leaf_keys_are_the_composite_leaves():
    levels = [np.array([[0, 0, 0], [1, 0, 0]]), np.array([[0, 0, 0], [1, 1, 0]])]
    assert leaf_keys(levels) == Composite(levels, 8).keys


def test_cube_outside_the_root_is_rejected():
    C = Composite([np.array([[0, 0, 0]])], 8)
    with pytest.raises(ValueError):
        treetop(C.keys, 1, 2, 10)
    C = Composite([np.array([[-1, 0, 0]])], 8)
    with pytest.raises(ValueError):
        treetop(C.keys, 1, 5, 10)
