"""Pins of the oracle's joint solve across levels (composite grid over 2:1 faces).

The paper does not print the octree operators; the reading is in oracle/composite.py.
Pins: on one level the composite operators and iteration equal the single-level
oracle (independent C code); constants are in the null space; the rows at a
2:1 face by hand; ||K||^2 by power iteration against a dense eigenvalue; the
step sizes satisfy tau sigma ||K||^2 < 1.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle.composite import Composite


def ragged(seed, n=4, drop=0.2):
    rng = np.random.default_rng(seed)
    box = synth.dense_bricks(n)
    return box[rng.random(len(box)) > drop]


def test_single_level_operators_equal_the_level_oracle():
    b = ragged(1)
    C = Composite([b], 8)
    fwd, bwd = oracle.links(b)
    rng = np.random.default_rng(2)
    u = rng.normal(size=C.n)
    v = rng.normal(size=(C.n, 3))
    p = rng.normal(size=(C.n, 3))
    q = rng.normal(size=(C.n, 6))
    zu, zv = np.zeros(1), np.zeros(3)
    np.testing.assert_allclose(C.grad(u), oracle.grad(fwd, u, zu), atol=1e-12)
    np.testing.assert_allclose(C.symgrad(v), oracle.symgrad(bwd, v, zv), atol=1e-12)
    np.testing.assert_allclose(C.div1(p), oracle.div1(fwd, bwd, p), atol=1e-12)
    np.testing.assert_allclose(C.div2(q), oracle.div2(fwd, bwd, q), atol=1e-12)


def test_single_level_iteration_equals_the_level_oracle():
    b = ragged(3, n=3)
    desc = synth.DomainDesc(np.zeros(3), 1.0, b)
    hist = synth.random_histograms(np.random.default_rng(4), desc.nvox, 8, max_count=12)
    lvl = oracle.OracleLevel(desc, 8)
    lvl.hist[:] = hist
    lvl.iterate(25)
    C = Composite([b], 8)
    C.set_level_histograms(0, hist)
    C.iterate(25)
    np.testing.assert_allclose(C.u, lvl.u, atol=1e-11)


def two_levels():
    coarse = synth.dense_bricks(2)                    # coarse voxels 0..15
    fine = synth.dense_bricks(2, offset=(1, 1, 1))    # refines coarse voxels 4..11
    return [coarse, fine]


def test_constants_have_zero_gradient_and_symmetric_gradient():
    C = Composite(two_levels(), 8)
    one = np.ones(C.n)
    assert np.max(np.abs(C.grad(3.0 * one))) < 1e-12
    v = np.tile([0.5, -2.0, 1.0], (C.n, 1))
    assert np.max(np.abs(C.symgrad(v))) < 1e-12


def test_rows_at_a_two_to_one_face_by_hand():
    C = Composite(two_levels(), 8)
    # coarse leaf (3, 5, 6): its +x neighbour (4, 5, 6) is refined -> the 4 fine voxels
    # (8, 10..11, 12..13) with weight 1/4 each, and -1 on itself
    i = C.index[(0, 3, 5, 6)]
    row = C.G[0].getrow(i)
    want = {C.index[(1, 8, y, z)]: 0.25 for y in (10, 11) for z in (12, 13)}
    want[i] = -1.0
    assert dict(zip(row.indices.tolist(), row.data.tolist())) == want
    # fine leaf (8, 10, 12): its -x neighbour is the coarse leaf (3, 5, 6)
    j = C.index[(1, 8, 10, 12)]
    rowb = C.B[0].getrow(j)
    assert dict(zip(rowb.indices.tolist(), rowb.data.tolist())) == {j: 1.0, i: -1.0}
    # a fine leaf on the outer face of the fine region has no same-level +x voxel at
    # x = 24: its +x neighbour is the coarse leaf (12, 5, 6)
    k = C.index[(1, 23, 10, 12)]
    rowf = C.G[0].getrow(k)
    assert dict(zip(rowf.indices.tolist(), rowf.data.tolist())) == {k: -1.0, C.index[(0, 12, 5, 6)]: 1.0}


def test_power_iteration_matches_the_dense_norm_and_step_sizes_are_safe():
    tiny = Composite([synth.dense_bricks(1), np.array([[0, 0, 0]], np.int32)], 4)
    n = tiny.n
    cols = []
    for k in range(4 * n):
        x = np.zeros(4 * n)
        x[k] = 1.0
        u, v = x[:n], x[n:].reshape(n, 3)
        g = tiny.grad(u) - v
        e = tiny.symgrad(v)
        cols.append(np.concatenate([g.ravel(), e[:, :3].ravel(), np.sqrt(2.0) * e[:, 3:].ravel()]))
    K = np.stack(cols, 1)
    dense = float(np.linalg.eigvalsh(K.T @ K)[-1])
    assert tiny.op_norm2(iters=2000) == pytest.approx(dense, rel=1e-6)
    three = Composite([synth.dense_bricks(2), synth.dense_bricks(2, offset=(1, 1, 1)),
                       synth.dense_bricks(2, offset=(3, 3, 3))], 8)
    assert 0.2 * 0.2 * three.op_norm2() < 1.0
