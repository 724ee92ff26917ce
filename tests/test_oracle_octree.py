"""Pins of the oracle's octree domain builder (Sec. 3.3 Eq. 4, Sec. 4.1-4.2).

Expected values are worked out by hand on planes seen head-on (dyadic camera,
where FP32 is exact), or are properties the construction must have: the cube
inequality of Eq. 4, containment of each sample, Z-curve order, band, 2:1
nesting and frozen shells.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def plane_cam(W=64, zc=-0.5):
    return synth.Camera(64.0, 64.0, W / 2, W / 2, np.eye(3), np.array([0.5, 0.5, zc]), W, W)


@pytest.mark.parametrize("z,d", [(0.5, 7), (1.0, 6), (2.0, 5)])
def test_eq4_depth_on_planes(z, d):
    """A head-on plane at z-depth z: neighbouring samples z/64 apart, r = z/128; Eq. 4
    with r_root = 1/2 gives the smallest d with 2^-d / 2 < 1.5 r."""
    cam = plane_cam()
    dep = synth.plane_depth(64, 64, z)
    dep[10, 10] = np.nan  # its neighbours keep three valid neighbours: same mean distance
    dd, qq, rr = oracle.octree_samples(cam, dep, np.array([-2.0, -2.0, -2.0]), 4.0, 3, 12)
    ok = dd >= 0
    assert ok.sum() == 64 * 64 - 1
    assert np.all(rr[ok] == np.float32(z / 128))
    # root edge 4: r_root = 2 -> smallest d with 2 * 2^-d < 1.5 z / 128
    want = next(k for k in range(3, 13) if 2 * 2.0 ** -k < 1.5 * z / 128)
    assert np.all(dd[ok] == want)
    assert 0.75 * z / 128 <= 2 * 2.0 ** -want < 1.5 * z / 128


def test_cube_coordinates_by_hand():
    """Camera at (0.5, 0.5, -0.5) looking along +z at a plane of z-depth 1 (world z 0.5),
    root [0, 1)^3: pixel (i, j) lands at x = 0.5 + (i + 0.5 - 32) / 64, depth 6."""
    dd, qq, _ = oracle.octree_samples(plane_cam(), synth.plane_depth(64, 64, 1.0), np.zeros(3), 1.0, 3, 9)
    assert np.all(dd == 6)
    for i, j in [(0, 0), (31, 7), (32, 32), (63, 63)]:
        x = 0.5 + (i + 0.5 - 32) / 64
        y = 0.5 + (j + 0.5 - 32) / 64
        assert list(qq[j, i]) == [math.floor(x * 64), math.floor(y * 64), 32]


def test_plane_levels_by_hand():
    """Depth 6 bricks of the plane: x, y in 0..7, z = 4 (64); band 1 -> z 3..5 (192), frozen
    z = 2 and 6 (128); depth 5 gains the parents (z 1..2) dilated: all 4^3 = 64; depth 4:
    all 8; depth 3: the single brick; depth 7: nothing."""
    levels, ns = oracle.octree_build([plane_cam()], [synth.plane_depth(64, 64, 1.0)], np.zeros(3), 1.0, 3, 7, band=1)
    assert ns == 64 * 64
    assert [(a.shape[0], f.shape[0]) for a, f in levels] == [(1, 0), (8, 0), (64, 0), (192, 128), (0, 0)]
    a3, f3 = levels[3]
    assert set(np.unique(a3[:, 2])) == {3, 4, 5} and set(np.unique(f3[:, 2])) == {2, 6}


def morton(c):
    k = 0
    for b in range(21):
        for a in range(3):
            k |= ((int(c[a]) >> b) & 1) << (3 * b + a)
    return k


def dilate(s, nbr):
    out = set()
    for (x, y, z) in s:
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    p = (x + dx, y + dy, z + dz)
                    if all(0 <= v < nbr for v in p):
                        out.add(p)
    return out


def test_sphere_scene_construction_properties(sphere_scene):
    sc = sphere_scene
    rm, E, dmin, dmax = np.array([-0.5, -0.5, -0.5]), 2.0, 3, 8
    levels, ns = oracle.octree_build(sc.cameras, sc.depths, rm, E, dmin, dmax, band=1)
    assert ns > 100_000
    occupied = [set() for _ in levels]
    for cam, dep in zip(sc.cameras, sc.depths):
        dd, qq, rr = oracle.octree_samples(cam, dep, rm, E, dmin, dmax)
        ok = dd >= 0
        for d, q, r in zip(dd[ok], qq[ok], rr[ok]):
            cube = E / 2 * 2.0 ** -d
            if dmin < d < dmax:
                assert 0.75 * r * (1 - 1e-6) <= cube < 1.5 * r * (1 + 1e-6)
            occupied[d - dmin].add(tuple(int(v) >> 3 for v in q))
    for l, (act, frz) in enumerate(levels):
        nbr = max((1 << (dmin + l)) >> 3, 1)
        A = set(map(tuple, act.tolist()))
        F = set(map(tuple, frz.tolist()))
        keys = [morton(c) for c in act.tolist()]
        assert keys == sorted(keys) and len(set(keys)) == len(keys)  # Z-curve order, unique
        assert dilate(occupied[l], nbr) <= A  # band of one ring
        assert not (A & F) and F <= dilate(A, nbr)
        if l > 0:
            assert F == dilate(A, nbr) - A
        if l + 1 < len(levels):
            parents = {(x >> 1, y >> 1, z >> 1) for (x, y, z) in map(tuple, levels[l + 1][0].tolist())}
            assert dilate(parents, nbr) <= A  # 2:1: the finer level is wrapped by this one
