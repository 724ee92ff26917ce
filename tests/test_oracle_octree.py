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


# ---- spherical maps (LIDAR scans): the own sin / cos and the unprojection

def test_sincos_against_the_library_and_by_hand():
    x = np.linspace(-3.3, 3.3, 100001).astype(np.float32)
    s, c = oracle.sincos_tay(x)
    assert np.abs(s - np.sin(x.astype(np.float64))).max() < 1.2e-7
    assert np.abs(c - np.cos(x.astype(np.float64))).max() < 1.2e-7
    s, c = oracle.sincos_tay(np.array([0.0, np.float32(math.pi)], np.float32))
    assert s[0] == 0.0 and c[0] == 1.0 and c[1] == -1.0
    # sin of the float nearest pi is pi - float(pi) (to FP32)
    assert s[1] == np.float32(math.pi - float(np.float32(math.pi)))
    # odd and even, quadrant by quadrant
    y = np.float32([0.3, 1.9, 2.7])
    s1, c1 = oracle.sincos_tay(y)
    s2, c2 = oracle.sincos_tay(-y)
    np.testing.assert_array_equal(s1, -s2)
    np.testing.assert_array_equal(c1, c2)


def test_spherical_sample_by_hand():
    """Scanner at (0.5, 0.5, 0.5), world axes, 8 pixels per radian, range 0.25
    everywhere: pixel (8, 4) looks along +x (azimuth 0, elevation 0), so X =
    (0.75, 0.5, 0.5); its 4 neighbours are 1/8 rad away, r = 0.25 sin(1/16) and
    Eq. 4 gives depth 5 (2^-5 / 2 < 1.5 r <= 2^-4 / 2): cube (24, 16, 16)."""
    cam = synth.Camera(8.0, 8.0, 8.5, 4.5, np.eye(3), np.array([0.5, 0.5, 0.5]), 16, 8, model=1)
    dep = np.full((8, 16), 0.25, np.float32)
    dd, qq, rr = oracle.octree_samples(cam, dep, np.zeros(3), 1.0, 3, 8)
    r = 0.25 * math.sin(1.0 / 16.0)
    assert abs(rr[4, 8] - r) < 1e-7
    assert 0.5 * 2.0 ** -5 < 1.5 * r <= 0.5 * 2.0 ** -4
    assert dd[4, 8] == 5
    assert list(qq[4, 8]) == [24, 16, 16]


def test_spherical_scan_from_inside_a_sphere():
    """A full scan from the centre of a sphere of radius 0.3: every sample's cube lies on
    the sphere (its centre within half a cube diagonal plus the sample radius)."""
    C = np.array([0.5, 0.5, 0.5])
    cam = synth.spherical_scanner(C, 256, 128)
    dep = np.full((128, 256), 0.3, np.float32)
    dd, qq, rr = oracle.octree_samples(cam, dep, np.zeros(3), 1.0, 3, 10)
    ok = dd >= 0
    assert ok.all()
    edge = 2.0 ** -dd[ok].astype(np.float64)
    centre = (qq[ok] + 0.5) * edge[:, None]
    dist = np.linalg.norm(centre - C, axis=1)
    assert np.all(np.abs(dist - 0.3) <= 0.5 * math.sqrt(3) * edge + 1e-6)
    # Eq. 4: the cube radius lies in [0.75 r, 1.5 r) wherever the depth range allows
    inner = (dd[ok] > 3) & (dd[ok] < 10)
    rc = 0.5 * edge[inner]
    assert np.all((0.75 * rr[ok][inner] <= rc) & (rc < 1.5 * rr[ok][inner]))
