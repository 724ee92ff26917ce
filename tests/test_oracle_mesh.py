"""Pins of the oracle's marching cubes (Sec. 4.6) against hand-worked meshes, closed
forms, topology and brute force; none of the expected values comes from the oracle.

The extraction reads an FP32 indicator u given per voxel (seeded or analytic
fields below): cells of 8 voxel centres, zero crossings by linear interpolation,
per-cell polygons, minimum-area triangulation by dynamic programming.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth


def centres(desc, frozen=False):
    b = desc.frozen if frozen else desc.bricks
    loc = np.arange(512)
    lx, ly, lz = loc & 7, (loc >> 3) & 7, loc >> 6
    g = np.stack([8 * b[:, 0:1] + lx, 8 * b[:, 1:2] + ly, 8 * b[:, 2:3] + lz], -1).reshape(-1, 3)
    return np.asarray(desc.origin) + (g + 0.5) * desc.h, g


def directed_edges(T):
    E = {}
    for t in T:
        for a, c in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])):
            E[(int(a), int(c))] = E.get((int(a), int(c)), 0) + 1
    return E


def closed_oriented(T):
    """Every directed edge once and its reverse once: a closed, consistently oriented surface."""
    E = directed_edges(T)
    return all(k == 1 and E.get((c, a), 0) == 1 for (a, c), k in E.items())


def normals(V, T):
    return np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]]).astype(np.float64)


def one_brick():
    return synth.DomainDesc(np.zeros(3), 1.0 / 8, synth.dense_bricks(1))


def test_single_inside_voxel_is_an_octahedron():
    """u = -1 at voxel (3,3,3), +1 elsewhere: the 8 cells around it each cut off one
    corner at the edge midpoints (t = 1/2): 6 vertices, 8 triangles facing away."""
    d = one_brick()
    X, g = centres(d)
    u = np.ones(512, np.float32)
    u[3 + 8 * 3 + 64 * 3] = -1.0
    V, T = oracle.mesh(d, u)
    assert V.shape == (6, 3) and T.shape == (8, 3)
    c = (np.array([3, 3, 3]) + 0.5) / 8
    want = sorted(tuple(c + s * np.eye(3)[a] / 16) for a in range(3) for s in (-1, 1))
    assert sorted(map(tuple, V.astype(np.float64))) == pytest.approx(want, abs=0)
    assert closed_oriented(T)
    n = normals(V, T)
    assert np.all(np.einsum("ij,ij->i", n, V[T].mean(1) - c) > 0)
    # each face a right isosceles triangle of legs 1/16 * sqrt(2): area 1/512 * ... = (1/16)^2 * sqrt(3)/2
    assert 0.5 * np.linalg.norm(n, axis=1) == pytest.approx(np.full(8, (1 / 16) ** 2 * math.sqrt(3) / 2), rel=1e-6)


def test_plane_closed_form():
    """u = z - c over a 3x2x2-brick block: a flat sheet at z = c spanning the cells'
    x, y extent ((24-1) x (16-1) voxel spacings), normals +z."""
    d = synth.DomainDesc(np.zeros(3), 1.0 / 32, synth.dense_bricks(3, 2, 2))
    X, _ = centres(d)
    c = 0.3 + 1.0 / 1024
    u = (X[:, 2] - c).astype(np.float32)
    V, T = oracle.mesh(d, u)
    assert np.max(np.abs(V[:, 2] - c)) < 2e-6
    n = normals(V, T)
    assert np.all(n[:, 2] > 0) and np.allclose(n[:, :2], 0, atol=1e-7)
    area = 0.5 * n[:, 2].sum()
    assert area == pytest.approx((23 / 32) * (15 / 32), rel=1e-5)


@pytest.mark.parametrize("R", [0.3, 0.21])
def test_sphere_is_a_closed_genus_zero_surface(R):
    d = synth.DomainDesc(np.zeros(3), 1.0 / 40, synth.dense_bricks(5))
    X, _ = centres(d)
    u = (np.linalg.norm(X - 0.5, axis=1) - R).astype(np.float32)
    V, T = oracle.mesh(d, u)
    assert closed_oriented(T)
    E = directed_edges(T)
    assert len(V) - len(E) // 2 + len(T) == 2  # Euler characteristic of a sphere
    n = normals(V, T)
    assert np.all(np.einsum("ij,ij->i", n, V[T].mean(1) - 0.5) > 0)
    assert 0.5 * np.linalg.norm(n, axis=1).sum() == pytest.approx(4 * math.pi * R * R, rel=0.01)
    r = np.linalg.norm(V - 0.5, axis=1)
    assert np.max(np.abs(r - R)) < 0.1 / 40  # linear interpolation of a distance field


def test_torus_has_euler_characteristic_zero():
    d = synth.DomainDesc(np.zeros(3), 1.0 / 48, synth.dense_bricks(6))
    X, _ = centres(d)
    q = np.hypot(X[:, 0] - 0.5, X[:, 1] - 0.5) - 0.28
    u = (np.hypot(q, X[:, 2] - 0.5) - 0.1).astype(np.float32)
    V, T = oracle.mesh(d, u)
    assert closed_oriented(T)
    assert len(V) - len(directed_edges(T)) // 2 + len(T) == 0


@pytest.mark.parametrize("seed,amp", [(3, 1.2), (0, 1.2), (6, 0.6), (2, 2.5), (5, 5.0)])
def test_noisy_field_stays_watertight(seed, amp):
    """A sphere with voxel-scale noise: many faces with four crossings (the face-sum
    rule must agree between the two cells of a face), polygons carrying several of
    them (no triangulation free of in-face chords: centroid fans), and the surface
    is still closed and consistently oriented."""
    rng = np.random.default_rng(seed)
    d = synth.DomainDesc(np.zeros(3), 1.0 / 32, synth.dense_bricks(4))
    X, _ = centres(d)
    u = (np.linalg.norm(X - 0.5, axis=1) - 0.3 + rng.uniform(-1, 1, len(X)) * amp / 32).astype(np.float32)
    V, T = oracle.mesh(d, u)
    assert len(T) > 3000 and closed_oriented(T)
    assert len(np.unique(T)) == len(V)  # every vertex is used


def test_frozen_bricks_give_corners_not_cells():
    """Cells are extracted for active bricks only, with corners read from frozen
    bricks too: an active brick whose +x neighbour is frozen has cells with i = 7."""
    act = np.array([[0, 0, 0]], np.int32)
    frz = np.array([[1, 0, 0]], np.int32)
    d = synth.DomainDesc(np.zeros(3), 1.0 / 16, act, frozen=frz)
    Xa, _ = centres(d)
    Xf, _ = centres(d, frozen=True)
    u = np.concatenate([Xa[:, 0], Xf[:, 0]]) - 0.5  # crossing between voxel x = 7 and x = 8
    V, T = oracle.mesh(d, u.astype(np.float32))
    assert np.allclose(V[:, 0], 0.5, atol=1e-7) and len(T) == 2 * 7 * 7
    d2 = synth.DomainDesc(np.zeros(3), 1.0 / 16, act)
    V2, T2 = oracle.mesh(d2, (Xa[:, 0] - 0.5).astype(np.float32))
    assert len(T2) == 0  # without the frozen brick those cells have missing corners


def _all_triangulations(k):
    """Every triangulation of a convex-indexed polygon 0..k-1 (as sets of (i, m, j))."""
    def rec(i, j):
        if j - i < 2:
            return [[]]
        out = []
        for m in range(i + 1, j):
            for a in rec(i, m):
                for b in rec(m, j):
                    out.append([(i, m, j)] + a + b)
        return out
    return rec(0, k - 1)


@pytest.mark.parametrize("k", [4, 5, 6, 7])
def test_triangulation_is_the_minimum_area_one(k):
    rng = np.random.default_rng(k)
    for _ in range(20):
        ang = np.sort(rng.uniform(0, 2 * math.pi, k))
        P = np.stack([np.cos(ang), np.sin(ang), rng.normal(0, 0.4, k)], 1).astype(np.float32)
        tri = oracle.triangulate_min_area(P)
        assert tri.shape == (k - 2, 3) and np.all(tri[:, 0] < tri[:, 1]) and np.all(tri[:, 1] < tri[:, 2])
        P64 = P.astype(np.float64)

        def area(ts):
            return sum(np.linalg.norm(np.cross(P64[m] - P64[i], P64[j] - P64[i])) for i, m, j in ts)
        best = min(area(t) for t in _all_triangulations(k))
        assert area(tri) == pytest.approx(best, rel=2e-6)
