"""The scatter form of the histogram kernel (one thread per depth-pyramid pixel,
atomic votes; Alg. 1 with the ownership test of Sec. 3.4's level of detail)
against the oracle and against the gather form: integer counts bit for bit.

Cases reach every level of detail: coarse voxels seen by 512^2 maps (projected
voxels of up to ~20 pixels), cameras inside the domain (the coarsest pyramid
levels, whose pixels span most of the field of view), oblique views along no
axis, ragged brick sets with holes, LIDAR-strength votes on pinhole maps.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2107_14790_b300 import tgv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2107_14790_b300 import build
    build.build()
    assert torch.cuda.is_available()
    tgv.lib()


def stream():
    return torch.cuda.current_stream().cuda_stream


def sphere_views(res, eyes, centre=(0.5, 0.5, 0.5), radius=0.35, fov=45.0, seed=0):
    """Pinhole maps of a sphere from the given eye points (z-depth, small noise)."""
    rng = np.random.default_rng(seed)
    fx, fy, cx, cy = synth.pinhole_intrinsics(res, res, fov)
    centre = np.asarray(centre, np.float64)
    cams, deps = [], []
    for k, C in enumerate(eyes):
        C = np.asarray(C, np.float64)
        cam = synth.Camera(fx, fy, cx, cy, synth.look_at(C, centre), C, res, res)
        d = cam.ray_directions()
        oc = C - centre
        a = np.einsum("hwk,hwk->hw", d, d)
        b = np.einsum("hwk,k->hw", d, oc)
        disc = b * b - a * (float(oc @ oc) - radius * radius)
        t = np.full(a.shape, np.nan)
        ok = disc >= 0
        t[ok] = (-b[ok] - np.sqrt(disc[ok])) / a[ok]
        t[t <= 0] = np.nan
        t = t + rng.normal(0.0, 0.002, size=t.shape)
        cams.append(cam)
        deps.append(t.astype(np.float32))
    return cams, deps


def counts(desc, nbins, cams, deps, votes, form):
    with tgv.Domain([desc], nbins=nbins, stream=stream(), hist_form=form) as dom:
        dom.accumulate(0, cams, torch.from_numpy(np.stack(deps)).cuda(), votes)
        return dom.histograms(0)


def lod_levels(desc, cams, res):
    """Levels of detail Alg. 1 picks over all (voxel, map) pairs in front of the cameras
    (FP64; a property of the test inputs, not of the kernels)."""
    g = desc.bricks[:, None, :] * 8 + np.stack(np.meshgrid(np.arange(8), np.arange(8), np.arange(8),
                                                            indexing="ij"), -1).reshape(-1, 3)[:, ::-1][None]
    X = desc.origin + (g.reshape(-1, 3) + 0.5) * desc.h
    lmax = int(math.floor(math.log2(res)))
    out = set()
    for c in cams:
        zc = (X - c.C) @ np.asarray(c.R).reshape(3, 3)[2]
        fp = c.fx * desc.h / zc[zc > 0]
        out |= set(np.clip(np.floor(np.log2(np.maximum(fp, 1.0))), 0, lmax).astype(int).tolist())
    return out


def check(desc, nbins, cams, deps, votes=None):
    votes = votes or [1] * len(cams)
    orc = oracle.OracleLevel(desc, nbins)
    for c, d, v in zip(cams, deps, votes):
        orc.accumulate(c, d, v)
    sc = counts(desc, nbins, cams, deps, votes, "scatter")
    np.testing.assert_array_equal(sc, orc.hist)
    ga = counts(desc, nbins, cams, deps, votes, "gather")
    np.testing.assert_array_equal(sc, ga)
    return sc


def ring(n, dist, el_deg, centre=(0.5, 0.5, 0.5), phase=0.3):
    c = np.asarray(centre)
    el = math.radians(el_deg)
    return [c + dist * np.array([math.cos(el) * math.cos(2 * math.pi * k / n + phase),
                                 math.cos(el) * math.sin(2 * math.pi * k / n + phase), math.sin(el)])
            for k in range(n)]


def test_sphere_scene_matches_oracle_and_gather(sphere_scene):
    sc = sphere_scene
    h = check(sc.domain, 8, sc.cameras, sc.depths)
    assert h.sum() > 300_000


def test_coarse_voxels_in_fine_maps_use_many_levels():
    """32^3 voxels seen by 512^2 maps: projected voxels of 8 to 200 pixels (levels 3-7)."""
    desc = synth.DomainDesc(np.zeros(3), 1.0 / 32, synth.dense_bricks(4))
    cams, deps = sphere_views(512, ring(6, 1.1, 25.0) + ring(4, 0.9, -35.0, phase=1.1), seed=1)
    assert {3, 4, 5, 6, 7} <= lod_levels(desc, cams, 512)
    h = check(desc, 10, cams, deps)
    assert h.sum() > 10_000


def test_cameras_inside_the_domain_and_oblique_views():
    """Eyes inside the box (the nearest voxels fall to the coarsest levels) and views
    along no axis, on a ragged brick set."""
    rng = np.random.default_rng(3)
    box = synth.dense_bricks(4)
    desc = synth.DomainDesc(np.zeros(3), 1.0 / 32, box[rng.random(len(box)) > 0.25])
    eyes = [(0.08, 0.1, 0.12), (0.93, 0.9, 0.07), (0.5, 0.03, 0.95), (0.97, 0.52, 0.5),
            (1.6, 1.3, 1.4), (-0.7, 1.4, -0.5)]
    cams, deps = sphere_views(512, eyes, seed=2)
    assert max(lod_levels(desc, cams, 512)) == 9
    h = check(desc, 12, cams, deps, votes=[1, 5, 1, 5, 1, 5])
    assert h.sum() > 5_000


def test_fine_voxels_and_sub_pixel_footprints():
    """96^3 voxels seen by 128^2 maps from afar: several voxels per pixel (level 0)."""
    desc = synth.DomainDesc(np.zeros(3), 1.0 / 96, synth.dense_bricks(12))
    cams, deps = sphere_views(128, ring(5, 2.5, 10.0) + ring(3, 1.5, 60.0), fov=30.0, seed=4)
    assert 0 in lod_levels(desc, cams, 128)
    h = check(desc, 8, cams, deps)
    assert h.sum() > 100_000


def test_terrain_maps():
    sc = synth.terrain_scene(1002, 64, 16, 256, 10, 10)
    check(sc.domain, 10, sc.cameras, sc.depths)


def test_offset_domain_with_negative_brick_coordinates():
    bricks = synth.dense_bricks(4, offset=(-2, -1, -3))
    desc = synth.DomainDesc(np.array([2, 1, 3]) * 8 / 32, 1.0 / 32, bricks)  # covers [0, 1)^3
    cams, deps = sphere_views(256, ring(4, 1.2, 15.0), seed=5)
    check(desc, 8, cams, deps)


def test_spherical_maps_are_rejected():
    sc = synth.lidar_sphere_scene()
    with tgv.Domain([sc.domain], nbins=8, stream=stream(), hist_form="scatter") as dom:
        with pytest.raises(tgv.TgvError):
            dom.accumulate(0, sc.cameras[:1], torch.from_numpy(np.stack(sc.depths[:1])).cuda(), [5])
