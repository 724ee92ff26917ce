"""Octree domain builder (Eq. 4, Sec. 4.1-4.2) through the C-ABI against the oracle:
the brick lists of every level must be identical (the sample decisions are taken
in FP32 with the same operation order on both sides; the set operations are
exact), and the levels must drive a coarse-to-fine solve."""
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


def dev(depths):
    return torch.from_numpy(np.stack(depths).astype(np.float32)).cuda()


def check_same(cams, depths, rm, E, dmin, dmax, band):
    lv, ns = tgv.tgv_octree_build(cams, dev(depths), rm, E, dmin, dmax, band,
                                  stream=torch.cuda.current_stream().cuda_stream)
    ref, ns_ref = oracle.octree_build(cams, depths, rm, E, dmin, dmax, band)
    assert ns == ns_ref
    assert len(lv) == len(ref)
    for l, (L, (a, f)) in enumerate(zip(lv, ref)):
        np.testing.assert_array_equal(L.bricks, a, err_msg=f"level {l} active")
        np.testing.assert_array_equal(L.frozen, f, err_msg=f"level {l} frozen")
        assert L.h == E / 2 ** (dmin + l)
    return lv


def test_sphere_scene_levels_identical(sphere_scene):
    sc = sphere_scene
    lv = check_same(sc.cameras, sc.depths, np.array([-0.5, -0.5, -0.5]), 2.0, 3, 8, 1)
    assert sum(L.nbricks for L in lv) > 500


@pytest.mark.parametrize("band", [0, 2])
def test_terrain_levels_identical(band):
    sc = synth.terrain_scene(1002, 64, 16, 256, 10, 10)
    check_same(sc.cameras, sc.depths, np.zeros(3), 1.0, 4, 9, band)


def test_built_levels_drive_a_coarse_to_fine_solve(sphere_scene):
    sc = sphere_scene
    lv, _ = tgv.tgv_octree_build(sc.cameras, dev(sc.depths), np.array([-0.5, -0.5, -0.5]), 2.0, 5, 7, 1,
                                 stream=torch.cuda.current_stream().cuda_stream)
    lv = [L for L in lv if L.nbricks > 0]
    with tgv.Domain(lv, nbins=8, stream=torch.cuda.current_stream().cuda_stream) as dom:
        for l in range(len(lv)):
            dom.accumulate(l, sc.cameras, dev(sc.depths))
        for l in range(len(lv)):
            if l > 0:
                dom.prolong(l - 1)
            dom.solve(l, 60)
            e = dom.energy(l)
            assert e[3] == 1.0 and e[2] >= -1e-6 * abs(e[0])
        u = dom.field(len(lv) - 1, "u")[:, 0]
    assert np.all(np.abs(u) <= 1.0) and (u < 0).any() and (u > 0).any()


def test_invalid_configs_and_camera_models(sphere_scene):
    sc = sphere_scene
    d = dev(sc.depths[:1])
    for bad in [dict(root_edge=0.0), dict(depth_min=2), dict(depth_max=22), dict(band=-1)]:
        kw = dict(root_min=np.zeros(3), root_edge=1.0, depth_min=3, depth_max=6, band=1)
        kw.update(bad)
        with pytest.raises(tgv.TgvError):
            tgv.tgv_octree_build(sc.cameras[:1], d, **kw)
    bad = synth.spherical_scanner(np.array([0.5, 0.5, 0.5]), 128, 64)
    bad.model = 2  # neither pinhole nor spherical
    with pytest.raises(tgv.TgvError) as e:
        tgv.tgv_octree_build([bad], torch.ones((1, 64, 128), device="cuda"), np.zeros(3), 1.0, 3, 6, 1)
    assert e.value.status == 1


def test_lidar_scan_levels_identical():
    """Four full spherical scans of the sphere (ranges, Sec. 3.4): the samples unproject
    through the same FP32 sin / cos on both sides, so every level is identical."""
    sc = synth.lidar_sphere_scene(n=64, nscans=4, width=512, height=256)
    lv = check_same(sc.cameras, sc.depths, np.zeros(3), 1.0, 3, 7, 1)
    assert sum(L.nbricks for L in lv) > 100


def test_scan_from_inside_a_sphere_identical():
    C = np.array([0.5, 0.5, 0.5])
    cam = synth.spherical_scanner(C, 1024, 512)
    dep = np.full((512, 1024), 0.3, np.float32)
    check_same([cam], [dep], np.zeros(3), 1.0, 3, 9, 1)


def test_maps_without_samples_give_empty_levels(sphere_scene):
    sc = sphere_scene
    nan = torch.full((2, sc.depths[0].shape[0], sc.depths[0].shape[1]), float("nan"), device="cuda")
    lv, ns = tgv.tgv_octree_build(sc.cameras[:2], nan, np.zeros(3), 1.0, 3, 6, 1)
    assert ns == 0 and all(L.nbricks == 0 and L.nfrozen == 0 for L in lv)


def test_scattered_samples_outgrow_the_first_level_table():
    """About 2000 isolated sample bricks on one deep level, dilated by 4 rings: 9^3 = 729
    bricks each, about 1.5 M in all, above the level-set table's first size (2 x 32 slots
    per sample brick, rounded up to 2^20), so the build redoes the sets in a larger table;
    the levels still equal the oracle's."""
    rng = np.random.default_rng(11)
    W = H = 512
    fx, fy, cx, cy = synth.pinhole_intrinsics(W, H, 20.0)
    cams, deps = [], []
    for k in range(2):
        C = np.array([0.5 + 0.01 * k, 0.5, 2.5])
        cams.append(synth.Camera(fx, fy, cx, cy, synth.look_at(C, np.array([0.5, 0.5, 0.0]), up=(0.0, 1.0, 0.0)),
                                 C, W, H))
        d = np.full((H, W), np.nan, np.float32)
        for by in range(0, H, 16):
            for bx in range(0, W, 16):
                d[by + 7:by + 9, bx + 7:bx + 9] = rng.uniform(1.7, 2.3)  # a 2 x 2 patch: radius from its neighbours
        deps.append(d)
    lv = check_same(cams, deps, np.zeros(3), 1.0, 12, 12, 4)
    assert lv[0].nbricks > 1_100_000


def test_deep_level_long_keys(sphere_scene):
    """One level at depth 18 (2^15 bricks per axis: 45-bit Morton codes, six radix passes
    of the device sort), every sample its own brick, one ring of band."""
    sc = sphere_scene
    lv = check_same(sc.cameras[:4], sc.depths[:4], np.array([-0.5, -0.5, -0.5]), 2.0, 18, 18, 1)
    assert lv[0].nbricks > 100_000
