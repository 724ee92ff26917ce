"""Pins of the oracle's depth pyramid and Alg. 1 binning against hand-derived values.

Every expected value here is worked out by hand from Alg. 1 (Sec. 3.4) and the
distance-field widths of Sec. 3.1 (delta = 6 r, eta = 3 delta), on dyadic
geometry where FP32 and exact arithmetic agree; none is produced by the oracle.
"""
import math

import numpy as np
import pytest

import oracle
import synth

NAN = float("nan")


def test_pyramid_hand_example():
    d = np.array([[1, 2, NAN, 4, 5],
                  [3, NAN, NAN, 0, 6],
                  [7, 8, 9, -1, np.inf]], dtype=np.float32)
    lv = oracle.pyramid_levels(d)
    assert len(lv) == 3  # Lmax = floor(log2 5) = 2
    l0 = np.array([[1, 2, NAN, 4, 5], [3, NAN, NAN, NAN, 6], [7, 8, 9, NAN, NAN]], np.float32)
    l1 = np.array([[1, 4, 5], [7, 9, NAN]], np.float32)
    l2 = np.array([[1, 5]], np.float32)
    for got, want in zip(lv, [l0, l1, l2]):
        np.testing.assert_array_equal(got, want)


def test_pyramid_level_counts():
    for (W, H, n) in [(128, 128, 8), (512, 512, 10), (1024, 1024, 11), (5, 3, 3), (1, 1, 1), (2, 1, 2)]:
        dims, offs, total = oracle.pyramid_layout(W, H)
        assert len(offs) == n
        assert total == int(sum(dims[:, 0] * dims[:, 1]))
    dims, _, _ = oracle.pyramid_layout(128, 128)
    assert tuple(dims[-1]) == (1, 1)


# --- a camera at the origin looking along +z, fx = fy = 64, 64x64 pixels --------------
def _cam(W=64):
    return synth.Camera(64.0, 64.0, 32.0, 32.0, np.eye(3), np.zeros(3), W, W)


H_VOX = 1.0 / 64
ORIGIN = np.array([-1.0 / 128, -1.0 / 128, 1.0 / 128])  # voxel (0, 0, k) centre = (0, 0, (k+1)/64)
R_VOX = H_VOX / 2  # delta = 3/64, eta = 9/64


def _bins(ks, depth, nbins=8, xs=None):
    xs = [0] * len(ks) if xs is None else xs
    idx = np.array([[x, 0, k] for x, k in zip(xs, ks)], np.int64)
    return list(oracle.vote_list(idx, ORIGIN, H_VOX, R_VOX, _cam(), depth, nbins))


def test_alg1_plane_bins_by_hand():
    depth = synth.plane_depth(64, 64, 1.0)
    # voxel k has z-depth (k+1)/64, a = (63-k)/64, a/delta = (63-k)/3
    cases = {
        59: 7,   # a = 4/64 > delta: clamp to +1, bin 8 -> n-1
        60: 7,   # a = +delta exactly: bin 8 -> n-1
        61: 6,   # a/delta = 2/3 -> floor(4 * 5/3) = 6
        62: 5,   # 1/3 -> floor(5.33)
        63: 4,   # a = 0 -> n/2
        64: 2,   # -1/3 -> floor(2.67)
        65: 1,   # -2/3 -> floor(1.33)
        66: 0,   # a = -delta
        70: 0,   # occluded band, clamped to -1
        72: 0,   # a = -eta exactly: still votes (Alg. 1 returns only for a < -eta)
        73: -1,  # a < -eta: no vote
        -1: -1,  # z-depth 0: not in front of the camera
        -2: -1,  # behind the camera
    }
    got = _bins(list(cases), depth)
    assert got == list(cases.values())


def test_alg1_plane_bins_ten_bins():
    depth = synth.plane_depth(64, 64, 1.0)
    got = _bins([63, 62, 64, 60, 66], depth, nbins=10)
    # a/delta = 0, 1/3, -1/3, 1, -1  ->  floor(5), floor(6.67), floor(3.33), 10 -> 9, 0
    assert got == [5, 6, 3, 9, 0]


def test_alg1_invalid_pixel_and_image_bounds():
    depth = synth.plane_depth(64, 64, 1.0)
    depth[32, 32] = np.nan  # voxel (0, 0, 63) projects to pixel (32, 32)
    assert _bins([63], depth) == [-1]
    depth = synth.plane_depth(64, 64, 1.0)
    depth[32, 32] = -3.0  # negative depth is invalid too
    assert _bins([63], depth) == [-1]
    depth = synth.plane_depth(64, 64, 1.0)
    # x index 31 -> X = 31/64 at z-depth 1 -> pixel 63 (inside); x = 32 -> pixel 64 (outside)
    assert _bins([63, 63], depth, xs=[31, 32]) == [4, -1]
    assert _bins([63], depth, xs=[-32]) == [4]  # X = -1/2 -> pixel 0
    assert _bins([63], depth, xs=[-33]) == [-1]


def test_alg1_lod_uses_min_of_children():
    # voxel k = 31 has z-depth 1/2: projected diameter fx*2r/Zc = 2 pixels -> LOD 1
    depth = synth.plane_depth(64, 64, 33.0 / 64)
    depth[32, 33] = 0.5  # one child of LOD-1 pixel (16, 16) is nearer
    # LOD 1 reads min(33/64, 1/2, ...) = 1/2 -> a = 0 -> bin 4 (LOD 0 would read 33/64 -> bin 5)
    assert _bins([31], depth) == [4]
    # voxel k = 32 (z-depth 33/64) has diameter 64/33 < 2 pixels -> LOD 0 -> a = 0 -> bin 4
    assert _bins([32], depth) == [4]
    # a voxel at z-depth 1/4 has diameter 4 -> LOD 2: pixel (8, 8) covers level-0 [32, 36)^2
    depth = synth.plane_depth(64, 64, 1.0)
    depth[35, 35] = 0.25 + 1.0 / 64  # min over that block; k = 15 has z-depth 16/64
    assert _bins([15], depth) == [5]  # a = 1/64 -> a/delta = 1/3 -> bin 5


def test_vote_totals_plane_block():
    """A 16x16x32 voxel block in front of a plane: per-bin totals by counting layers."""
    cam = _cam()
    depth = synth.plane_depth(64, 64, 1.0)
    bricks = np.array([[bx, by, bz] for bz in (6, 7, 8, 9) for by in (-1, 0) for bx in (-1, 0)], np.int32)
    dom = synth.DomainDesc(origin=ORIGIN, h=H_VOX, bricks=bricks)
    for vote in (1, 5):
        lvl = oracle.OracleLevel(dom, 8)
        nv = lvl.accumulate(cam, depth, vote=vote)
        # z layers 48..79: 48..60 -> bin 7 (13 layers), 61 -> 6, 62 -> 5, 63 -> 4, 64 -> 2,
        # 65 -> 1, 66..72 -> 0 (7 layers), 73.. -> no vote; 256 columns per layer
        want = np.array([7, 1, 1, 0, 1, 1, 1, 13]) * 256 * vote
        np.testing.assert_array_equal(lvl.hist.sum(axis=0), want)
        assert nv == 25 * 256


def test_sphere_fp32_decision_matches_fp64_nearly_everywhere(sphere_scene):
    sc = sphere_scene
    lvl = oracle.OracleLevel(sc.domain, sc.nbins)
    votes, diffs = 0, 0
    for cam, d in zip(sc.cameras, sc.depths):
        v, nd = lvl.accumulate(cam, d, 1, diag=True)
        votes += v
        diffs += nd
    assert votes > 300_000
    assert diffs <= 1e-3 * votes
    # every voxel is seen by at most 16 maps, one vote each
    assert lvl.hist.sum(axis=1).max() <= 16
    # free space (bin n-1) and occluded (bin 0) dominate, as the depth band is thin
    tot = lvl.hist.sum(axis=0)
    assert tot[-1] > tot[1:-1].max() and tot[0] > tot[1:-1].max()


def test_sphere_band_bins_follow_signed_distance(sphere_scene):
    """Votes of voxels well outside the sphere are mostly free space (bin n-1); voxels
    deeper inside than eta (9 voxels) plus the field-of-view slant are never observed."""
    sc = sphere_scene
    lvl = oracle.OracleLevel(sc.domain, sc.nbins)
    for cam, d in zip(sc.cameras, sc.depths):
        lvl.accumulate(cam, d, 1)
    g = lvl.global_voxels()
    xyz = (g + 0.5) * sc.domain.h
    sd = (np.linalg.norm(xyz - 0.5, axis=1) - 0.35) / sc.domain.h  # signed distance in voxels
    far_out = (sd > 6) & (lvl.hist.sum(1) > 0)
    assert far_out.sum() > 1000
    assert lvl.hist[far_out, -1].sum() >= 0.9 * lvl.hist[far_out].sum()
    deep_in = (sd < -12)
    assert deep_in.sum() > 4000  # ball of radius 22.4 - 12 voxels: about 4700 voxels
    assert lvl.hist[deep_in].sum() == 0  # deeper than eta = 9 voxels: never observed
    assert math.isclose(sc.domain.h, 1 / 64)
