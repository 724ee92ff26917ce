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


# --- spherical (LIDAR) maps: scanner at the origin, world axes, 64 x 32 full scan --------
import math as _m


def _scan(W=64, H=32):
    return synth.spherical_scanner(np.zeros(3), W, H)


S_ORIGIN = np.array([-1.0 / 128] * 3)  # voxel (i, j, k) centre = (i, j, k) / 64 exactly


def _sbins(idx, depth, nbins=8):
    return list(oracle.vote_list(np.asarray(idx, np.int64), S_ORIGIN, H_VOX, R_VOX, _scan(), depth, nbins))


def test_atan2_polynomial_against_the_library():
    """A&S 4.4.49 plus octant reduction, in FP32: within 4e-7 rad of atan2 over a grid
    spanning all octants and magnitudes; exact on the axes; odd in y."""
    vals = np.concatenate([-np.logspace(-3, 3, 25), [0.0], np.logspace(-3, 3, 25)]).astype(np.float32)
    worst = 0.0
    for y in vals:
        for x in vals:
            a = oracle.atan2_as(y, x)
            if x == 0 and y == 0:
                assert a == 0.0
                continue
            worst = max(worst, abs(a - _m.atan2(float(y), float(x))))
            assert oracle.atan2_as(-y, x) == -a or y == 0
    assert worst <= 4e-7, worst
    assert oracle.atan2_as(0.0, 1.0) == 0.0
    assert oracle.atan2_as(1.0, 0.0) == float(np.float32(_m.pi / 2))
    assert oracle.atan2_as(0.0, -1.0) == float(np.float32(_m.pi))


def test_spherical_bins_by_range_along_an_axis():
    """Along +x the angles are exactly 0: pixel (32, 16); a = depth - range.  With a
    constant range map of 1 the voxel at range k/64 has a/delta = (64-k)/3."""
    depth = np.ones((32, 64), np.float32)
    cases = {60: 7, 61: 7, 62: 6, 63: 5, 64: 4, 65: 2, 66: 1, 67: 0,
             73: 0,    # a = -eta exactly still votes
             74: -1,   # a < -eta
             0: -1}    # range 0: no direction
    got = _sbins([(k, 0, 0) for k in cases], depth)
    assert got == list(cases.values())
    only = np.full((32, 64), np.nan, np.float32)
    only[16, 32] = 1.0  # the single pixel the +x axis maps to
    assert _sbins([(64, 0, 0), (65, 0, 0)], only) == [4, 2]


def test_spherical_bins_depend_on_range_not_direction():
    """Voxels at equal range in different directions (away from the poles and the
    azimuth seam) take the same bin from a constant range map."""
    depth = np.ones((32, 64), np.float32)
    # range exactly 1 on the axes; 65/64 on the 39-52-65 diagonals (a/delta = -1/3)
    pts = [(64, 0, 0), (0, 64, 0), (0, -64, 0), (39, 52, 0), (-39, 52, 0), (39, -52, 0), (-39, -52, 0), (52, 0, 39)]
    want = [4, 4, 4, 2, 2, 2, 2, 2]
    assert _sbins(pts, depth) == want


def test_spherical_pixel_follows_the_library_angles():
    """Each voxel votes only where its pixel (from numpy's arctan2 in FP64) holds the
    single valid sample; voxels within 1e-4 pixel of a pixel edge are skipped."""
    rng = np.random.default_rng(5)
    cam = _scan(256, 128)
    checked = 0
    for _ in range(60):
        idx = rng.integers(-60, 61, size=3)
        c = idx / 64.0
        rho = float(np.linalg.norm(c))
        if rho < 0.5:
            continue
        x = cam.fx * _m.atan2(c[1], c[0]) + cam.cx
        y = cam.cy - cam.fy * _m.atan2(c[2], _m.hypot(c[0], c[1]))
        if min(abs(x - round(x)), abs(y - round(y))) < 1e-4 or not (0 <= x < 256 and 0 <= y < 128):
            continue
        fp = cam.fx * H_VOX / rho
        assert fp < 2.0  # level of detail 0
        depth = np.full((128, 256), np.nan, np.float32)
        depth[int(_m.floor(y)), int(_m.floor(x))] = rho + 0.25 * 3 / 64  # a = delta / 4
        got = oracle.vote_list(idx[None, :].astype(np.int64), S_ORIGIN, H_VOX, R_VOX, cam, depth, 8)
        assert got[0] == 5, (idx, x, y)
        checked += 1
    assert checked > 30


def test_spherical_level_of_detail_uses_the_pyramid():
    """At range 1/16 the projected diameter is 16/(2 pi) = 2.55 pixels: level 1, pixel
    (16, 8), the minimum of level-0 pixels (32..33, 16..17); at range 1, level 0."""
    depth = np.full((32, 64), np.nan, np.float32)
    depth[17, 33] = 1.0
    assert _sbins([(4, 0, 0), (64, 0, 0)], depth) == [7, -1]


def test_spherical_votes_of_five():
    sc = synth.lidar_sphere_scene(n=32, nscans=2, width=128, height=64)
    lvl = oracle.OracleLevel(sc.domain, sc.nbins)
    votes = sum(lvl.accumulate(c, d, 5) for c, d in zip(sc.cameras, sc.depths))
    assert votes > 0 and int(lvl.hist.sum()) == 5 * votes and np.all(lvl.hist % 5 == 0)


def _pyramid_np(depth):
    """Depth pyramid written independently: level l+1 = min of the valid children (NaN none)."""
    d = np.where(np.isfinite(depth) & (depth > 0), depth.astype(np.float64), np.nan)
    levels = [d]
    while max(levels[-1].shape) > 1:
        a = levels[-1]
        h, w = a.shape
        p = np.full((h + h % 2, w + w % 2), np.nan)
        p[:h, :w] = a
        blocks = p.reshape(p.shape[0] // 2, 2, p.shape[1] // 2, 2).transpose(0, 2, 1, 3).reshape(-1, 4)
        ok = ~np.all(np.isnan(blocks), axis=1)
        m = np.full(blocks.shape[0], np.nan)
        m[ok] = np.nanmin(blocks[ok], axis=1)
        levels.append(m.reshape(p.shape[0] // 2, p.shape[1] // 2))
    return levels


def test_scatter_from_pixels_equals_the_gather(sphere_scene):
    """Alg. 1 from the pixel side: every valid pyramid pixel (level l, i, j) gives its vote to
    the voxels it owns (centre in its square at level l, level of detail l, a >= -eta), in
    FP64 numpy with its own pyramid; the oracle's FP32 gather must give the same counts on
    every voxel none of whose decisions lies within 1e-4 of a border (pixel edge, level
    threshold, bin edge, occlusion cut)."""
    sc = sphere_scene
    n = 32
    desc = synth.DomainDesc(np.zeros(3), 1.0 / n, synth.dense_bricks(n // 8))
    nbins = 8
    cams = sc.cameras[:3] + [synth.Camera(*synth.pinhole_intrinsics(128, 128, 50.0),
                                          synth.look_at(np.array([0.1, 0.12, 0.15]), np.array([0.5, 0.5, 0.5])),
                                          np.array([0.1, 0.12, 0.15]), 128, 128)]
    deps = [d for d in sc.depths[:3]]
    c4 = cams[3]
    dirs = c4.ray_directions()
    oc = c4.C - np.array([0.5, 0.5, 0.5])
    b = np.einsum("hwk,k->hw", dirs, oc)
    aa = np.einsum("hwk,hwk->hw", dirs, dirs)
    disc = b * b - aa * (oc @ oc - 0.35 ** 2)
    t = np.where(disc >= 0, (-b - np.sqrt(np.maximum(disc, 0))) / aa, np.nan)
    deps.append(t.astype(np.float32))
    g = desc.bricks[:, None, :] * 8 + np.stack(np.meshgrid(np.arange(8), np.arange(8), np.arange(8),
                                                            indexing="ij"), -1).reshape(-1, 3)[:, ::-1][None]
    g = g.reshape(-1, 3)  # global voxel index, in the oracle's voxel order (x fastest within a brick)
    X = desc.origin + (g + 0.5) * desc.h
    r = desc.h / 2
    delta, eta = 6 * r, 18 * r
    scatter = np.zeros((len(X), nbins), np.int64)
    safe = np.ones(len(X), bool)
    used_levels = set()
    for cam, dep in zip(cams, deps):
        levels = _pyramid_np(dep)
        R = np.asarray(cam.R).reshape(3, 3)
        Xc = (X - cam.C) @ R.T
        front = Xc[:, 2] > 0
        zc = np.where(front, Xc[:, 2], 1.0)
        px = cam.fx * Xc[:, 0] / zc + cam.cx
        py = cam.fy * Xc[:, 1] / zc + cam.cy
        fp = cam.fx * 2 * r / zc
        lod = np.clip(np.floor(np.log2(np.maximum(fp, 1.0))), 0, len(levels) - 1).astype(int)
        # borders: the level threshold, the pixel edges at that level
        lg = np.log2(np.maximum(fp, 1.0))
        safe &= ~front | (np.abs(lg - np.round(lg)) > 1e-4) | (fp < 1.0) | (lg > len(levels) - 1 + 1e-4)
        sx, sy = px / 2.0 ** lod, py / 2.0 ** lod
        safe &= ~front | ((np.abs(sx - np.round(sx)) > 1e-4) & (np.abs(sy - np.round(sy)) > 1e-4))
        # the pixel side: each valid pixel of each level collects the voxels it owns
        owner = {}
        for v in np.nonzero(front)[0]:
            l = lod[v]
            i, j = int(np.floor(sx[v])), int(np.floor(sy[v]))
            hl, wl = levels[l].shape
            if 0 <= i < wl and 0 <= j < hl:
                owner.setdefault((l, i, j), []).append(v)
        for (l, i, j), vox in owner.items():
            D = levels[l][j, i]
            if np.isnan(D):
                continue
            used_levels.add(l)
            for v in vox:
                a = D - zc[v]
                if abs(a + eta) < 1e-4:
                    safe[v] = False
                if a < -eta:
                    continue
                s = (min(1.0, max(-1.0, a / delta)) + 1.0) / 2.0 * nbins
                if abs(s - round(s)) < 1e-4 and 0 < round(s) < nbins:
                    safe[v] = False
                scatter[v, min(int(np.floor(s)), nbins - 1)] += 1
    orc = oracle.OracleLevel(desc, nbins)
    for cam, dep in zip(cams, deps):
        orc.accumulate(cam, dep, 1)
    assert safe.mean() > 0.9
    assert scatter[safe].sum() > 10_000 and len(used_levels) >= 3
    np.testing.assert_array_equal(orc.hist[safe].astype(np.int64), scatter[safe])
