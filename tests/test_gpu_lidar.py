"""Spherical (LIDAR) depth maps with vote 5 (Sec. 3.4) through the C-ABI against the oracle.

Bars: histogram counts bit-exact (the pixel and bin decisions are taken in FP32
on both sides, the angles by the same published arctangent polynomial); the
FP32 field after the iterations within 1e-4 of the FP64 oracle.
"""
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


@pytest.fixture(scope="module")
def lidar():
    return synth.lidar_sphere_scene()


def dom_of(desc, nbins, **kw):
    return tgv.Domain([desc], nbins=nbins, stream=torch.cuda.current_stream().cuda_stream, **kw)


def dev(depths):
    return torch.from_numpy(np.stack(depths).astype(np.float32)).cuda()


def test_lidar_histograms_bit_exact(lidar):
    sc = lidar
    orc = oracle.OracleLevel(sc.domain, sc.nbins)
    ndiff = 0
    for cam, d, v in zip(sc.cameras, sc.depths, sc.votes):
        ndiff += orc.accumulate(cam, d, v, diag=True)[1]
    with dom_of(sc.domain, sc.nbins) as dom:
        dom.accumulate(0, sc.cameras, dev(sc.depths), sc.votes)
        h = dom.histograms(0)
    np.testing.assert_array_equal(h, orc.hist)
    assert h.sum() > 300_000 and np.all(h % 5 == 0)
    assert ndiff <= 10  # votes an FP64 evaluation with exact atan2 would decide otherwise


def test_lidar_single_calls_match_batch(lidar):
    sc = lidar
    with dom_of(sc.domain, sc.nbins) as dom:
        dom.accumulate(0, sc.cameras, dev(sc.depths), sc.votes)
        batch = dom.histograms(0)
    with dom_of(sc.domain, sc.nbins) as dom:
        for cam, d, v in zip(reversed(sc.cameras), reversed(sc.depths), reversed(sc.votes)):
            tgv.tgv_accumulate_depthmap(dom.handle, 0, cam, torch.from_numpy(d).cuda(), v)
        single = dom.histograms(0)
    np.testing.assert_array_equal(single, batch)


def test_pinhole_and_lidar_maps_together_then_solve(lidar, sphere_scene):
    """Close-range photos (vote 1) and LIDAR scans (vote 5) of the same sphere, as in the
    paper's mixed datasets: counts bit-exact, then 120 iterations within 1e-4."""
    ph, li = sphere_scene, lidar
    orc = oracle.OracleLevel(ph.domain, 8)
    for cam, d in zip(ph.cameras, ph.depths):
        orc.accumulate(cam, d, 1)
    for cam, d, v in zip(li.cameras, li.depths, li.votes):
        orc.accumulate(cam, d, v)
    with dom_of(ph.domain, 8) as dom:
        dom.accumulate(0, ph.cameras, dev(ph.depths))
        dom.accumulate(0, li.cameras, dev(li.depths), li.votes)
        h = dom.histograms(0)
        np.testing.assert_array_equal(h, orc.hist)
        dom.solve(0, 120)
        u = dom.field(0, "u")[:, 0]
    orc.iterate(120)
    assert np.max(np.abs(u - orc.u)) <= 1e-4


def test_unknown_camera_model_is_rejected(lidar):
    sc = lidar
    cam = synth.spherical_scanner(sc.cameras[0].C, sc.cameras[0].width, sc.cameras[0].height)
    cam.model = 7
    with dom_of(sc.domain, sc.nbins) as dom:
        with pytest.raises(tgv.TgvError):
            dom.accumulate(0, [cam], dev(sc.depths[:1]), [5])


def test_pinhole_and_spherical_maps_in_one_batch(lidar):
    """One accumulate call may mix camera models (maps of one size)."""
    sc = lidar
    W, H = sc.cameras[0].width, sc.cameras[0].height
    fx, fy, cx, cy = synth.pinhole_intrinsics(W, H, 60.0)
    ph = synth.Camera(fx, fy, cx, cy, synth.look_at(np.array([0.5, -0.9, 0.5]), np.array([0.5, 0.5, 0.5])),
                      np.array([0.5, -0.9, 0.5]), W, H)
    dep = np.full((H, W), 1.4, np.float32)
    cams = [sc.cameras[0], ph, sc.cameras[1]]
    deps = [sc.depths[0], dep, sc.depths[1]]
    votes = [5, 1, 5]
    orc = oracle.OracleLevel(sc.domain, sc.nbins)
    for c, d, v in zip(cams, deps, votes):
        orc.accumulate(c, d, v)
    with dom_of(sc.domain, sc.nbins) as dom:
        dom.accumulate(0, cams, dev(deps), votes)
        np.testing.assert_array_equal(dom.histograms(0), orc.hist)
