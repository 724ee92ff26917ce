"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle.

Bars (written into each test):
* histogram counts: bit-exact (integer work, decision taken in FP32 on both sides);
* FP32 field after the configured iterations: |u_gpu - u_oracle|_inf <= 1e-4;
* energy / dual value / gap on an identical state: within 1e-6 of the energy;
* zero level set: identical sign pattern where both |u| > 1e-3, crossings within 1e-3 h.
"""
import itertools

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2107_14790_b300 import tgv
from tests._geom import dense_from_bricks, edge_crossings

pytestmark = pytest.mark.gpu

U_TOL = 1e-4
KERNEL = {"form": "paired"}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2107_14790_b300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    tgv.lib()


@pytest.fixture(autouse=True, params=["paired", "pipelined", "one_brick_per_cta"])
def iter_kernel(request):
    """Every parity test runs with each form of the fused iteration kernel."""
    KERNEL["form"] = request.param
    yield request.param
    KERNEL["form"] = "paired"


def gdomain(levels, nbins, **kw):
    if not isinstance(levels, (list, tuple)):
        levels = [levels]
    kw.setdefault("iter_kernel", KERNEL["form"])
    return tgv.Domain(levels, nbins=nbins, stream=torch.cuda.current_stream().cuda_stream, **kw)


def dev_depths(depths):
    return torch.from_numpy(np.stack(depths).astype(np.float32)).cuda()


# --------------------------------------------------------------------------- histograms
def test_histograms_sphere_bit_exact(sphere_scene):
    sc = sphere_scene
    orc = oracle.OracleLevel(sc.domain, sc.nbins)
    for cam, d in zip(sc.cameras, sc.depths):
        orc.accumulate(cam, d, 1)
    with gdomain(sc.domain, sc.nbins) as dom:
        dom.accumulate(0, sc.cameras, dev_depths(sc.depths))
        h = dom.histograms(0)
        assert dom.launches > 0
    np.testing.assert_array_equal(h, orc.hist)
    assert h.sum() > 300_000


def test_histograms_single_calls_padded_pitch_and_votes(sphere_scene):
    sc = sphere_scene
    orc = oracle.OracleLevel(sc.domain, sc.nbins)
    votes = [1 + (k % 3) * 2 for k in range(len(sc.cameras))]  # 1, 3, 5
    for cam, d, v in zip(sc.cameras, sc.depths, votes):
        orc.accumulate(cam, d, v)
    H, W = sc.depths[0].shape
    with gdomain(sc.domain, sc.nbins) as dom:
        for cam, d, v in zip(sc.cameras, sc.depths, votes):
            buf = torch.full((H, W + 13), float("nan"), device="cuda")
            buf[:, :W] = torch.from_numpy(d).cuda()
            tgv.tgv_accumulate_depthmap(dom.handle, 0, cam, buf[:, :W], v)
        h = dom.histograms(0)
    np.testing.assert_array_equal(h, orc.hist)


def test_histograms_plane_cases_and_ragged_domain():
    """The hand-pinned plane geometry (dyadic values) on a ragged brick set, 10 bins."""
    cam = synth.Camera(64.0, 64.0, 32.0, 32.0, np.eye(3), np.zeros(3), 64, 64)
    depth = synth.plane_depth(64, 64, 1.0)
    depth[40, 40] = np.nan
    depth[10:20, 5:9] = 0.75
    bricks = np.array([[bx, by, bz] for bz in (3, 6, 7, 8, 9) for by in (-2, -1, 0, 1) for bx in (-1, 0, 2)
                       if (bx + by + bz) % 4 != 0], np.int32)
    dom_desc = synth.DomainDesc(origin=np.array([-1 / 128, -1 / 128, 1 / 128]), h=1 / 64, bricks=bricks)
    orc = oracle.OracleLevel(dom_desc, 10)
    orc.accumulate(cam, depth, 1)
    with gdomain(dom_desc, 10) as dom:
        dom.accumulate(0, [cam], dev_depths([depth]))
        h = dom.histograms(0)
    np.testing.assert_array_equal(h, orc.hist)
    assert h.sum() > 5000


def test_histogram_count_budget_is_enforced(sphere_scene):
    sc = sphere_scene
    with gdomain(sc.domain, sc.nbins) as dom:
        d = dev_depths(sc.depths[:1])
        tgv.tgv_accumulate_depthmap(dom.handle, 0, sc.cameras[0], d[0], 60000)
        with pytest.raises(tgv.TgvError) as e:
            tgv.tgv_accumulate_depthmap(dom.handle, 0, sc.cameras[0], d[0], 6000)
        assert e.value.status == 3
        with pytest.raises(tgv.TgvError):
            dom.set_histograms(0, np.full((dom.voxels(0), sc.nbins), 70000, np.uint32))


# --------------------------------------------------------------------------- TGV iteration
def run_pair(desc, hist, nbins, iters, orc_kw=None, gpu_kw=None, levels=None):
    orc_kw = orc_kw or {}
    gpu_kw = gpu_kw or {}
    orc = oracle.OracleLevel(desc, nbins, **orc_kw)
    orc.hist[:] = hist
    orc.iterate(iters)
    dom = gdomain(desc, nbins, **gpu_kw)
    dom.set_histograms(0, hist)
    dom.solve(0, iters)
    return orc, dom


def assert_fields_close(orc, dom, tol_u=U_TOL, tol_other=None):
    u = dom.field(0, "u")[:, 0]
    err = np.max(np.abs(u - orc.u)) if u.size else 0.0
    assert err <= tol_u, f"|u_gpu - u_oracle|_inf = {err}"
    if tol_other is not None:
        for name, ref in (("v", orc.v), ("p", orc.p), ("q", orc.q), ("ubar", orc.ubar[:, None]),
                          ("vbar", orc.vbar)):
            got = dom.field(0, name)
            e = np.max(np.abs(got - ref.reshape(got.shape))) if got.size else 0.0
            assert e <= tol_other, f"{name}: {e}"
    return err


@pytest.fixture(scope="module")
def sphere_hist(sphere_scene):
    sc = sphere_scene
    orc = oracle.OracleLevel(sc.domain, sc.nbins)
    for cam, d in zip(sc.cameras, sc.depths):
        orc.accumulate(cam, d, 1)
    return orc.hist.copy()


def test_tgv_sphere_200_iterations_fp32(sphere_scene, sphere_hist):
    sc = sphere_scene
    orc, dom = run_pair(sc.domain, sphere_hist, sc.nbins, sc.iterations)
    with dom:
        err = assert_fields_close(orc, dom, tol_other=1e-3)
        # zero level set agreement
        u = dom.field(0, "u")[:, 0]
        n = 64
        Ug = dense_from_bricks(u, sc.domain.bricks, n)
        Uo = dense_from_bricks(orc.u, sc.domain.bricks, n)
        both = (np.abs(Ug) > 1e-3) & (np.abs(Uo) > 1e-3)
        for ax in range(3):
            a0 = [slice(None)] * 3
            a1 = [slice(None)] * 3
            a0[ax] = slice(0, -1)
            a1[ax] = slice(1, None)
            m = both[tuple(a0)] & both[tuple(a1)]
            sg = np.sign(Ug[tuple(a0)]) != np.sign(Ug[tuple(a1)])
            so = np.sign(Uo[tuple(a0)]) != np.sign(Uo[tuple(a1)])
            assert np.array_equal(sg[m], so[m])
        mask = np.ones_like(Ug, bool)
        pg, ig = edge_crossings(Ug, mask, sc.domain.h, eps=1e-3)
        po, io = edge_crossings(Uo, mask, sc.domain.h, eps=1e-3)
        common = {tuple(r): k for k, r in enumerate(io.tolist())}
        idx = [(k, common[tuple(r)]) for k, r in enumerate(ig.tolist()) if tuple(r) in common]
        assert len(idx) > 5000
        kg, ko = np.array(idx).T
        disp = np.max(np.linalg.norm(pg[kg] - po[ko], axis=1)) / sc.domain.h
        assert disp <= 1e-3, disp
    print(f"sphere: |du|_inf = {err:.3g}")


def test_tgv_random_hist_ragged_domain_and_bins():
    rng = np.random.default_rng(21)
    box = synth.dense_bricks(4)
    keep = rng.random(len(box)) > 0.3
    desc = synth.DomainDesc(np.zeros(3), 1.0, box[keep])
    # 8, 10 and 12 bins are compile-time instantiations of the paired kernel; the others
    # take the bin count at run time
    for nbins, centres in ((2, 0), (10, 1), (16, 0), (5, 0), (12, 0), (8, 1)):
        hist = synth.random_histograms(rng, desc.nvox, nbins, max_count=12)
        orc, dom = run_pair(desc, hist, nbins, 40, orc_kw=dict(centres=centres), gpu_kw=dict(centres=centres))
        with dom:
            assert_fields_close(orc, dom, tol_other=1e-4)


def test_tgv_frozen_halo_chunk():
    specs = synth.chunk_workload(seed=123, nchunks=2, min_vox=8 * 512, max_vox=30 * 512, nbins_range=(8, 12))
    for sp in specs:
        orc, dom = run_pair(sp.domain, sp.hist, sp.nbins, 60)
        with dom:
            assert_fields_close(orc, dom, tol_other=1e-4)


def test_tgv_parameters_and_no_clamp():
    rng = np.random.default_rng(4)
    desc = synth.DomainDesc(np.zeros(3), 1.0, synth.dense_bricks(2, 2, 3))
    hist = synth.random_histograms(rng, desc.nvox, 8, max_count=4)
    kw = dict(alpha1=0.7, alpha0=1.3, lam=0.5, tau=0.1, sigma=0.3, clamp_u=False)
    orc, dom = run_pair(desc, hist, 8, 50, orc_kw=kw, gpu_kw=kw)
    with dom:
        assert_fields_close(orc, dom, tol_other=1e-4)


def test_tgv_single_brick_and_empty_domain():
    rng = np.random.default_rng(8)
    desc = synth.DomainDesc(np.zeros(3), 1.0, np.array([[5, -3, 2]], np.int32))
    hist = synth.random_histograms(rng, desc.nvox, 8)
    orc, dom = run_pair(desc, hist, 8, 30)
    with dom:
        assert_fields_close(orc, dom, tol_other=1e-4)
        e = dom.energy(0)
        assert e[3] == 1.0
    empty = synth.DomainDesc(np.zeros(3), 1.0, np.zeros((0, 3), np.int32))
    with gdomain(empty, 8) as dom:
        dom.solve(0, 5)
        assert dom.field(0, "u").shape == (0, 1)
        assert list(dom.energy(0)) == [0.0, 0.0, 0.0, 1.0]


def test_energy_and_gap_on_identical_state(sphere_scene, sphere_hist):
    sc = sphere_scene
    orc = oracle.OracleLevel(sc.domain, sc.nbins)
    orc.hist[:] = sphere_hist
    orc.iterate(60)
    # round the state to FP32 and evaluate both sides on exactly that state
    for f in ("u", "v", "p", "q"):
        setattr(orc, f, getattr(orc, f).astype(np.float32).astype(np.float64))
    ref = orc.energy()
    with gdomain(sc.domain, sc.nbins) as dom:
        dom.set_histograms(0, sphere_hist)
        for f in ("u", "v", "p", "q"):
            dom.set_field(0, f, getattr(orc, f).reshape(orc.n, -1).astype(np.float32))
        got = dom.energy(0)
    scale = abs(ref[0])
    for k in range(3):
        assert abs(got[k] - ref[k]) <= 1e-6 * scale, (k, got, ref)
    assert got[3] == ref[3] == 1.0


def test_energy_with_frozen_constants():
    sp = synth.chunk_workload(seed=5, nchunks=1, min_vox=12 * 512, max_vox=12 * 512, nbins_range=(10, 10))[0]
    rng = np.random.default_rng(2)
    orc = oracle.OracleLevel(sp.domain, sp.nbins)
    orc.hist[:] = sp.hist
    orc.u[:] = rng.uniform(-1, 1, orc.n).astype(np.float32)
    orc.v[:] = rng.normal(0, 0.1, (orc.n, 3)).astype(np.float32)
    orc.p[:] = oracle.project_p(rng.normal(0, 0.5, (orc.n, 3)), 1.0).astype(np.float32)
    orc.q[:] = oracle.project_q(rng.normal(0, 0.5, (orc.n, 6)), 2.0).astype(np.float32)
    ref = orc.energy()
    with gdomain(sp.domain, sp.nbins) as dom:
        dom.set_histograms(0, sp.hist)
        for f in ("u", "v", "p", "q"):
            dom.set_field(0, f, getattr(orc, f).reshape(orc.n, -1).astype(np.float32))
        got = dom.energy(0)
    for k in range(3):
        assert abs(got[k] - ref[k]) <= 1e-6 * abs(ref[0]), (k, got, ref)


def test_prolongation_two_levels():
    rng = np.random.default_rng(17)
    coarse = synth.DomainDesc(np.zeros(3), 1 / 16, synth.dense_bricks(2))
    fb = synth.dense_bricks(3, 3, 3, offset=(0, 0, 0))
    act = fb[(fb[:, 0] < 3) & (fb[:, 2] < 2)]
    frz = np.array([c for c in fb.tolist() if not ((c[0] < 3) and (c[2] < 2))], np.int32)
    fine = synth.DomainDesc(np.zeros(3), 1 / 32, act, frozen=frz)
    hc = synth.random_histograms(rng, coarse.nvox, 8)
    hf = synth.random_histograms(rng, fine.nvox, 8)
    oc = oracle.OracleLevel(coarse, 8)
    oc.hist[:] = hc
    oc.iterate(20)
    of = oracle.OracleLevel(fine, 8)
    of.hist[:] = hf
    of.prolong_from(oc)
    oracle.prolong_frozen(of, oc)
    of.iterate(15)
    with gdomain([coarse, fine], 8) as dom:
        dom.set_histograms(0, hc)
        dom.set_histograms(1, hf)
        dom.solve(0, 20)
        dom.prolong(0)
        dom.solve(1, 15)
        u = dom.field(1, "u")[:, 0]
    assert np.max(np.abs(u - of.u)) <= U_TOL


def test_set_and_extract_roundtrip_and_determinism(sphere_scene, sphere_hist):
    sc = sphere_scene
    runs = []
    for _ in range(2):
        with gdomain(sc.domain, sc.nbins) as dom:
            dom.set_histograms(0, sphere_hist)
            dom.solve(0, 50)
            runs.append({f: dom.field(0, f).copy() for f in ("u", "v", "p", "q", "ubar", "vbar")})
            np.testing.assert_array_equal(dom.histograms(0), sphere_hist)
            dom.reset(0)
            assert np.all(dom.field(0, "u") == 0)
    for f in runs[0]:
        np.testing.assert_array_equal(runs[0][f], runs[1][f])


def test_device_pointer_io(sphere_scene, sphere_hist):
    sc = sphere_scene
    with gdomain(sc.domain, sc.nbins) as dom:
        dom.set_histograms(0, torch.from_numpy(sphere_hist.astype(np.int32)).cuda())
        dom.solve(0, 10)
        out = torch.empty((dom.voxels(0), 1), dtype=torch.float32, device="cuda")
        dom.field(0, "u", out=out)
        host = dom.field(0, "u")
        np.testing.assert_array_equal(out.cpu().numpy(), host)


def test_kernel_forms_agree_on_a_large_ragged_domain():
    """Pipelined and one-brick-per-CTA forms on 6^3 bricks with holes and a frozen shell."""
    rng = np.random.default_rng(77)
    box = synth.dense_bricks(6)
    keep = rng.random(len(box)) > 0.15
    act = box[keep]
    frz = box[~keep][:10]
    fu = rng.uniform(-1, 1, (len(frz), 512)).astype(np.float32)
    fv = rng.normal(0, 0.1, (len(frz), 3, 512)).astype(np.float32)
    desc = synth.DomainDesc(np.zeros(3), 1.0, act, frozen=frz, frozen_u=fu, frozen_v=fv)
    hist = synth.random_histograms(rng, desc.nvox, 10, max_count=15)
    out = {}
    forms = ("paired", "pipelined", "one_brick_per_cta")
    for form in forms:
        with gdomain(desc, 10, iter_kernel=form) as dom:
            dom.set_histograms(0, hist)
            dom.solve(0, 37)
            out[form] = {f: dom.field(0, f) for f in ("u", "v", "p", "q", "ubar", "vbar")}
    for form in forms[1:]:
        for f in out["paired"]:
            np.testing.assert_allclose(out["paired"][f], out[form][f], atol=2e-6, rtol=0)
    orc = oracle.OracleLevel(desc, 10)
    orc.hist[:] = hist
    orc.iterate(37)
    assert np.max(np.abs(out["paired"]["u"][:, 0] - orc.u)) <= U_TOL
