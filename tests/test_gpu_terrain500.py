"""Parity after the full iteration count: the terrain workload's parameters at 128^3.

The dense terrain workload (Sec. 5's aerial scenes stood in for by a seeded terrain:
64 depth maps 512^2, 10 bins, alpha1 = 1, alpha0 = 2, tau = sigma = 0.2, lambda = 1)
is run for all of its 500 primal-dual iterations (Eq. 2-3, Sec. 3.2) on a 128^3 grid
(4096 bricks), with the paired kernel and its automatic run length, in the launch
configuration the benchmark uses.  The oracle runs the same 500 iterations in FP64 on
the whole grid (about 1e9 voxel-updates), so every voxel is compared.

Bars:
* histograms bit-exact (integer counts);
* u within 1e-4 everywhere (the benchmark spec's bound on the FP32 form after the
  configured iterations);
* v, p, q within 1e-3: they are not bounded by the benchmark spec; the stated bound
  is ten times u's, since v and the duals are unclamped and p, q live on the
  scale alpha1, alpha0 (1, 2) rather than u's [-1, 1];
* the zero level set: identical signs wherever both |u| > 1e-3, and crossings on
  voxel edges within 1e-3 h.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from _geom import dense_from_bricks, edge_crossings
from paper_2107_14790_b300 import tgv

pytestmark = pytest.mark.gpu
N = 128
ITERS = 500


@pytest.fixture(scope="module")
def runs():
    from paper_2107_14790_b300 import build
    build.build()
    sc = synth.terrain_scene(seed=1002, n=N, nmaps=64, res=512, nbins=10, iterations=ITERS, device="cuda")
    s = torch.cuda.Stream()
    depth = torch.from_numpy(np.stack(sc.depths)).cuda()
    with tgv.Domain([sc.domain], nbins=10, stream=s.cuda_stream) as dom:
        dom.accumulate(0, sc.cameras, depth)
        hist = dom.histograms(0)
        dom.solve(0, ITERS)
        gpu = {f: dom.field(0, f) for f in ("u", "v", "p", "q")}
        e_gpu = dom.energy(0)
    for storage in ("fx16", "fp16"):  # reduced-precision storage forms, same workload
        with tgv.Domain([sc.domain], nbins=10, storage=storage, stream=s.cuda_stream) as dom:
            dom.accumulate(0, sc.cameras, depth)
            dom.solve(0, ITERS)
            gpu["u_" + storage] = dom.field(0, "u")
            gpu["energy_" + storage] = dom.energy(0)
            gpu["state_" + storage] = {f: dom.field(0, f) for f in ("v", "p", "q")}
    orc = oracle.OracleLevel(sc.domain, 10)
    for c, d in zip(sc.cameras, sc.depths):
        orc.accumulate(c, d, 1)
    hist_orc = orc.hist.copy()
    orc.iterate(ITERS)
    return sc, hist, hist_orc, gpu, orc, e_gpu


def test_histograms_bit_exact(runs):
    _, hist, hist_orc, _, _, _ = runs
    assert hist.sum() > 10_000_000  # the maps see the terrain
    np.testing.assert_array_equal(hist, hist_orc)


def test_u_after_500_iterations_within_1e4(runs):
    _, _, _, gpu, orc, _ = runs
    du = np.abs(gpu["u"][:, 0] - orc.u)
    assert np.abs(orc.u).max() > 0.9  # a converging field, not a trivial one
    print(f"terrain 128^3, {ITERS} iterations: max |du| = {du.max():.3e}, rms {np.sqrt(np.mean(du ** 2)):.3e}")
    assert du.max() <= 1e-4, f"max |du| = {du.max():.3e} at voxel {int(du.argmax())}"


def test_v_p_q_after_500_iterations_within_1e3(runs):
    _, _, _, gpu, orc, _ = runs
    for f, want in (("v", orc.v), ("p", orc.p), ("q", orc.q)):
        d = np.abs(gpu[f] - want).max()
        print(f"terrain 128^3, {ITERS} iterations: max |d{f}| = {d:.3e}")
        assert np.abs(want).max() > 0.01
        assert d <= 1e-3, f"max |d{f}| = {d:.3e}"


def test_energy_and_gap_of_the_final_state(runs):
    """The GPU's energy / dual / gap of its own final state equals the oracle's evaluation of
    that same (FP32) state within 1e-6 relative, and the gap is certified and non-negative."""
    sc, hist, _, gpu, _, e_gpu = runs
    ev = oracle.OracleLevel(sc.domain, 10)
    ev.hist[:] = hist
    ev.u[:] = gpu["u"][:, 0]
    ev.v[:] = gpu["v"]
    ev.p[:] = gpu["p"]
    ev.q[:] = gpu["q"]
    e_orc = ev.energy()
    for k in range(3):
        assert abs(e_gpu[k] - e_orc[k]) <= 1e-6 * abs(e_orc[0]), (k, e_gpu[k], e_orc[k])
    assert e_gpu[3] == 1.0 and e_orc[3] == 1.0
    assert e_gpu[2] >= 0.0


def test_zero_level_set_agrees(runs):
    sc, _, _, gpu, orc, _ = runs
    h = sc.domain.h
    ug = dense_from_bricks(gpu["u"][:, 0].astype(np.float64), sc.domain.bricks, N)
    uo = dense_from_bricks(orc.u, sc.domain.bricks, N)
    both = (np.abs(ug) > 1e-3) & (np.abs(uo) > 1e-3)
    assert np.array_equal(np.sign(ug[both]), np.sign(uo[both]))
    mask = np.ones_like(ug, dtype=bool)
    pg, ig = edge_crossings(ug, mask, h, eps=1e-3)
    po, io = edge_crossings(uo, mask, h, eps=1e-3)
    assert len(pg) > 10_000
    # compare crossings on the edges both fields cross
    kg = {tuple(r): k for k, r in enumerate(ig.tolist())}
    common = [(kg[tuple(r)], k) for k, r in enumerate(io.tolist()) if tuple(r) in kg]
    assert len(common) >= 0.99 * len(po)
    a = np.array([c[0] for c in common])
    b = np.array([c[1] for c in common])
    disp = np.linalg.norm(pg[a] - po[b], axis=1).max() / h
    print(f"terrain 128^3, {ITERS} iterations: {len(common)} crossings, max displacement {disp:.2e} h")
    assert disp <= 1e-3, f"crossing displacement {disp:.2e} h"


def _crossing_displacement(sc, u_a, u_b, hist):
    """Max distance (in h) between the zero crossings of two fields on the voxel edges both
    cross with all four end values away from zero (|u| > 1e-3): over every such edge, and
    over the observed ones (both end voxels with >= 2 votes, the observed region of the
    sphere pin).  Returns (max all, count all, max observed, count observed)."""
    A = dense_from_bricks(u_a.astype(np.float64), sc.domain.bricks, N)
    B = dense_from_bricks(u_b.astype(np.float64), sc.domain.bricks, N)
    votes = dense_from_bricks(hist.sum(1).astype(np.float64), sc.domain.bricks, N)
    d_all, d_obs = [], []
    for ax in range(3):
        s0 = [slice(None)] * 3
        s1 = [slice(None)] * 3
        s0[ax] = slice(0, -1)
        s1[ax] = slice(1, None)
        aa, ab, ba, bb = A[tuple(s0)], A[tuple(s1)], B[tuple(s0)], B[tuple(s1)]
        ok = (np.abs(aa) > 1e-3) & (np.abs(ab) > 1e-3) & (np.abs(ba) > 1e-3) & (np.abs(bb) > 1e-3)
        both = ok & (np.sign(aa) != np.sign(ab)) & (np.sign(ba) != np.sign(bb))
        t = np.abs(aa[both] / (aa[both] - ab[both]) - ba[both] / (ba[both] - bb[both]))
        obs = ((votes[tuple(s0)] >= 2) & (votes[tuple(s1)] >= 2))[both]
        d_all.append(t)
        d_obs.append(t[obs])
    d_all, d_obs = np.concatenate(d_all), np.concatenate(d_obs)
    return d_all.max(), len(d_all), d_obs.max(), len(d_obs)


def test_fixed_point_duals_meet_the_stated_accuracy(runs):
    """16-bit storage (v, vbar FP16; p, q 16-bit fixed point scaled by alpha1, alpha0) after
    all 500 iterations against the FP64 oracle: the stated accuracy of the reduced forms,
    max |du| <= 5e-3 at every voxel and zero crossings within 0.05 h in the observed region
    (edges between voxels that >= 2 maps voted for; outside it no data places the surface
    and the iteration has near-flat directions, so crossings there are reported, not bounded).
    FP16 duals are reported beside it."""
    sc, hist, _, gpu, orc, _ = runs
    for storage in ("fx16", "fp16"):
        u = gpu["u_" + storage][:, 0]
        du = np.abs(u - orc.u)
        d_all, n_all, d_obs, n_obs = _crossing_displacement(sc, u, orc.u, hist)
        print(f"terrain 128^3, {ITERS} iterations, {storage} storage: max |du| = {du.max():.3e}, "
              f"rms {np.sqrt(np.mean(du ** 2)):.3e}; crossing displacement max {d_obs:.3e} h over {n_obs} "
              f"observed edges, {d_all:.3e} h over all {n_all}")
        if storage == "fx16":
            assert du.max() <= 5e-3
            assert n_obs > 50_000
            assert d_obs <= 0.05


def test_fixed_point_energy_of_its_state(runs):
    """The energy / gap the FX16 form reports is that of its own decoded state (oracle
    evaluation of the same values within 1e-6 relative)."""
    sc, hist, _, gpu, _, _ = runs
    st = gpu["state_fx16"]
    ev = oracle.OracleLevel(sc.domain, 10)
    ev.hist[:] = hist
    ev.u[:] = gpu["u_fx16"][:, 0]
    ev.v[:] = st["v"]
    ev.p[:] = st["p"]
    ev.q[:] = st["q"]
    e_orc = ev.energy()
    e_gpu = gpu["energy_fx16"]
    for k in range(3):
        assert abs(e_gpu[k] - e_orc[k]) <= 1e-6 * abs(e_orc[0]), (k, e_gpu[k], e_orc[k])
    # decoded duals are multiples of alpha / 32767 and stay in their balls
    assert np.abs(st["p"]).max() <= 1.0 + 1e-6 and np.abs(st["q"]).max() <= 2.0 + 1e-6
