"""Joint solve of all levels on the composite grid (Sec. 3.3, 2:1 faces) through the
C-ABI against the FP64 oracle of oracle/composite.py: |u_gpu - u_oracle| <= 1e-4
after the iterations (FP32 against FP64, as for the single-level solve)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle.composite import Composite as OracleComposite
from oracle.composite import leaf_keys as oracle_leaf_keys
from oracle.composite import treetop as oracle_treetop
from paper_2107_14790_b300 import tgv

pytestmark = pytest.mark.gpu
U_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2107_14790_b300 import build
    build.build()
    assert torch.cuda.is_available()
    tgv.lib()


def stream():
    return torch.cuda.current_stream().cuda_stream


def run_both(levels, hists, nbins, iters, u0=None):
    """levels: DomainDesc list (nested 2:1); hists: per-level (nvox, nbins) counts."""
    with tgv.Domain(levels, nbins=nbins, stream=stream()) as dom:
        for l, h in enumerate(hists):
            dom.set_histograms(l, h)
            if u0 is not None:
                dom.set_field(l, "u", u0[l].reshape(-1, 1).astype(np.float32))
        with tgv.Composite(dom) as comp:
            comp.solve(iters)
            ug = comp.u()
            per_level = [comp.level_leaves(l) for l in range(len(levels))]
            comp.scatter()
            scattered = [dom.field(l, "u")[:, 0] for l in range(len(levels))]
    orc = OracleComposite([L.bricks for L in levels], nbins)
    for l, h in enumerate(hists):
        orc.set_level_histograms(l, h)
        if u0 is not None:
            orc.set_level_field(l, u0[l].astype(np.float32))
    orc.iterate(iters)
    assert per_level == [len(s) for s in orc.level_slots]
    return ug, orc, scattered


def test_single_level_matches_the_oracle():
    rng = np.random.default_rng(1)
    box = synth.dense_bricks(4)
    desc = synth.DomainDesc(np.zeros(3), 1.0 / 32, box[rng.random(len(box)) > 0.2])
    hist = synth.random_histograms(rng, desc.nvox, 8, max_count=15)
    ug, orc, _ = run_both([desc], [hist], 8, 40)
    assert np.max(np.abs(ug - orc.u)) <= U_TOL


def test_two_levels_with_a_refined_block():
    rng = np.random.default_rng(2)
    coarse = synth.DomainDesc(np.zeros(3), 1.0 / 16, synth.dense_bricks(2))
    fine = synth.DomainDesc(np.zeros(3), 1.0 / 32, synth.dense_bricks(2, offset=(1, 1, 1)))
    hists = [synth.random_histograms(rng, L.nvox, 10, max_count=12) for L in (coarse, fine)]
    u0 = [rng.uniform(-1, 1, L.nvox) for L in (coarse, fine)]
    ug, orc, scattered = run_both([coarse, fine], hists, 10, 50, u0)
    assert np.max(np.abs(ug - orc.u)) <= U_TOL
    # scatter wrote every leaf's value into its level (and left refined voxels alone)
    o = 0
    for l, slots in enumerate(orc.level_slots):
        np.testing.assert_array_equal(scattered[l][slots], ug[o:o + len(slots)])
        o += len(slots)


def test_octree_levels_of_the_sphere(sphere_scene):
    """Three levels built from the sphere's maps (Eq. 4, band, 2:1 nesting), Alg. 1
    histograms on each level, joint iterations."""
    sc = sphere_scene
    dep = torch.from_numpy(np.stack(sc.depths)).cuda()
    lv, _ = tgv.tgv_octree_build(sc.cameras, dep, np.array([-0.5, -0.5, -0.5]), 2.0, 5, 7, 1, stream=stream())
    levels = [synth.DomainDesc(L.origin, L.h, L.bricks) for L in lv]
    hists = []
    for L in levels:
        o = oracle.OracleLevel(L, 8)
        for c, d in zip(sc.cameras, sc.depths):
            o.accumulate(c, d, 1)
        hists.append(o.hist.copy())
    with tgv.Domain(levels, nbins=8, stream=stream()) as dom:  # the library's own histograms agree
        for l in range(len(levels)):
            dom.accumulate(l, sc.cameras, dep)
            np.testing.assert_array_equal(dom.histograms(l), hists[l])
    ug, orc, _ = run_both(levels, hists, 8, 60)
    assert orc.n > 100_000
    assert np.max(np.abs(ug - orc.u)) <= U_TOL


def test_levels_that_are_not_nested_are_rejected():
    coarse = synth.DomainDesc(np.zeros(3), 1.0 / 16, synth.dense_bricks(1))
    fine = synth.DomainDesc(np.zeros(3), 1.0 / 32, np.array([[0, 0, 0]], np.int32))   # refines an octant
    finer = synth.DomainDesc(np.zeros(3), 1.0 / 64, np.array([[1, 0, 0]], np.int32))  # touches level 0 directly
    with tgv.Domain([coarse, fine, finer], nbins=8, stream=stream()) as dom:
        with pytest.raises(tgv.TgvError):
            tgv.Composite(dom)


def test_frozen_bricks_of_the_levels_are_ignored(sphere_scene):
    """Octree levels carry frozen shells for the level-by-level solve; the joint solve
    uses the active bricks only, so it equals the solve of the same levels without them."""
    sc = sphere_scene
    dep = torch.from_numpy(np.stack(sc.depths)).cuda()
    lv, _ = tgv.tgv_octree_build(sc.cameras, dep, np.array([-0.5, -0.5, -0.5]), 2.0, 5, 6, 1, stream=stream())
    bare = [synth.DomainDesc(L.origin, L.h, L.bricks) for L in lv]
    outs = []
    for levels in (lv, bare):
        with tgv.Domain(levels, nbins=8, stream=stream()) as dom:
            for l in range(len(levels)):
                dom.accumulate(l, sc.cameras, dep)
            with tgv.Composite(dom) as comp:
                comp.solve(15)
                outs.append(comp.u())
    np.testing.assert_array_equal(outs[0], outs[1])


# ---- treetop (Sec. 4.3) against the oracle's recursive definition

def gpu_treetops(levels, root_bits, Ns):
    with tgv.Domain(levels, nbins=8, stream=stream()) as dom:
        with tgv.Composite(dom) as comp:
            return [comp.treetop(root_bits, N) for N in Ns]


def same_treetop(got, want):
    for g, w, name in zip(got, want, ("depth", "code", "first", "last", "part")):
        np.testing.assert_array_equal(g, w, err_msg=name)


def test_treetop_two_levels_by_hand():
    levels = [synth.DomainDesc(np.zeros(3), 1.0 / 16, np.array([[0, 0, 0]], np.int32)),
              synth.DomainDesc(np.zeros(3), 1.0 / 32, np.array([[0, 0, 0]], np.int32))]
    keys = oracle_leaf_keys([L.bricks for L in levels])
    Ns = [600, 100, 961, 2]
    for N, got in zip(Ns, gpu_treetops(levels, 4, Ns)):
        same_treetop(got, oracle_treetop(keys, 2, 4, N))
    assert len(gpu_treetops(levels, 4, [100])[0][0]) == 15


def test_treetop_of_the_sphere_octree(sphere_scene):
    """Three octree levels (depths 5..7 of the root cube, voxel depth 10): parts of many
    sizes, from single cubes to the whole root."""
    sc = sphere_scene
    dep = torch.from_numpy(np.stack(sc.depths)).cuda()
    lv, _ = tgv.tgv_octree_build(sc.cameras, dep, np.array([-0.5, -0.5, -0.5]), 2.0, 5, 7, 1, stream=stream())
    levels = [synth.DomainDesc(L.origin, L.h, L.bricks) for L in lv]
    keys = oracle_leaf_keys([L.bricks for L in levels])
    assert len(keys) > 100_000
    Ns = [2, 37, 4096, 1 << 17, 1 << 30]
    for N, got in zip(Ns, gpu_treetops(levels, 10, Ns)):
        same_treetop(got, oracle_treetop(keys, 3, 10, N))


def test_treetop_argument_errors():
    inside = [synth.DomainDesc(np.zeros(3), 1.0 / 16, np.array([[0, 0, 0]], np.int32))]
    with tgv.Domain(inside, nbins=8, stream=stream()) as dom:
        with tgv.Composite(dom) as comp:
            assert tgv.lib().tgv_composite_treetop_parts(comp.handle, None, None, None, None, None) == 6  # STATE
            for root_bits, N in ((3, 1), (0, 10), (22, 10), (2, 10)):  # N < 2, bits out of range, cube outside
                with pytest.raises(tgv.TgvError):
                    comp.treetop(root_bits, N)
            d, c, f, l, p = comp.treetop(3, 10 ** 9)
            assert list(d) == [0] and list(f) == [0] and list(l) == [511] and np.all(p == 0)
    negative = [synth.DomainDesc(np.zeros(3), 1.0 / 16, np.array([[-1, 0, 0]], np.int32))]
    with tgv.Domain(negative, nbins=8, stream=stream()) as dom:
        with tgv.Composite(dom) as comp:
            with pytest.raises(tgv.TgvError):
                comp.treetop(10, 100)
