"""Sparse three-level domain (terrain at level 0, a blob refined 4x at level 2, a level-1
transition shell), coarse-to-fine (Sec. 4.5): histograms per level bit-exact, and u after
the level-by-level solve with prolongation and frozen set-B shells within 1e-4 of the
FP64 oracle; 16-bit storage error stated."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2107_14790_b300 import tgv

pytestmark = pytest.mark.gpu
ITERS = 40


@pytest.fixture(scope="module")
def scene():
    from paper_2107_14790_b300 import build
    build.build()
    return synth.multilevel_scene(n0=64, blob_radius_vox=6, nmaps_aerial=12, nmaps_ring=8, res=64,
                                  iterations=ITERS, device="cpu")


@pytest.fixture(scope="module")
def oracle_run(scene):
    L, nb = scene["levels"], scene["nbins"]
    orcs = [oracle.OracleLevel(d, nb) for d in L]
    for o in orcs:
        for cam, dep in zip(scene["cameras"], scene["depths"]):
            o.accumulate(cam, dep, 1)
    hists = [o.hist.copy() for o in orcs]
    orcs[0].iterate(ITERS)
    for l in (1, 2):
        orcs[l].prolong_from(orcs[l - 1])
        oracle.prolong_frozen(orcs[l], orcs[l - 1])
        orcs[l].iterate(ITERS)
    return hists, [o.u.copy() for o in orcs]


def gpu_run(scene, storage="fp32", form="paired"):
    L, nb = scene["levels"], scene["nbins"]
    depth = torch.from_numpy(np.stack(scene["depths"])).cuda()
    s = torch.cuda.Stream()
    with tgv.Domain(L, nbins=nb, storage=storage, stream=s.cuda_stream, iter_kernel=form) as dom:
        hists = []
        for l in range(3):
            dom.accumulate(l, scene["cameras"], depth)
            hists.append(dom.histograms(l))
        dom.solve(0, ITERS)
        for l in (1, 2):
            dom.prolong(l - 1)
            dom.solve(l, ITERS)
        us = [dom.field(l, "u")[:, 0] for l in range(3)]
        e = dom.energy(2)
    return hists, us, e


@pytest.mark.parametrize("form", ["paired", "one_brick_per_cta"])
def test_multilevel_matches_oracle(scene, oracle_run, form):
    ref_h, ref_u = oracle_run
    hists, us, e = gpu_run(scene, form=form)
    for l in range(3):
        np.testing.assert_array_equal(hists[l], ref_h[l])
        assert hists[l].sum() > 0
        err = np.max(np.abs(us[l] - ref_u[l]))
        assert err <= 1e-4, (l, err)
    assert e[3] == 1.0 and e[2] >= 0.0


def test_multilevel_reduced_precision_error(scene, oracle_run):
    _, ref_u = oracle_run
    errs = {}
    for storage in ("fx16", "fp16", "bf16"):
        _, us, _ = gpu_run(scene, storage=storage)
        errs[storage] = max(float(np.max(np.abs(us[l] - ref_u[l]))) for l in range(3))
    print("multilevel |du|_inf vs FP64 oracle:", errs)
    assert errs["fx16"] <= 5e-3
    assert errs["fp16"] <= 5e-3
    assert errs["bf16"] <= 5e-2
