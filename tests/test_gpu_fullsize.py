"""Parity at the bench's full size and launch configuration, on sampled outputs.

The dense 256^3 terrain workload (64 maps 512^2, 10 bins; the paired kernel with
its automatic run length, as bench.py times it) is accumulated and iterated on
the GPU.  The oracle cannot run 16.8 M voxels, but it does not need to: after N
iterations a voxel depends only on voxels within 2N of it (each iteration reads
one neighbour in the dual step and one in the primal step), so a sub-domain of
bricks around a sample brick, with a margin of more than 2N voxels, reproduces
that brick exactly -- its own boundary (Neumann) only disturbs voxels within 2N
of it.  Bars: histograms of every sub-domain brick bit-exact; u of the sample
brick within 1e-4.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2107_14790_b300 import tgv

pytestmark = pytest.mark.gpu
ITERS = 20
MARGIN = 6  # bricks = 48 voxels > 2 * ITERS


@pytest.fixture(scope="module")
def terrain():
    return synth.terrain_scene(seed=1002, n=256, nmaps=64, res=512, nbins=10, iterations=500, device="cuda")


@pytest.fixture(scope="module")
def gpu_run(terrain):
    from paper_2107_14790_b300 import build
    build.build()
    sc = terrain
    with tgv.Domain([sc.domain], nbins=10, stream=torch.cuda.current_stream().cuda_stream) as dom:
        dom.accumulate(0, sc.cameras, torch.from_numpy(np.stack(sc.depths)).cuda())
        hist = dom.histograms(0)
        dom.solve(0, ITERS)
        u = dom.field(0, "u")[:, 0]
    return hist, u


def surface_brick(sc, gx, gy):
    """Brick (gx, gy, z) holding the terrain surface above brick column (gx, gy)."""
    t = sc.meta["terrain"]
    x, y = (8 * gx + 4) / 256, (8 * gy + 4) / 256
    z = float(t.height(np.array([x]), np.array([y]))[0])
    return np.array([gx, gy, int(z * 32)])


@pytest.mark.parametrize("col", [(16, 16), (5, 27)])
def test_sampled_brick_matches_the_oracle(terrain, gpu_run, col):
    sc = terrain
    hist, u = gpu_run
    centre = surface_brick(sc, *col)
    all_b = sc.domain.bricks
    lo, hi = centre - MARGIN, centre + MARGIN
    sel = np.all((all_b >= lo) & (all_b <= hi), axis=1)
    idx = np.nonzero(sel)[0]
    sub = synth.DomainDesc(sc.domain.origin, sc.domain.h, all_b[idx])
    orc = oracle.OracleLevel(sub, 10)
    for c, d in zip(sc.cameras, sc.depths):
        orc.accumulate(c, d, 1)
    rows = (idx[:, None] * 512 + np.arange(512)[None, :]).ravel()
    np.testing.assert_array_equal(hist[rows], orc.hist)
    orc.iterate(ITERS)
    k = int(np.nonzero(np.all(all_b[idx] == centre, axis=1))[0][0])
    b = int(idx[k])
    got = u[512 * b:512 * (b + 1)]
    want = orc.u[512 * k:512 * (k + 1)]
    assert np.abs(want).max() > 0.05  # the sample sees the surface
    assert np.max(np.abs(got - want)) <= 1e-4
