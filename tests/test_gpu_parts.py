"""A level solved part by part (Sec. 4.3 treetop parts; Sec. 4.5: a part's cubes are the set
A, its neighbouring cubes the set B whose indicator stays at the parent level's values).

Coarse-to-fine on the sphere scene: level 0 (32^3) is solved, level 1 (64^3) starts from
its prolongation.  The treetop of level 1's cubes (parts of fewer than 5000 cubes) splits
the level into parts; each part becomes a chunk whose border bricks are frozen to the
prolonged field, and all parts run together in one persistent launch
(tgv_solve_chunks).  Checks:
* every part equals the oracle's run of that part (same frozen border) within 1e-4;
* the parts' results, scattered back into the level, mesh (Sec. 4.6) without seams: each
  part meshed with its border bricks frozen to the scattered field gives the whole
  level's triangles, none twice, and the whole mesh is consistently oriented.
The per-part and whole-level solves are timed and their difference reported.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2107_14790_b300 import tgv
from paper_2107_14790_b300.batching import part_chunks, union_level
from tests.test_oracle_mesh import directed_edges

pytestmark = pytest.mark.gpu
ITERS = 80


@pytest.fixture(scope="module")
def setup():
    from paper_2107_14790_b300 import build
    build.build()
    sc = synth.sphere_scene()  # 64^3, 16 maps 128^2, 8 bins
    fine = sc.domain
    coarse = synth.DomainDesc(np.zeros(3), 2 * fine.h, synth.dense_bricks(4))
    s = torch.cuda.Stream()
    depth = torch.from_numpy(np.stack(sc.depths)).cuda()
    with tgv.Domain([coarse, fine], nbins=8, stream=s.cuda_stream) as dom:
        dom.accumulate(0, sc.cameras, depth)
        dom.accumulate(1, sc.cameras, depth)
        dom.solve(0, 60)
        dom.prolong(0)
        u0, v0 = dom.field(1, "u")[:, 0], dom.field(1, "v")
        hist = dom.histograms(1)
    # treetop of the fine level's cubes (root 64^3 voxels = 2^6)
    with tgv.Domain([fine], nbins=8, stream=s.cuda_stream) as dom:
        dom.set_histograms(0, hist)
        with tgv.Composite(dom) as comp:
            _, _, _, _, leaf_part = comp.treetop(6, 5000)
    brick_part = leaf_part.reshape(-1, 512)
    assert np.all(brick_part == brick_part[:, :1])  # parts hold whole bricks (5000 > 512)
    brick_part = brick_part[:, 0]
    parts = part_chunks(fine, brick_part, u0, v0)
    return sc, fine, hist, u0, v0, parts, s


def test_treetop_gives_several_parts(setup):
    _, fine, _, _, _, parts, _ = setup
    assert len(parts) >= 8
    assert sum(p.nbricks for p in parts) == fine.nbricks
    assert all(p.nvox < 5000 for p in parts) and max(p.nbricks for p in parts) == 8


@pytest.fixture(scope="module")
def solved(setup):
    sc, fine, hist, u0, v0, parts, s = setup
    U = union_level(parts)
    rows = np.concatenate([(p.level_bricks[:, None] * 512 + np.arange(512)).ravel() for p in parts])
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    with tgv.Domain([U], nbins=8, stream=s.cuda_stream) as dom:
        dom.set_histograms(0, hist[rows])
        for f, val in (("u", u0[rows, None]), ("ubar", u0[rows, None]), ("v", v0[rows]), ("vbar", v0[rows])):
            dom.set_field(0, f, val)
        ev[0].record(s)
        dom.solve_chunks(0, U.first, [ITERS] * len(parts))
        ev[1].record(s)
        u_parts = dom.field(0, "u")[:, 0]
    u_level = np.empty_like(u0)
    u_level[rows] = u_parts
    # the whole level from the same start (no frozen borders between parts)
    with tgv.Domain([fine], nbins=8, stream=s.cuda_stream) as dom:
        dom.set_histograms(0, hist)
        for f, val in (("u", u0[:, None]), ("ubar", u0[:, None]), ("v", v0), ("vbar", v0)):
            dom.set_field(0, f, val)
        ev[2].record(s)
        dom.solve(0, ITERS)
        ev[3].record(s)
        u_whole = dom.field(0, "u")[:, 0]
    s.synchronize()
    print(f"per-part solve of {len(parts)} parts: {ev[0].elapsed_time(ev[1]):.2f} ms; whole level "
          f"{ev[2].elapsed_time(ev[3]):.2f} ms; max |u_parts - u_whole| = {np.abs(u_level - u_whole).max():.3e}")
    return U, u_parts, u_level


def test_each_part_equals_the_oracle_run_of_that_part(setup, solved):
    _, _, hist, u0, v0, parts, _ = setup
    U, u_parts, _ = solved
    for k in range(0, len(parts), max(1, len(parts) // 8)):  # every eighth part
        p = parts[k]
        rows = (p.level_bricks[:, None] * 512 + np.arange(512)).ravel()
        o = oracle.OracleLevel(p, 8)
        o.hist[:] = hist[rows]
        o.u[:] = u0[rows]
        o.ubar[:] = u0[rows]
        o.v[:] = v0[rows]
        o.vbar[:] = v0[rows]
        o.iterate(ITERS)
        a, b = U.ranges[k]
        err = np.abs(u_parts[512 * a:512 * b] - o.u).max()
        assert err <= 1e-4, f"part {k}: max |du| = {err:.2e}"


def test_parts_mesh_without_seams(setup, solved):
    _, fine, _, _, _, parts, s = setup
    _, _, u_level = solved

    def mesh(desc, u_active):
        with tgv.Domain([desc], nbins=8, stream=s.cuda_stream) as dom:
            dom.set_field(0, "u", u_active.reshape(-1, 1).astype(np.float32))
            return dom.mesh(0)

    def triangles(V, T):
        return [V[t].tobytes() for t in T]

    V, T = mesh(fine, u_level)
    whole = triangles(V, T)
    assert len(T) > 1000 and len(set(whole)) == len(whole)
    # consistently oriented and manifold: no directed edge twice (the zero set may meet the
    # level's outer boundary where no map sees the scene, so it need not be closed)
    assert max(directed_edges(T).values()) == 1
    seen = []
    u_b = u_level.reshape(-1, 512)
    index = {tuple(x): i for i, x in enumerate(np.asarray(fine.bricks).tolist())}
    for p in parts:
        frz = p.frozen
        fu = None if frz is None else u_b[[index[tuple(x)] for x in frz.tolist()]]
        d = synth.DomainDesc(fine.origin, fine.h, p.bricks, frozen=frz, frozen_u=fu)
        Vp, Tp = mesh(d, u_b[p.level_bricks])
        seen += triangles(Vp, Tp)
    assert len(seen) == len(set(seen))  # no seam triangle made twice
    assert set(seen) == set(whole)  # none missing
